// Launchers of the hot-path passes for one precision (included by gfp_k64.cu and gfp_k32.cu).
#pragma once
#include "gfp_kernels.cuh"

namespace gfp {

template <typename R>
cudaError_t Passes<R>::setup() {
  const int mx = 220 * 1024;  // below the 227 KB opt-in limit, leaving room for static shared memory
  cudaError_t e = cudaFuncSetAttribute(pass_x_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_z_gamma_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

template <typename R>
void Passes<R>::pass_x(cudaStream_t s, const LaunchCfg& lc, T* spec, R* eps, const R* lam, const R* mu, const T* tw,
                       const FftPlan& plan, const Dims& d, int flags, const float* corr, const double* corr_mean,
                       const SolveState* st) {
  const long long nlines = (long long)d.n2 * d.n3;
  const unsigned blocks = (unsigned)((nlines + lc.x_lines - 1) / lc.x_lines);
  const size_t sm = sizeof(T) * (size_t)(d.n1 + 6 * lc.x_lines * d.n1);
  pass_x_kernel<R><<<blocks, lc.x_threads, sm, s>>>(spec, eps, lam, mu, tw, plan, d, lc.x_lines, flags, corr,
                                                     corr_mean, st);
}

template <typename R>
void Passes<R>::pass_y(cudaStream_t s, const LaunchCfg& lc, bool inverse, T* spec, const T* tw, const FftPlan& plan,
                       const Dims& d, const SolveState* st) {
  dim3 grid((d.n1h + lc.y_cols - 1) / lc.y_cols, d.n3, 6);
  const size_t sm = sizeof(T) * (size_t)(d.n2 + 2 * lc.y_cols * d.n2);
  if (inverse) pass_y_kernel<R, true><<<grid, lc.y_threads, sm, s>>>(spec, tw, plan, d, lc.y_cols, st);
  else pass_y_kernel<R, false><<<grid, lc.y_threads, sm, s>>>(spec, tw, plan, d, lc.y_cols, st);
}

template <typename R>
void Passes<R>::pass_z(cudaStream_t s, const LaunchCfg& lc, T* spec, const T* tw, const FftPlan& plan, const Dims& d,
                       const GammaParams<R>& gp, double* partials, SolveState* st, int mode, float2* vsrc) {
  dim3 grid((d.n1h + lc.z_cols - 1) / lc.z_cols, d.n2, 1);
  const size_t sm = sizeof(T) * (size_t)(d.n3 + 12 * lc.z_cols * d.n3);
  pass_z_gamma_kernel<R><<<grid, lc.z_threads, sm, s>>>(spec, tw, plan, d, lc.z_cols, gp, partials, st, mode, vsrc);
}

}  // namespace gfp
