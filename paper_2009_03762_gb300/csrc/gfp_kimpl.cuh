// Launchers of the hot-path passes for one precision (included by gfp_k64.cu and gfp_k32.cu).
// Grid sizes with a compile-time FFT plan (CPlan) use the register-resident kernels of
// gfp_fftc.cuh; every other 2^a 3^b size uses the generic shared-memory Stockham kernels.
#pragma once
#include "gfp_tma.cuh"

namespace gfp {

template <typename R>
cudaError_t Passes<R>::setup() {
  const int mx = 220 * 1024;  // below the 227 KB opt-in limit, leaving room for static shared memory
  cudaError_t e = cudaFuncSetAttribute(pass_x_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_z_gamma_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
#define GFP_SET(N)                                                                                          \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_x_c_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_x_a_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_c_kernel<R, N, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_c_kernel<R, N, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_c_kernel<R, N, false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_y_c_kernel<R, N, true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_z_c_kernel<R, N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_z_c_kernel<R, N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if constexpr (ZBound<R, N>::small)                                                                  \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_z_c2_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  GFP_FOR_CSIZES(GFP_SET)
#undef GFP_SET
#define GFP_SET_TMA(N) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_z_tma_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if constexpr (sizeof(R) == 4 && SPlanOk<N>::ok)                                                     \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_z_s_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  GFP_FOR_CSIZES(GFP_SET_TMA)
#undef GFP_SET_TMA
  return e;
}

// Persistent-grid size of the TMA z-pass: resident CTAs per SM x SMs (cached per configuration).
template <typename R, int N>
inline int tma_grid(int threads, size_t smem) {
  static int sms = 0;
  static int cached_threads = -1, cached_blocks = 0;
  static size_t cached_smem = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (threads != cached_threads || smem != cached_smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_z_tma_kernel<R, N>, threads, smem);
    cached_threads = threads;
    cached_smem = smem;
    cached_blocks = nb > 0 ? nb : 1;
  }
  return sms * cached_blocks;
}

// shared memory of the compile-time x-pass for `lines` x-lines per CTA: twiddles and 3 padded
// complex lines per x-line
template <typename R, int N> inline size_t cx_smem_bytes(int lines) {
  return sizeof(typename C<R>::T) * (size_t)(N + 3 * lines * (N + N / 16));
}
// lines per CTA of the compile-time x-pass: at most 512 threads (3 pair-lines x T each) and at most
// 200 KB of shared memory
template <typename R, int N> inline int cx_lines_max() {
  const int by_threads = 512 / (3 * CPlan<N>::T);
  int by_smem = 16;
  while (by_smem > 1 && cx_smem_bytes<R, N>(by_smem) > 200 * 1024) --by_smem;
  return std::max(1, std::min(16, std::min(by_threads, by_smem)));
}

template <typename R, int N>
inline void launch_x_c(cudaStream_t s, int want_lines, int async, typename C<R>::T* spec, R* eps, const R* lam,
                       const R* mu, const typename C<R>::T* tw, const Dims& d, int flags, const float* corr,
                       const double* corr_mean, const PolarParams& pp, const SolveState* st) {
  typedef typename C<R>::T T;
  if (async && !(flags & (PX_POLAR | PX_STRAIN | PX_OUTPUT | PX_DRES)) && !pp.estar) {
    int lines = want_lines > 0 ? want_lines : 2;
    lines = std::min(lines, 512 / (3 * CPlan<N>::T));
    while (lines > 1 && xa_smem_bytes<R, N>(lines) > 200 * 1024) --lines;
    const long long nlines = (long long)d.n2 * d.n3;
    const unsigned blocks = (unsigned)((nlines + lines - 1) / lines);
    pass_x_a_kernel<R, N><<<blocks, 3 * lines * CPlan<N>::T, xa_smem_bytes<R, N>(lines), s>>>(
        spec, eps, lam, mu, tw, d, lines, flags, corr, corr_mean, st);
    return;
  }
  const int lines = want_lines > 0 ? std::min(want_lines, cx_lines_max<R, N>()) : cx_lines_max<R, N>();
  const long long nlines = (long long)d.n2 * d.n3;
  const unsigned blocks = (unsigned)((nlines + lines - 1) / lines);
  const size_t sm = cx_smem_bytes<R, N>(lines);
  pass_x_c_kernel<R, N><<<blocks, 3 * lines * CPlan<N>::T, sm, s>>>(spec, eps, lam, mu, tw, d, lines, flags, corr,
                                                                     corr_mean, pp, st);
}

template <typename R>
void Passes<R>::pass_x(cudaStream_t s, const LaunchCfg& lc, T* spec, R* eps, const R* lam, const R* mu, const T* tw,
                       const FftPlan& plan, const Dims& d, int flags, const float* corr, const double* corr_mean,
                       const SolveState* st, const PolarParams* ppp) {
  PolarParams pp;
  if (ppp) pp = *ppp;
  else {
    for (int c = 0; c < 6; ++c) pp.E[c] = 0;
    pp.lam_h = pp.mu_h = 0;
    pp.partials = nullptr;
    pp.estar = nullptr;
  }
  switch (d.n1) {
#define GFP_CASE(N) \
    case N: launch_x_c<R, N>(s, lc.cx_lines, lc.x_async, spec, eps, lam, mu, tw, d, flags, corr, corr_mean, pp, st); return;
    GFP_FOR_CSIZES(GFP_CASE)
#undef GFP_CASE
    default: break;
  }
  const long long nlines = (long long)d.n2 * d.n3;
  const unsigned blocks = (unsigned)((nlines + lc.x_lines - 1) / lc.x_lines);
  const size_t sm = sizeof(T) * (size_t)(d.n1 + 6 * lc.x_lines * d.n1);
  pass_x_kernel<R><<<blocks, lc.x_threads, sm, s>>>(spec, eps, lam, mu, tw, plan, d, lc.x_lines, flags, corr,
                                                     corr_mean, pp, st);
}

template <typename R>
void Passes<R>::pass_y(cudaStream_t s, const LaunchCfg& lc, bool inverse, T* spec, const T* tw, const FftPlan& plan,
                       const Dims& d, const SolveState* st, int comps) {
  dim3 grid((d.n1h + lc.y_cols - 1) / lc.y_cols, d.n3, comps);
  switch (d.n2) {
#define GFP_CASE(N)                                                                                 \
    case N: {                                                                                       \
      const size_t smc = sizeof(T) * (size_t)(N + N * lc.y_cols);                                   \
      const int th = lc.y_cols * CPlan<N>::T;                                                       \
      if (lc.y_cols == 16) {                                                                        \
        if (inverse) pass_y_c_kernel<R, N, true, 16><<<grid, th, smc, s>>>(spec, tw, d, 16, st);    \
        else pass_y_c_kernel<R, N, false, 16><<<grid, th, smc, s>>>(spec, tw, d, 16, st);           \
      } else if (inverse) pass_y_c_kernel<R, N, true, 0><<<grid, th, smc, s>>>(spec, tw, d, lc.y_cols, st); \
      else pass_y_c_kernel<R, N, false, 0><<<grid, th, smc, s>>>(spec, tw, d, lc.y_cols, st);       \
      return;                                                                                       \
    }
    GFP_FOR_CSIZES(GFP_CASE)
#undef GFP_CASE
    default: break;
  }
  const size_t sm = sizeof(T) * (size_t)(d.n2 + 2 * lc.y_cols * d.n2);
  if (inverse) pass_y_kernel<R, true><<<grid, lc.y_threads, sm, s>>>(spec, tw, plan, d, lc.y_cols, st);
  else pass_y_kernel<R, false><<<grid, lc.y_threads, sm, s>>>(spec, tw, plan, d, lc.y_cols, st);
}

template <typename R>
void Passes<R>::pass_z(cudaStream_t s, const LaunchCfg& lc, T* spec, const T* tw, const FftPlan& plan, const Dims& d,
                       const GammaParams<R>& gp, double* partials, SolveState* st, int mode, float2* vsrc) {
  const int ntx = (d.n1h + lc.z_cols - 1) / lc.z_cols;
  dim3 grid(ntx, d.n2, 1);
  switch (d.n3) {
#define GFP_CASE(N)                                                                                           \
    case N: {                                                                                                 \
      const int th = 6 * lc.z_cols * CPlan<N>::T;                                                             \
      const size_t smt = sizeof(T) * (size_t)(N + 12 * N * lc.z_cols) + 128;                                 \
      if constexpr (sizeof(R) == 4 && SPlanOk<N>::ok) {                                                       \
        if (mode == PZ_INNER && lc.z_tma && lc.ztmap && lc.z_cols == 8 && !gp.nyq_avg) {                      \
          pass_z_s_kernel<N><<<grid, 24 * CPlan<N>::T, zs_smem_bytes<N>(), s>>>(                              \
              *reinterpret_cast<const CUtensorMap*>(lc.ztmap), reinterpret_cast<const float2*>(tw), d,        \
              *reinterpret_cast<const GammaParams<float>*>(&gp), partials, st, vsrc);                         \
          return;                                                                                             \
        }                                                                                                     \
      }                                                                                                       \
      if (mode != PZ_DGO && mode != PZ_DISP && lc.z_tma && lc.ztmap && (lc.z_cols * sizeof(T)) % 16 == 0 && th <= 384 &&        \
          smt <= 220 * 1024) {                    \
        const int ntiles = ntx * d.n2;                                                                        \
        const int gsz = std::min(ntiles, tma_grid<R, N>(th, smt));                                            \
        pass_z_tma_kernel<R, N><<<gsz, th, smt, s>>>(*reinterpret_cast<const CUtensorMap*>(lc.ztmap), spec, tw, \
                                                      d, lc.z_cols, ntx, gp, partials, st, mode, vsrc,        \
                                                      g_inject_tma_timeout);                                 \
        return;                                                                                               \
      }                                                                                                       \
      const size_t smc = sizeof(T) * (size_t)(2 * N + 7 * N * lc.z_cols) +                                   \
                         (mode == PZ_INNER && (lc.z_cols == 2 || lc.z_cols == 4 || lc.z_cols == 8)                    \
                              ? sizeof(float2) * 3 * N * lc.z_cols : 0);                                      \
      if constexpr (ZBound<R, N>::small) {                                                                    \
        if (lc.z_cols == 8) {                                                                                 \
          const size_t sm2 = sizeof(T) * (size_t)(2 * N + 48 * N);                                            \
          pass_z_c2_kernel<R, N><<<grid, 24 * CPlan<N>::T, sm2, s>>>(spec, tw, d, gp, partials, st, mode, vsrc); \
          return;                                                                                             \
        }                                                                                                     \
      }                                                                                                       \
      if (lc.z_cols == 4)                                                                                     \
        pass_z_c_kernel<R, N, 4><<<grid, th, smc, s>>>(spec, tw, d, 4, gp, partials, st, mode, vsrc);         \
      else                                                                                                    \
        pass_z_c_kernel<R, N, 0><<<grid, th, smc, s>>>(spec, tw, d, lc.z_cols, gp, partials, st, mode, vsrc); \
      return;                                                                                                 \
    }
    GFP_FOR_CSIZES(GFP_CASE)
#undef GFP_CASE
    default: break;
  }
  const size_t sm = sizeof(T) * (size_t)(d.n3 + 12 * lc.z_cols * d.n3);
  pass_z_gamma_kernel<R><<<grid, lc.z_threads, sm, s>>>(spec, tw, plan, d, lc.z_cols, gp, partials, st, mode, vsrc);
}

}  // namespace gfp

namespace gfp {
// Whether the z-pass accepts a tile of `cols` k1 columns for this length and precision: any width
// up to the limit of the one-line-per-thread kernel, and 8 where the two-lines-per-thread kernel runs.
template <typename R> bool cz_cols_ok(int n3, int cols) {
  if (cols < 1) return false;
  switch (n3) {
#define GFP_CASE(N)                                                                 \
    case N:                                                                         \
      return 6 * cols * CPlan<N>::T <= ZBound<R, N>::threads || (cols == 8 && ZBound<R, N>::small);
    GFP_FOR_CSIZES(GFP_CASE)
#undef GFP_CASE
    default: return cols <= 64;
  }
}
// Whether a TMA-fed z-pass can serve a tile of `cols` columns: the persistent kernel up to 384 threads,
// and the 8-column warp-shuffle kernel for FP32 square plans.
template <typename R> bool cz_tma_ok(int n3, int cols) {
  switch (n3) {
#define GFP_CASE(N) \
    case N: return (cols >= 1 && 6 * cols * CPlan<N>::T <= 384) || (cols == 8 && sizeof(R) == 4 && SPlanOk<N>::ok);
    GFP_FOR_CSIZES(GFP_CASE)
#undef GFP_CASE
    default: return false;
  }
}
template <typename R> int cy_cols_max(int n2) {
  switch (n2) {
#define GFP_CASE(N) \
    case N: return std::max(1, 512 / CPlan<N>::T);
    GFP_FOR_CSIZES(GFP_CASE)
#undef GFP_CASE
    default: return 64;
  }
}
}  // namespace gfp
