// Hot-path kernels of one fixed-point iteration (Sec. 5.2 Algorithm T-3D in strain form):
//
//   pass_x      : inverse x-transform of the previous increment -> eps += d_eps ->
//                 sigma = lambda tr(eps) I + 2 mu eps (Sec. 5.1) -> forward real-to-complex x-transform
//   pass_y      : complex transform along x2 (forward, or inverse)
//   pass_z_gamma: forward transform along x3 -> residual partial |T kt|^2 and T(0) ->
//                 Delta E = -Gamma0(kt) T / N (eq. EquMecFunGre3D in its real isotropic form) ->
//                 inverse transform along x3
//   reduce_eta  : eta = ||T q^b|| / ||T(0)||_F and the convergence decision (device flag)
//
// Data layout (HBM): real fields [c][i3][i2][i1]; the half spectrum [c][k3][k2][k1] with
// k1 in [0, n1/2] and a row pitch P >= n1/2 + 1 (rows start on 64-byte boundaries).
#pragma once
#include "gfp_fft.cuh"

namespace gfp {

enum { OP_F = 0, OP_CD = 1, OP_ACD = 2, OP_HC = 3, OP_AHC = 4, OP_AFB_R = 5, OP_DGO = 6 };

struct Dims {
  int n1, n2, n3;
  int n1h;      // n1/2 + 1
  int P;        // spectrum row pitch (complex elements)
  long long N;  // n1 n2 n3
  long long S;  // spectrum component stride = n3 n2 P
  // Spectrum rows are ordered (k3, k2), k2 fastest, like the real-space x-lines li = i3 n2 + i2: the
  // x-pass then reads and writes whole runs of consecutive rows.  (The transposed order (k2, k3)
  // makes the Green pass's z-columns contiguous but slows the x-pass by more than it gains.)
  __host__ __device__ long long row(int k3, int k2) const { return (long long)k3 * n2 + k2; }
  __host__ __device__ long long xrow(long long li) const { return li; }
  __host__ __device__ int ystride() const { return P; }                        // elements between k2 and k2 + 1
  __host__ __device__ long long zstride() const { return (long long)n2 * P; }  // elements between k3 and k3 + 1
};

// SolveState::done values besides 0 (running): 1 converged, 2 maxit, 3 diverged, DONE_TIMEOUT when a
// bounded device-side wait gave up; DONE_HELD (batched solves only) holds a slot's FP64 outer pass
// for one window while its inner iterations continue.
enum { DONE_TIMEOUT = 4, DONE_HELD = 5 };

// Device-side solver state; one per solve, reset by the host before the first iteration.
struct SolveState {
  int it;          // iterations done
  int done;        // 0 running, 1 converged, 2 maxit reached, 3 diverged
  int maxit;
  int growth;      // consecutive iterations with growing eta
  int restart;     // 1: the next x-pass starts from a zero strain correction (PX_ZERO); reduce_eta clears it
  double tol;
  double eta;      // last residual
  double eta_min;
  double T0[6];    // last unnormalised T(k = 0), tensor components
  double crit;     // stop_rule 1: the increment criterion of the last iteration
};

// Per-axis wave-vector tables: kt_r = A_r[i_r] B_s[i_s] B_t[i_t] ((s, t) the other two axes),
// indexed by storage index i_r in 0..n_r-1 (kappa = i_r, or i_r - n_r past the middle; the Nyquist
// index n_r/2 of an even axis is kappa = -n_r/2 as in the paper's index range).
template <typename R>
struct GammaParams {
  const R* A[3];
  const R* B[3];
  R c_mu;              // 1 / (2 mu_H)
  R c_lm;              // (lambda_H + mu_H) / (mu_H (lambda_H + 2 mu_H))
  R invN;
  int nyq_avg;         // average Gamma over the Hermitian partner on Nyquist planes (F, HC)
  int half_shift;      // displacement recovery: q^a = e^{i (th1 + th2 + th3)/2} i kt (AFB/R), else i kt
  const double* dgo;   // DGO: 21 Mandel entries per half-spectrum point, [21][k3][k2][P] (mode PZ_DGO)
  // stop_rule 1 (FP64, PZ_GAMMA): the previous iteration's T kt per point, [3][k3][k2][P], updated in
  // place, and 1 / mu_H and (lambda_H + mu_H) / (lambda_H + 2 mu_H) of G_iso; null when not in use
  double2* vprev = nullptr;
  double inv_mu = 0.0, c_g = 0.0;
  double* cpart = nullptr;  // per-CTA sums of the criterion (same indexing as the residual partials)
};

// Increment criterion of the paper's stopping rule at one half-spectrum point: with q^a = a i kt and
// q^b = b i kt (|a| = |b| = 1, the pairings CD, ACD, AHC, AFB/R), the displacement increment of
// Algorithm T/P is (i / a) G_iso(kt) (T kt) with G_iso(kt) = [I - c kt kt / |kt|^2] / (mu_H |kt|^2), so
// |du_it - du_(it-1)| = |G_iso(kt) (v - v_prev)| for v = T kt.  Returns that norm (unnormalised
// transform) and stores v as the next iteration's v_prev.
template <typename R, typename T>
__device__ __forceinline__ R incr_point(T v1, T v2, T v3, R k1, R k2, R k3, const GammaParams<R>& gp, long long vi,
                                        long long S) {
  double2* pv = gp.vprev;
  const double2 p1 = pv[vi], p2 = pv[S + vi], p3 = pv[2 * S + vi];
  pv[vi] = make_double2((double)v1.x, (double)v1.y);
  pv[S + vi] = make_double2((double)v2.x, (double)v2.y);
  pv[2 * S + vi] = make_double2((double)v3.x, (double)v3.y);
  const R s = k1 * k1 + k2 * k2 + k3 * k3;
  if (s == (R)0) return (R)0;
  T w1, w2, w3;
  w1.x = v1.x - (R)p1.x; w1.y = v1.y - (R)p1.y;
  w2.x = v2.x - (R)p2.x; w2.y = v2.y - (R)p2.y;
  w3.x = v3.x - (R)p3.x; w3.y = v3.y - (R)p3.y;
  const R f = (R)gp.c_g / s;
  T kw; kw.x = k1 * w1.x + k2 * w2.x + k3 * w3.x; kw.y = k1 * w1.y + k2 * w2.y + k3 * w3.y;
  T g1, g2, g3;
  g1.x = w1.x - f * k1 * kw.x; g1.y = w1.y - f * k1 * kw.y;
  g2.x = w2.x - f * k2 * kw.x; g2.y = w2.y - f * k2 * kw.y;
  g3.x = w3.x - f * k3 * kw.x; g3.y = w3.y - f * k3 * kw.y;
  const R n2 = g1.x * g1.x + g1.y * g1.y + g2.x * g2.x + g2.y * g2.y + g3.x * g3.x + g3.y * g3.y;
  return sqrt(n2) * (R)gp.inv_mu / s;
}

// Discrete Green operator (Algorithm D) at one half-spectrum point: out = invN * Gamma^c t, with
// Gamma^c stored as the upper triangle of its symmetric 6x6 Mandel matrix (basis 11,22,33,23,13,12
// with sqrt(2) on the shear components), 21 planes of stride S.
template <typename R, typename T>
__device__ __forceinline__ void dgo_apply_point(const T t[6], const double* __restrict__ tab, long long vi,
                                                long long S, R invN, T out[6]) {
  const R r2 = (R)1.41421356237309504880, ir2 = (R)0.70710678118654752440;
  T a[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const R f = c < 3 ? (R)1 : r2;
    a[c].x = f * t[c].x;
    a[c].y = f * t[c].y;
  }
  T o[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) { o[c].x = 0; o[c].y = 0; }
  int q = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j, ++q) {
      const R m = (R)tab[q * S + vi];
      o[i].x += m * a[j].x; o[i].y += m * a[j].y;
      if (j != i) { o[j].x += m * a[i].x; o[j].y += m * a[i].y; }
    }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const R f = (c < 3 ? (R)1 : ir2) * invN;
    out[c].x = f * o[c].x;
    out[c].y = f * o[c].y;
  }
}

// v = t kt for a symmetric complex tensor t (components 11,22,33,23,13,12) and a real vector kt
template <typename R, typename T>
__device__ __forceinline__ void tk_vec(const T t[6], R k1, R k2, R k3, T& v1, T& v2, T& v3) {
  v1.x = t[0].x * k1 + t[5].x * k2 + t[4].x * k3;  v1.y = t[0].y * k1 + t[5].y * k2 + t[4].y * k3;
  v2.x = t[5].x * k1 + t[1].x * k2 + t[3].x * k3;  v2.y = t[5].y * k1 + t[1].y * k2 + t[3].y * k3;
  v3.x = t[4].x * k1 + t[3].x * k2 + t[2].x * k3;  v3.y = t[4].y * k1 + t[3].y * k2 + t[2].y * k3;
}

// 1 / |kt|^2 for the Green operator: exact in FP64; in FP32 (only the inner correction iterations,
// whose result the FP64 residual pass re-checks) the hardware reciprocal, within 2 ulp.
__device__ __forceinline__ double recip_gamma(double s) { return 1.0 / s; }
__device__ __forceinline__ float recip_gamma(float s) { return __fdividef(1.0f, s); }

// Real isotropic Gamma0(kt) applied to a tensor whose product with kt is v, times -scale:
// out_ij = -scale [ (k_i v_j + k_j v_i) / (2 mu s) - c_lm k_i k_j (k.v) / s^2 ],  s = |kt|^2;
// out = 0 where kt = 0 (k = 0 and the modes where the scheme's wave vector vanishes).
template <typename R, typename T>
__device__ __forceinline__ void gamma0_from_v(T v1, T v2, T v3, R k1, R k2, R k3, R c_mu, R c_lm, R scale, T out[6]) {
  const R s = k1 * k1 + k2 * k2 + k3 * k3;
  if (s == (R)0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) { out[c].x = 0; out[c].y = 0; }
    return;
  }
  const R is = recip_gamma(s);
  const R a = c_mu * is * scale;               // scale / (2 mu s)
  T kv; kv.x = k1 * v1.x + k2 * v2.x + k3 * v3.x; kv.y = k1 * v1.y + k2 * v2.y + k3 * v3.y;
  const R b = c_lm * is * is * scale;
  T bkv; bkv.x = b * kv.x; bkv.y = b * kv.y;
  out[0].x = -(a * 2 * k1 * v1.x - k1 * k1 * bkv.x); out[0].y = -(a * 2 * k1 * v1.y - k1 * k1 * bkv.y);
  out[1].x = -(a * 2 * k2 * v2.x - k2 * k2 * bkv.x); out[1].y = -(a * 2 * k2 * v2.y - k2 * k2 * bkv.y);
  out[2].x = -(a * 2 * k3 * v3.x - k3 * k3 * bkv.x); out[2].y = -(a * 2 * k3 * v3.y - k3 * k3 * bkv.y);
  out[3].x = -(a * (k2 * v3.x + k3 * v2.x) - k2 * k3 * bkv.x); out[3].y = -(a * (k2 * v3.y + k3 * v2.y) - k2 * k3 * bkv.y);
  out[4].x = -(a * (k1 * v3.x + k3 * v1.x) - k1 * k3 * bkv.x); out[4].y = -(a * (k1 * v3.y + k3 * v1.y) - k1 * k3 * bkv.y);
  out[5].x = -(a * (k1 * v2.x + k2 * v1.x) - k1 * k2 * bkv.x); out[5].y = -(a * (k1 * v2.y + k2 * v1.y) - k1 * k2 * bkv.y);
}

template <typename R, typename T>
__device__ __forceinline__ void gamma0_apply(const T t[6], R k1, R k2, R k3, R c_mu, R c_lm, R scale, T out[6]) {
  T v1, v2, v3;
  tk_vec<R>(t, k1, k2, k3, v1, v2, v3);
  gamma0_from_v<R>(v1, v2, v3, k1, k2, k3, c_mu, c_lm, scale, out);
}

template <typename T>
__device__ __forceinline__ auto vnorm2(T v1, T v2, T v3) -> decltype(v1.x) {
  return v1.x * v1.x + v1.y * v1.y + v2.x * v2.x + v2.y * v2.y + v3.x * v3.x + v3.y * v3.y;
}

// |T kt|^2 for a symmetric complex tensor (6 comps) and a real vector
template <typename R, typename T>
__device__ __forceinline__ R tk_norm2(const T t[6], R k1, R k2, R k3) {
  const R v1x = t[0].x * k1 + t[5].x * k2 + t[4].x * k3;
  const R v1y = t[0].y * k1 + t[5].y * k2 + t[4].y * k3;
  const R v2x = t[5].x * k1 + t[1].x * k2 + t[3].x * k3;
  const R v2y = t[5].y * k1 + t[1].y * k2 + t[3].y * k3;
  const R v3x = t[4].x * k1 + t[3].x * k2 + t[2].x * k3;
  const R v3y = t[4].y * k1 + t[3].y * k2 + t[2].y * k3;
  return v1x * v1x + v1y * v1y + v2x * v2x + v2y * v2y + v3x * v3x + v3y * v3y;
}

// --------------------------------------------------------------------------------------------
// pass_x: one CTA handles `lines` consecutive x1-lines (fixed i3, consecutive i2).
// --------------------------------------------------------------------------------------------
// PX_STRAIN: transform the strain fluctuation eps - E (pp.E) instead of the stress (no state update).
// PX_OUTPUT (with PX_DELTA): write the inverse transform of components 0-2 to `eps`, here a [3][N]
// output array, and stop (displacement output).
// PX_DRES (FP64, with PX_DELTA): accumulate ||increment||_F^2 per CTA into partials[blockIdx.x] as
// PX_POLAR does, with the plain update eps += increment and the stress C : eps (the stress form of
// Algorithm D).
enum { PX_DELTA = 1, PX_ZERO = 2, PX_POLAR = 4, PX_STRAIN = 8, PX_OUTPUT = 16, PX_DRES = 32 };

// Polarization form of the discrete-Green-operator iteration (Algorithm D with the polarization of
// Eloh2019): with PX_POLAR the x-pass forms eps = E_bar + inverse transform (instead of adding it),
// accumulates ||eps_new - eps_old||_F^2 per CTA into partials[blockIdx.x] when PX_DELTA is set, and
// transforms tau = (C - C_H) : eps instead of sigma = C : eps.
// estar (eigenstrain generalization at the end of Sec. 6, FP64 passes): if set, the stress is
// sigma = C : (eps - estar), estar [6][N] in the strain's layout; the stored strain stays total.
struct PolarParams {
  double E[6];
  double lam_h, mu_h;
  double* partials;
  const double* estar;
};

// Stress (or polarization) of one voxel, packed as the three complex pairs (11,22), (33,23), (13,12).
template <typename R, typename T>
__device__ __forceinline__ void pack_stress(const R e[6], R la, R mu, T z[3]) {
  const R m2 = (R)2 * mu, ltr = la * (e[0] + e[1] + e[2]);
  z[0].x = m2 * e[0] + ltr; z[0].y = m2 * e[1] + ltr;
  z[1].x = m2 * e[2] + ltr; z[1].y = m2 * e[3];
  z[2].x = m2 * e[4];       z[2].y = m2 * e[5];
}

// Polarization update of one voxel: e <- E_bar + d (d: the inverse transform), returns the squared
// Frobenius norm of the change (shear components count twice).
template <typename R>
__device__ __forceinline__ double polar_update(R e[6], const R d[6], const PolarParams& pp) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const R en = (R)pp.E[c] + d[c];
    const double df = (double)en - (double)e[c];
    s += (c < 3 ? 1.0 : 2.0) * df * df;
    e[c] = en;
  }
  return s;
}

// Squared Frobenius norm of a strain increment (shear components count twice).
template <typename R>
__device__ __forceinline__ double incr_norm2(const R d[6]) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) s += (c < 3 ? 1.0 : 2.0) * (double)d[c] * (double)d[c];
  return s;
}

// Block sum of one double per thread (thread 0 receives the result); all threads must call.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    s = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  }
  return s;
}

// flags: PX_DELTA adds the inverse x-transform of the spectrum (the previous increment) to the state;
// PX_ZERO starts from a zero state (not read, written as zeros).  corr (FP32, may be null) is an
// additive correction with FP64 mean corr_mean removed: state += corr - corr_mean (mixed-precision
// refinement of the FP64 strain).
template <typename R>
__global__ void pass_x_kernel(typename C<R>::T* __restrict__ spec, R* __restrict__ eps, const R* __restrict__ lam,
                              const R* __restrict__ mu, const typename C<R>::T* __restrict__ tw, FftPlan plan, Dims d,
                              int lines, int flags, const float* __restrict__ corr, const double* __restrict__ corr_mean,
                              PolarParams pp, const SolveState* __restrict__ st) {
  typedef typename C<R>::T T;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  T* twl = reinterpret_cast<T*>(smem_raw);
  T* bufa = twl + d.n1;                      // [3 pairs][lines][n1], two ping-pong copies
  T* bufb = bufa + 3 * lines * d.n1;
  T* buf = bufa;
  const int n1 = d.n1, n1h = d.n1h;
  const long long nlines = (long long)d.n2 * d.n3;
  const long long line0 = (long long)blockIdx.x * lines;
  const bool zero = (flags & PX_ZERO) != 0 || st->restart;
  const bool have_delta = (flags & PX_DELTA) != 0 && !st->restart;
  const bool outmode = (flags & PX_OUTPUT) != 0, strainmode = (flags & PX_STRAIN) != 0;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) twl[i] = tw[i];
  const int tot_lines = 3 * lines;
  if (have_delta) {
    // Hermitian-extend the two half spectra of each component pair into Z = A + i B.
    for (int i = threadIdx.x; i < tot_lines * n1h; i += blockDim.x) {
      const int k = i % n1h;
      const int pl = i / n1h;                 // pair * lines + l
      const int l = pl % lines, p = pl / lines;
      const long long li = line0 + l;
      T z0, z1;
      if (li < nlines) {
        const long long row = d.xrow(li) * d.P;
        T A = spec[(2 * p) * d.S + row + k];
        T B = spec[(2 * p + 1) * d.S + row + k];
        const bool selfconj = (k == 0) || (2 * k == n1);
        if (selfconj) { A.y = 0; B.y = 0; }
        z0.x = A.x - B.y; z0.y = A.y + B.x;     // Z[k] = A + iB
        z1.x = A.x + B.y; z1.y = -A.y + B.x;    // Z[n-k] = conj(A) + i conj(B)
      } else {
        z0.x = z0.y = z1.x = z1.y = 0;
      }
      T* line = buf + pl * n1;
      line[k] = z0;
      if (k > 0 && 2 * k != n1) line[n1 - k] = z1;
    }
    __syncthreads();
    buf = fft_lines<true>(bufa, bufb, twl, plan, LineLayout{tot_lines, 1, n1, false});
  } else {
    __syncthreads();
  }
  double cm[6];
  if (corr) {
#pragma unroll
    for (int c = 0; c < 6; ++c) cm[c] = corr_mean[c];
  }
  const bool polar = (flags & PX_POLAR) != 0;
  const bool dres = sizeof(R) == 8 && (flags & PX_DRES) != 0;
  double dacc = 0.0;
  // state update, sigma = C : eps, repack sigma pairs for the forward transform
  for (int i = threadIdx.x; i < lines * n1; i += blockDim.x) {
    const int x = i % n1, l = i / n1;
    const long long li = line0 + l;
    if (li >= nlines) continue;
    const long long v = li * n1 + x;
    R e[6];
    if (zero || outmode) {
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] = (R)0;
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] = eps[c * d.N + v];
    }
    if (have_delta) {
      R dd[6];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const T z = buf[(p * lines + l) * n1 + x];
        dd[2 * p] = z.x;
        dd[2 * p + 1] = z.y;
      }
      if (outmode) {
#pragma unroll
        for (int c = 0; c < 3; ++c) eps[c * d.N + v] = dd[c];
        continue;
      }
      if (polar) dacc += polar_update<R>(e, dd, pp);
      else {
        if (dres) dacc += incr_norm2<R>(dd);
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] += dd[c];
      }
    }
    if (corr) {
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] += (R)((double)corr[c * d.N + v] - cm[c]);
    }
    if (have_delta || zero || corr) {
#pragma unroll
      for (int c = 0; c < 6; ++c) eps[c * d.N + v] = e[c];
    }
    T zz[3];
    if (strainmode) {
      zz[0].x = e[0] - (R)pp.E[0]; zz[0].y = e[1] - (R)pp.E[1];
      zz[1].x = e[2] - (R)pp.E[2]; zz[1].y = e[3] - (R)pp.E[3];
      zz[2].x = e[4] - (R)pp.E[4]; zz[2].y = e[5] - (R)pp.E[5];
    } else if (polar) pack_stress<R>(e, lam[v] - (R)pp.lam_h, mu[v] - (R)pp.mu_h, zz);
    else if (pp.estar) {
      R es[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) es[c] = e[c] - (R)pp.estar[c * d.N + v];
      pack_stress<R>(es, lam[v], mu[v], zz);
    } else pack_stress<R>(e, lam[v], mu[v], zz);
#pragma unroll
    for (int p = 0; p < 3; ++p) buf[(p * lines + l) * n1 + x] = zz[p];
  }
  if (outmode) return;
  if ((polar || dres) && have_delta) {
    const double sum = block_sum(dacc, red);
    if (threadIdx.x == 0) pp.partials[blockIdx.x] = sum;
  }
  __syncthreads();
  buf = fft_lines<false>(buf, buf == bufa ? bufb : bufa, twl, plan, LineLayout{tot_lines, 1, n1, false});
  // split Z = FFT(a + i b) into the half spectra of a and b
  for (int i = threadIdx.x; i < tot_lines * n1h; i += blockDim.x) {
    const int k = i % n1h;
    const int pl = i / n1h;
    const int l = pl % lines, p = pl / lines;
    const long long li = line0 + l;
    if (li >= nlines) continue;
    const T* line = buf + pl * n1;
    const T zk = line[k];
    const T zn = line[(n1 - k) % n1];
    T A, B;
    A.x = (R)0.5 * (zk.x + zn.x); A.y = (R)0.5 * (zk.y - zn.y);
    B.x = (R)0.5 * (zk.y + zn.y); B.y = (R)-0.5 * (zk.x - zn.x);
    const long long row = d.xrow(li) * d.P;
    spec[(2 * p) * d.S + row + k] = A;
    spec[(2 * p + 1) * d.S + row + k] = B;
  }
}

// --------------------------------------------------------------------------------------------
// pass_y: tile = all n2 rows x `cols` consecutive k1 columns of one component at fixed k3.
// --------------------------------------------------------------------------------------------
template <typename R, bool INV>
__global__ void pass_y_kernel(typename C<R>::T* __restrict__ spec, const typename C<R>::T* __restrict__ tw,
                              FftPlan plan, Dims d, int cols, const SolveState* __restrict__ st) {
  typedef typename C<R>::T T;
  if (st->done && !(INV && st->done == 2)) return;  // as in pass_y_c_kernel
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* twl = reinterpret_cast<T*>(smem_raw);
  T* buf = twl + d.n2;                       // [n2][cols], plus a ping-pong copy
  T* buf2 = buf + d.n2 * cols;
  const int k10 = blockIdx.x * cols;
  const int k3 = blockIdx.y;
  const int c = blockIdx.z;
  for (int i = threadIdx.x; i < d.n2; i += blockDim.x) twl[i] = tw[i];
  T* g = spec + c * d.S + d.row(k3, 0) * d.P + k10;
  const long long ys = d.ystride();
  for (int i = threadIdx.x; i < d.n2 * cols; i += blockDim.x) {
    const int cc = i % cols, y = i / cols;
    T v; v.x = 0; v.y = 0;
    if (k10 + cc < d.n1h) v = g[(long long)y * ys + cc];
    buf[i] = v;
  }
  __syncthreads();
  buf = fft_lines<INV>(buf, buf2, twl, plan, LineLayout{cols, cols, 1, true});
  for (int i = threadIdx.x; i < d.n2 * cols; i += blockDim.x) {
    const int cc = i % cols, y = i / cols;
    if (k10 + cc < d.n1h) g[(long long)y * ys + cc] = buf[i];
  }
}

// --------------------------------------------------------------------------------------------
// pass_z_gamma: tile = all n3 rows x `cols` k1 columns x 6 components at fixed k2.
// smem layout [k3][comp][col] so that line (comp, col) has element stride 6 cols.
// --------------------------------------------------------------------------------------------
enum { PZ_GAMMA = 0, PZ_RESIDUAL = 1, PZ_INNER = 2, PZ_DGO = 3, PZ_DISP = 4 };

// mode PZ_DISP (displacement output, FP64): the tile holds the transformed strain fluctuation
// E~(k) = sym(u^(k) (x) q^a(k)) of a solution; it is replaced by u^(k) / N in components 0-2 (3-5 zeroed).
// With q^a = c i kt, |c| = 1: sym(u (x) kt) = E~ / (c i), so u = (2 E~ kt - kt (kt.E~ kt)/|kt|^2) / (c i |kt|^2);
// u = 0 where kt = 0 (as the Green operator there).
__device__ __forceinline__ double disp_theta(int i, int n) {
  const int kap = (i < (n + 1) / 2) ? i : i - n;  // the Nyquist index of an even axis is kappa = -n/2
  return 6.283185307179586476925286766559 * (double)kap / (double)n;
}
template <typename R, typename T>
__device__ __forceinline__ void disp_point(const T t[6], R k1, R k2, R k3, int half_shift, const Dims& d, int i1,
                                           int i2, int i3, R invN, T o[6]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) { o[c].x = 0; o[c].y = 0; }
  const R s = k1 * k1 + k2 * k2 + k3 * k3;
  if (s == (R)0) return;
  T v1, v2, v3;
  tk_vec<R>(t, k1, k2, k3, v1, v2, v3);
  T kv;
  kv.x = k1 * v1.x + k2 * v2.x + k3 * v3.x;
  kv.y = k1 * v1.y + k2 * v2.y + k3 * v3.y;
  const R is = (R)1 / s;
  T nn[3];
  nn[0].x = 2 * v1.x - k1 * kv.x * is; nn[0].y = 2 * v1.y - k1 * kv.y * is;
  nn[1].x = 2 * v2.x - k2 * kv.x * is; nn[1].y = 2 * v2.y - k2 * kv.y * is;
  nn[2].x = 2 * v3.x - k3 * kv.x * is; nn[2].y = 2 * v3.y - k3 * kv.y * is;
  // divide by c i: multiply by -i conj(c) = -ci - i cr  (c = cr + i ci)
  R cr = 1, ci = 0;
  if (half_shift) {
    const double ph = 0.5 * (disp_theta(i1, d.n1) + disp_theta(i2, d.n2) + disp_theta(i3, d.n3));
    double sn, cs;
    sincos(ph, &sn, &cs);
    cr = (R)cs;
    ci = (R)sn;
  }
  const R f = is * invN;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // (x + i y) (-ci - i cr) = (y cr - x ci) + i (-x cr - y ci)
    o[c].x = f * (nn[c].y * cr - nn[c].x * ci);
    o[c].y = -f * (nn[c].x * cr + nn[c].y * ci);
  }
}

// mode PZ_GAMMA: Delta E = -Gamma0(kt) T / N, residual, T(0), inverse z (the FP64 or FP32 iteration).
// mode PZ_RESIDUAL: residual and T(0) only; stores v = T kt (FP32, [3][k3][k2][P]) as the source of
// the inner iterations; no Green step, no inverse, the spectrum is not written back.
// mode PZ_INNER: v = T kt + vsrc (the FP64 outer residual), residual of v, Delta E from v, inverse z.
template <typename R>
__global__ void pass_z_gamma_kernel(typename C<R>::T* __restrict__ spec, const typename C<R>::T* __restrict__ tw,
                                    FftPlan plan, Dims d, int cols, GammaParams<R> gp, double* __restrict__ partials,
                                    SolveState* __restrict__ st, int mode, float2* __restrict__ vsrc) {
  typedef typename C<R>::T T;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* twl = reinterpret_cast<T*>(smem_raw);
  T* buf = twl + d.n3;                       // [n3][6][cols], plus a ping-pong copy
  T* buf2 = buf + d.n3 * 6 * cols;
  __shared__ double red[32];
  const int k10 = blockIdx.x * cols;
  const int k2 = blockIdx.y;
  const int w6 = 6 * cols;
  for (int i = threadIdx.x; i < d.n3; i += blockDim.x) twl[i] = tw[i];
  for (int i = threadIdx.x; i < d.n3 * w6; i += blockDim.x) {
    const int cc = i % cols, rest = i / cols;
    const int comp = rest % 6, z = rest / 6;
    T v; v.x = 0; v.y = 0;
    if (k10 + cc < d.n1h) v = spec[comp * d.S + d.row(z, k2) * d.P + k10 + cc];
    buf[i] = v;
  }
  __syncthreads();
  buf = fft_lines<false>(buf, buf2, twl, plan, LineLayout{w6, w6, 1, true});
  T* other = (buf == buf2) ? buf2 - d.n3 * w6 : buf2;
  // Green operator, residual and T(0)
  R acc = 0, acc2 = 0;
  const bool ny2 = ((d.n2 & 1) == 0) && (2 * k2 == d.n2);
  const R b2 = gp.B[1][k2], a2 = gp.A[1][k2];
  for (int i = threadIdx.x; i < d.n3 * cols; i += blockDim.x) {
    const int cc = i % cols, z = i / cols;
    const int k1 = k10 + cc;
    if (k1 >= d.n1h) continue;
    T t[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = buf[(z * 6 + c) * cols + cc];
    const R a1 = gp.A[0][k1], b1 = gp.B[0][k1];
    const R a3 = gp.A[2][z], b3 = gp.B[2][z];
    const R kt1 = a1 * b2 * b3, kt2 = a2 * b3 * b1, kt3 = a3 * b1 * b2;
    const bool ny1 = ((d.n1 & 1) == 0) && (2 * k1 == d.n1);
    const bool ny3 = ((d.n3 & 1) == 0) && (2 * z == d.n3);
    const bool self1 = (k1 == 0) || ny1;
    const long long vi = d.row(z, k2) * d.P + k1;
    if (mode == PZ_DISP) {
      T o[6];
      disp_point<R>(t, kt1, kt2, kt3, gp.half_shift, d, k1, k2, z, gp.invN, o);
#pragma unroll
      for (int c = 0; c < 6; ++c) buf[(z * 6 + c) * cols + cc] = o[c];
      continue;
    }
    if (mode != PZ_INNER && k1 == 0 && k2 == 0 && z == 0) {
#pragma unroll
      for (int c = 0; c < 6; ++c) st->T0[c] = (double)t[c].x;
    }
    T v1, v2, v3;
    tk_vec<R>(t, kt1, kt2, kt3, v1, v2, v3);
    if (mode == PZ_INNER) {
      const float2 s1 = vsrc[vi], s2 = vsrc[d.S + vi], s3 = vsrc[2 * d.S + vi];
      v1.x += (R)s1.x; v1.y += (R)s1.y; v2.x += (R)s2.x; v2.y += (R)s2.y; v3.x += (R)s3.x; v3.y += (R)s3.y;
    }
    // residual: stored point plus (for interior k1) its Hermitian partner, whose wave vector is
    // -kt with the components on Nyquist axes 2, 3 negated back
    R r2 = vnorm2(v1, v2, v3);
    if (!self1) {
      if (gp.nyq_avg && (ny2 || ny3)) r2 += tk_norm2<R>(t, kt1, ny2 ? -kt2 : kt2, ny3 ? -kt3 : kt3);
      else r2 *= (R)2;
    }
    acc += r2;
    if (sizeof(R) == 8 && mode == PZ_GAMMA && gp.vprev) {
      const R c = incr_point<R>(v1, v2, v3, kt1, kt2, kt3, gp, vi, d.S);
      acc2 += self1 ? c : (R)2 * c;
    }
    if (mode == PZ_RESIDUAL) {
      float2 o1, o2, o3;
      o1.x = (float)v1.x; o1.y = (float)v1.y; o2.x = (float)v2.x; o2.y = (float)v2.y;
      o3.x = (float)v3.x; o3.y = (float)v3.y;
      vsrc[vi] = o1; vsrc[d.S + vi] = o2; vsrc[2 * d.S + vi] = o3;
      continue;
    }
    T o[6];
    if (mode == PZ_DGO) {
      dgo_apply_point<R>(t, gp.dgo, vi, d.S, gp.invN, o);
#pragma unroll
      for (int c = 0; c < 6; ++c) buf[(z * 6 + c) * cols + cc] = o[c];
      continue;
    }
    gamma0_from_v<R>(v1, v2, v3, kt1, kt2, kt3, gp.c_mu, gp.c_lm, gp.invN, o);
    if (gp.nyq_avg && (ny1 || ny2 || ny3)) {
      T o2[6];
      gamma0_apply<R>(t, ny1 ? -kt1 : kt1, ny2 ? -kt2 : kt2, ny3 ? -kt3 : kt3, gp.c_mu, gp.c_lm, gp.invN, o2);
#pragma unroll
      for (int c = 0; c < 6; ++c) { o[c].x = (R)0.5 * (o[c].x + o2[c].x); o[c].y = (R)0.5 * (o[c].y + o2[c].y); }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) buf[(z * 6 + c) * cols + cc] = o[c];
  }
  if (sizeof(R) == 8 && mode == PZ_GAMMA && gp.vprev) {
    const double s2 = block_sum((double)acc2, red);
    if (threadIdx.x == 0) gp.cpart[blockIdx.y * gridDim.x + blockIdx.x] = s2;
    __syncthreads();
  }
  // deterministic block reduction of the residual partial (FP64 across threads)
  double accd = (double)acc;
  for (int off = 16; off > 0; off >>= 1) accd += __shfl_down_sync(0xffffffffu, accd, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = accd;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    double s = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
  if (mode == PZ_RESIDUAL) return;
  buf = fft_lines<true>(buf, other, twl, plan, LineLayout{w6, w6, 1, true});
  for (int i = threadIdx.x; i < d.n3 * w6; i += blockDim.x) {
    const int cc = i % cols, rest = i / cols;
    const int comp = rest % 6, z = rest / 6;
    if (k10 + cc < d.n1h) spec[comp * d.S + d.row(z, k2) * d.P + k10 + cc] = buf[i];
  }
}

// --------------------------------------------------------------------------------------------
// Launch configuration and host-side launchers (instantiated per precision in gfp_k64.cu / gfp_k32.cu)
// --------------------------------------------------------------------------------------------
// Lengths with a compile-time register-FFT plan (CPlan in gfp_fftc.cuh); other lengths 2^a 3^b run the
// shared-memory Stockham kernels with a runtime radix schedule.
#define GFP_FOR_CSIZES(X) X(32) X(64) X(96) X(128) X(192) X(256) X(512)
inline bool has_register_plan(int n) {
#define GFP_CS(N_) if (n == N_) return true;
  GFP_FOR_CSIZES(GFP_CS)
#undef GFP_CS
  return false;
}

struct LaunchCfg {
  int x_lines, x_threads;   // generic x-pass
  int y_cols, y_threads;
  int z_cols, z_threads;
  int z_blocks;             // number of pass_z CTAs (partials written)
  int cx_lines;             // lines per CTA of the register-FFT x-pass (0: default)
  const void* ztmap;        // host CUtensorMap of the spectrum for TMA z-tiles of z_cols columns, or null
  int z_tma;                // use the TMA-fed z-pass when eligible (1) or the register-FFT one (0)
  int x_async;              // register-FFT x-pass with cp.async staging (1) or direct loads (0)
  FftPlan plan[3];          // radix schedules of the shared-memory Stockham passes per axis (lengths
                            // without a register-FFT plan), chosen by the autotuner
};

template <typename R>
struct Passes {
  typedef typename C<R>::T T;
  static cudaError_t setup();   // opt-in shared memory limits
  static void pass_x(cudaStream_t s, const LaunchCfg& lc, T* spec, R* eps, const R* lam, const R* mu, const T* tw,
                     const FftPlan& plan, const Dims& d, int flags, const float* corr, const double* corr_mean,
                     const SolveState* st, const PolarParams* pp = nullptr);
  static void pass_y(cudaStream_t s, const LaunchCfg& lc, bool inverse, T* spec, const T* tw, const FftPlan& plan,
                     const Dims& d, const SolveState* st, int comps = 6);
  static void pass_z(cudaStream_t s, const LaunchCfg& lc, T* spec, const T* tw, const FftPlan& plan, const Dims& d,
                     const GammaParams<R>& gp, double* partials, SolveState* st, int mode, float2* vsrc);
};

void launch_reduce_eta(cudaStream_t s, const double* partials, int np, SolveState* st, double* hist, int hist_cap);

// Test-only fault injection: nonzero makes the TMA z-pass treat its first tile wait as timed out.
extern unsigned g_inject_tma_timeout;

template <typename R> bool cz_cols_ok(int n3, int cols);
template <typename R> bool cz_tma_ok(int n3, int cols);
template <typename R> int cy_cols_max(int n2);

}  // namespace gfp
