// C ABI of the GFP solver: grid handles, phases, the iteration driver, effective stiffness,
// sensitivities and checkpoint/resume.  See include/gfp.h for the contract of each call.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/gfp.h"
#include "gfp_kernels.cuh"
#include "gfp_outer.cuh"

using namespace gfp;

// ------------------------------------------------------------------------------- small kernels
namespace gfp {

__global__ void reduce_eta_kernel(const double* __restrict__ partials, int np, SolveState* st, double* hist,
                                  int hist_cap) {
  if (st->done) return;
  __shared__ double sh[32];
  // four independent partial sums per thread keep four L2 loads in flight (a single running sum
  // serialises one load latency per partial)
  const int step = blockDim.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = threadIdx.x;
  for (; i + 3 * step < np; i += 4 * step) {
    s0 += partials[i];
    s1 += partials[i + step];
    s2 += partials[i + 2 * step];
    s3 += partials[i + 3 * step];
  }
  for (; i < np; i += step) s0 += partials[i];
  double s = (s0 + s1) + (s2 + s3);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) sh[0] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->restart = 0;  // the x-pass of this iteration has run
    const double* t = st->T0;
    const double t0 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + 2.0 * (t[3] * t[3] + t[4] * t[4] + t[5] * t[5]);
    const double sum = sh[0];
    double eta;
    if (t0 > 0.0) eta = sqrt(sum / t0);
    else eta = (sum > 0.0) ? INFINITY : 0.0;
    const int it = st->it + 1;
    st->it = it;
    const double prev = st->eta;
    st->eta = eta;
    if (hist && it - 1 < hist_cap) hist[it - 1] = eta;
    if (!(eta == eta) || isinf(eta)) {
      st->done = 3;
    } else if (eta < st->tol) {
      st->done = 1;
    } else {
      if (it > 1 && eta > prev) st->growth += 1; else st->growth = 0;
      if (eta < st->eta_min) st->eta_min = eta;
      if (st->growth >= 50) st->done = 3;
      else if (it >= st->maxit) st->done = 2;
    }
  }
}

unsigned g_inject_tma_timeout = 0;

// The paper's stopping rule (stop_rule 1): eta as in reduce_eta_kernel (reported), and the decision on
// crit = scale * sum of the criterion partials, sum_k |du_it(k) - du_(it-1)(k)| over the whole spectrum
// of the unitary transform; the first iteration has no previous increment (crit = infinity).
__global__ void reduce_crit_kernel(const double* __restrict__ partials, const double* __restrict__ cpart, int np,
                                   double scale, SolveState* st, double* hist, int hist_cap) {
  if (st->done) return;
  __shared__ double sh[2][32];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    s += partials[i];
    c += cpart[i];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, off);
    c += __shfl_down_sync(0xffffffffu, c, off);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = s; sh[1][threadIdx.x >> 5] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    s = 0.0;
    c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s += sh[0][w]; c += sh[1][w]; }
    st->restart = 0;
    const double* t = st->T0;
    const double t0 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + 2.0 * (t[3] * t[3] + t[4] * t[4] + t[5] * t[5]);
    const double eta = t0 > 0.0 ? sqrt(s / t0) : (s > 0.0 ? INFINITY : 0.0);
    const int it = st->it + 1;
    st->it = it;
    const double prev = st->eta;
    st->eta = eta;
    const double crit = it == 1 ? INFINITY : scale * c;
    st->crit = crit;
    if (hist && it - 1 < hist_cap) hist[it - 1] = crit;
    if (!(eta == eta) || isinf(eta) || !(crit == crit)) {
      st->done = 3;
    } else if (crit < st->tol) {
      st->done = 1;
    } else {
      if (it > 1 && eta > prev) st->growth += 1; else st->growth = 0;
      if (eta < st->eta_min) st->eta_min = eta;
      if (st->growth >= 50) st->done = 3;
      else if (it >= st->maxit) st->done = 2;
    }
  }
}

void launch_reduce_eta(cudaStream_t s, const double* partials, int np, SolveState* st, double* hist, int hist_cap) {
  reduce_eta_kernel<<<1, 1024, 0, s>>>(partials, np, st, hist, hist_cap);
}

__global__ void fill_eps_kernel(double* eps, long long N, double e0, double e1, double e2, double e3, double e4,
                                double e5) {
  const double e[6] = {e0, e1, e2, e3, e4, e5};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 6; ++c) eps[c * N + i] = e[c];
  }
}

// min/max of lambda and mu and a count of invalid entries (mu <= 0 or non-finite values)
__global__ void phase_stats_kernel(const double* lam, const double* mu, long long N, double* out_minmax,
                                   unsigned long long* bad) {
  __shared__ double s[4][256];
  double lmin = INFINITY, lmax = -INFINITY, mmin = INFINITY, mmax = -INFINITY;
  unsigned long long nb = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double l = lam[i], m = mu[i];
    if (!isfinite(l) || !isfinite(m) || !(m > 0.0)) { nb++; continue; }
    lmin = fmin(lmin, l); lmax = fmax(lmax, l); mmin = fmin(mmin, m); mmax = fmax(mmax, m);
  }
  s[0][threadIdx.x] = lmin; s[1][threadIdx.x] = -lmax; s[2][threadIdx.x] = mmin; s[3][threadIdx.x] = -mmax;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = fmin(s[q][threadIdx.x], s[q][threadIdx.x + w]);
    __syncthreads();
  }
  if (nb) atomicAdd(bad, nb);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) out_minmax[blockIdx.x * 4 + q] = s[q][0];
  }
}

// dC_IJ/dlambda_i = (1/N) tr eI tr eJ, dC_IJ/dmu_i = (2/N) eI : eJ (symmetric tensors, 6 comps)
__global__ void grad_contract_kernel(const double* eI, const double* eJ, long long N, double* dl, double* dm) {
  const double invN = 1.0 / (double)N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double a[6], b[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { a[c] = eI[c * N + i]; b[c] = eJ[c * N + i]; }
    const double trI = a[0] + a[1] + a[2], trJ = b[0] + b[1] + b[2];
    const double dd = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + 2.0 * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5]);
    dl[i] = trI * trJ * invN;
    dm[i] = 2.0 * dd * invN;
  }
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Mean of the six FP32 correction components, accumulated in FP64 (stage 1: per-block partials).
// gate (may be null): skip while the inner state is paused at its window cap (state 2), i.e. unless
// an FP64 outer pass follows
__global__ void corr_mean_partial_kernel(const float* __restrict__ corr, long long N, double* __restrict__ part,
                                         const SolveState* gate) {
  if (gate && gate->done == 2) return;
  __shared__ double sh[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += (double)corr[c * N + i];
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// stage 2: one block, fixed order
__global__ void corr_mean_final_kernel(const double* __restrict__ part, int nb, long long N, double* __restrict__ mean,
                                       const SolveState* gate) {
  if (gate && gate->done == 2) return;
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b * 6 + threadIdx.x];
    mean[threadIdx.x] = s / (double)N;
  }
}


// ---- discrete Green operator (Algorithm D-3D): alias-sum table, residual, mean stress
// Gamma^c_ijab(omega) = -(1/(4 mu_H)) [d_ia S2_bj + d_ib S2_aj + d_ja S2_bi + d_jb S2_ai] + c/mu_H S4_ijab,
// S2_ab = sum_nu w k_a k_b / |k|^2, S4_ijab = sum_nu w k_i k_j k_a k_b / |k|^4, w = prod_r s_r^power,
// k = 2 pi (nu n + omega) / (n h), c = (lambda_H + mu_H) / (lambda_H + 2 mu_H); Gamma^c(0) = 0.
__constant__ int c_mono4[3][3][3][3];  // index of the degree-4 monomial k_i k_j k_a k_b
__constant__ int c_mono2[3][3];        // index of the degree-2 monomial k_a k_b

// Alias sums of Gamma^c at the representative points rep_pts (o1, o2, o3) packed as o1 | o2 << 11 | o3 << 22:
// the 21 Mandel entries of each into rep [21][F3][F2][F1] at (o1, o2, o3) (F_r = n_r/2 + 1 when the axes
// are folded, else F1 = n1/2 + 1, F2 = n2, F3 = n3).
// sym = 0: nu_r in [-m_r, m_r - 1] (Algorithm D-3D).  sym = 1: the Hermitian part of the sum over
// [-m_r, m_r], i.e. 1/2 (sum over [-m, m]^3 + sum over [-m - 1, m - 1]^3) at omega (omega -> n - omega on
// all three axes at once maps nu to -nu - 1 and k to -k, which leaves every moment unchanged), summed over
// [-m - 1, m]^3 with the factor c(nu) = 1/2 ([all nu_r >= -m_r] + [all nu_r <= m_r - 1]).  A flip of
// one axis alone does not map c onto itself, so the sym table is computed at every point, unfolded.  The
// weight tables w_r cover nu_r in [lo_r, lo_r + W_r), W_r = 2 m_r (+ 2 with sym).
__global__ void dgo_table_kernel(double* __restrict__ rep, const int* __restrict__ rep_pts, int nrep, Dims d,
                                 int F1, int F2, int F3, const double* __restrict__ w1,
                                 const double* __restrict__ w2, const double* __restrict__ w3, int m1, int m2,
                                 int m3, int sym, double h, double lam_h, double mu_h) {
  const double two_pi = 6.283185307179586476925;
  const double cc = (lam_h + mu_h) / (lam_h + 2.0 * mu_h);
  const long long RS = (long long)F1 * F2 * F3;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nrep; idx += gridDim.x * blockDim.x) {
    const int code = rep_pts[idx];
    const int o1 = code & 2047, o2 = (code >> 11) & 2047, o3 = (code >> 22) & 2047;
    double S2[6] = {0, 0, 0, 0, 0, 0};
    double S4[15];
    for (int q = 0; q < 15; ++q) S4[q] = 0.0;
    if (o1 != 0 || o2 != 0 || o3 != 0) {
      // FP64 division is slow on this GPU: the axis scales are precomputed, each term takes one
      // reciprocal of |k|^2, and the fourth moments are formed from the six pair products
      const double f1 = two_pi / ((double)d.n1 * h), f2 = two_pi / ((double)d.n2 * h), f3 = two_pi / ((double)d.n3 * h);
      const int lo1 = sym ? -m1 - 1 : -m1, lo2 = sym ? -m2 - 1 : -m2, lo3 = sym ? -m3 - 1 : -m3;
      const int W1 = sym ? 2 * m1 + 2 : 2 * m1, W2 = sym ? 2 * m2 + 2 : 2 * m2, W3 = sym ? 2 * m3 + 2 : 2 * m3;
      for (int v3 = lo3; v3 < lo3 + W3; ++v3) {
        const double s3 = w3[o3 * W3 + (v3 - lo3)];
        if (s3 == 0.0) continue;
        const double k3 = f3 * (double)((long long)v3 * d.n3 + o3);
        for (int v2 = lo2; v2 < lo2 + W2; ++v2) {
          const double s2 = w2[o2 * W2 + (v2 - lo2)];
          if (s2 == 0.0) continue;
          const double k2 = f2 * (double)((long long)v2 * d.n2 + o2);
          const double s23 = s2 * s3;
          const double p22 = k2 * k2, p33 = k3 * k3, p23 = k2 * k3;
          const bool a23 = v2 >= -m2 && v3 >= -m3, b23 = v2 <= m2 - 1 && v3 <= m3 - 1;
          for (int v1 = lo1; v1 < lo1 + W1; ++v1) {
            const double s1 = w1[o1 * W1 + (v1 - lo1)];
            if (s1 == 0.0) continue;
            const double cf = sym ? 0.5 * ((a23 && v1 >= -m1 ? 1.0 : 0.0) + (b23 && v1 <= m1 - 1 ? 1.0 : 0.0)) : 1.0;
            if (cf == 0.0) continue;
            const double k1 = f1 * (double)((long long)v1 * d.n1 + o1);
            const double p11 = k1 * k1;
            const double kk = p11 + p22 + p33;
            if (kk == 0.0) continue;
            const double inv = 1.0 / kk;
            const double a = cf * s1 * s23 * inv, b = a * inv;
            // pair products k_i k_j, i <= j: (11, 12, 13, 22, 23, 33)
            const double pp[6] = {p11, k1 * k2, k1 * k3, p22, p23, p33};
            S2[0] += a * p11; S2[1] += a * p22; S2[2] += a * p33;
            S2[3] += a * p23; S2[4] += a * pp[2]; S2[5] += a * pp[1];
            // S4 entries in the order i <= j <= p <= r: k_i k_j k_p k_r = (k_i k_j)(k_p k_r)
            int q = 0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = i; j < 3; ++j)
#pragma unroll
                for (int p = j; p < 3; ++p)
#pragma unroll
                  for (int r = p; r < 3; ++r, ++q) {
                    const int ij = i == 0 ? j : (i == 1 ? 2 + j : 5);
                    const int pr = p == 0 ? r : (p == 1 ? 2 + r : 5);
                    S4[q] += b * pp[ij] * pp[pr];
                  }
          }
        }
      }
    }
    // 6x6 Mandel matrix, upper triangle
    const int vi[6] = {0, 1, 2, 1, 0, 0}, vj[6] = {0, 1, 2, 2, 2, 1};
    auto s2 = [&](int a, int b) { return S2[c_mono2[a][b]]; };
    auto dl = [](int a, int b) { return a == b ? 1.0 : 0.0; };
    const long long pos = ((long long)o3 * F2 + o2) * F1 + o1;
    int q = 0;
    for (int P = 0; P < 6; ++P)
      for (int Q = P; Q < 6; ++Q, ++q) {
        const int i = vi[P], j = vj[P], a = vi[Q], b = vj[Q];
        double g = -(dl(i, a) * s2(b, j) + dl(i, b) * s2(a, j) + dl(j, a) * s2(b, i) + dl(j, b) * s2(a, i)) /
                       (4.0 * mu_h) +
                   cc / mu_h * S4[c_mono4[i][j][a][b]];
        const double f = (P < 3 ? 1.0 : 1.41421356237309504880) * (Q < 3 ? 1.0 : 1.41421356237309504880);
        rep[q * RS + pos] = (o1 == 0 && o2 == 0 && o3 == 0) ? 0.0 : f * g;
      }
  }
}

// The table at every half-spectrum point from the representatives.  With `fold`, axis r folds to
// f_r = min(o_r, n_r - o_r): the alias sum of n_r - o_r runs over the same terms with k_r negated
// (nu_r -> -nu_r - 1 keeps the weight and the range [-m, m - 1]), so an entry with tensor indices
// (i, j, a, b) takes the sign s_i s_j s_a s_b, s_r = -1 on folded axes.  On a cubic grid (`cubic`: equal
// lengths and alias ranges) the folded point is sorted, g = (f_sig(0), f_sig(1), f_sig(2)) ascending, and
// the isotropic Gamma_H gives Gamma^c(f)_ijab = Gamma^c(g)_{pi(i) pi(j) pi(a) pi(b)} with pi the inverse
// of sig.  Without `fold` every point is its own representative.
__global__ void dgo_expand_kernel(double* __restrict__ tab, const double* __restrict__ rep, Dims d, int F1, int F2,
                                  int F3, int fold, int cubic) {
  const long long RS = (long long)F1 * F2 * F3;
  const long long npts = (long long)d.n1h * d.n2 * d.n3;
  const int vi[6] = {0, 1, 2, 1, 0, 0}, vj[6] = {0, 1, 2, 2, 2, 1};
  const int mandel[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < npts;
       idx += (long long)gridDim.x * blockDim.x) {
    const int o[3] = {(int)(idx % d.n1h), (int)((idx / d.n1h) % d.n2), (int)(idx / ((long long)d.n1h * d.n2))};
    const int n[3] = {d.n1, d.n2, d.n3};
    int f[3], sg[3];
    for (int r = 0; r < 3; ++r) {
      const bool fl = fold && o[r] > n[r] / 2;
      f[r] = fl ? n[r] - o[r] : o[r];
      sg[r] = fl ? -1 : 1;
    }
    int pi[3] = {0, 1, 2};  // axis r of f is axis pi[r] of the representative
    int g[3] = {f[0], f[1], f[2]};
    if (cubic) {
      int sig[3] = {0, 1, 2};  // g[k] = f[sig[k]], ascending
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2 - a; ++b)
          if (f[sig[b]] > f[sig[b + 1]]) { const int t = sig[b]; sig[b] = sig[b + 1]; sig[b + 1] = t; }
      for (int k = 0; k < 3; ++k) { g[k] = f[sig[k]]; pi[sig[k]] = k; }
    }
    const long long rpos = ((long long)g[2] * F2 + g[1]) * F1 + g[0];
    const long long pos = d.row(o[2], o[1]) * d.P + o[0];
    int q = 0;
    for (int P = 0; P < 6; ++P)
      for (int Q = P; Q < 6; ++Q, ++q) {
        const int i = vi[P], j = vj[P], a = vi[Q], b = vj[Q];
        int P2 = mandel[pi[i]][pi[j]], Q2 = mandel[pi[a]][pi[b]];
        if (P2 > Q2) { const int t = P2; P2 = Q2; Q2 = t; }
        const int q2 = P2 * 6 - P2 * (P2 - 1) / 2 + (Q2 - P2);  // upper-triangle index of (P2, Q2)
        tab[q * d.S + pos] = (double)(sg[i] * sg[j] * sg[a] * sg[b]) * rep[q2 * RS + rpos];
      }
  }
}

// eta_D = sqrt(sum of partials) / (sqrt(N) ||E_bar||_F); one block, fixed order.
__global__ void reduce_dgo_kernel(const double* __restrict__ partials, int np, double enorm, SolveState* st,
                                  double* hist, int hist_cap) {
  if (st->done) return;
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partials[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double eta = enorm > 0.0 ? sqrt(sh[0]) / enorm : (sh[0] > 0.0 ? INFINITY : 0.0);
    const int it = st->it + 1;
    st->it = it;
    const double prev = st->eta;
    st->eta = eta;
    if (hist && it - 1 < hist_cap) hist[it - 1] = eta;
    if (!(eta == eta) || isinf(eta)) st->done = 3;
    else if (eta < st->tol) st->done = 1;
    else {
      if (it > 1 && eta > prev) st->growth += 1; else st->growth = 0;
      if (st->growth >= 50) st->done = 3;
      else if (it >= st->maxit) st->done = 2;
    }
  }
}

// Mean stress sum(C : eps) per component, FP64, per-block partials (stage 1).
__global__ void stress_sum_partial_kernel(const double* __restrict__ eps, const double* __restrict__ lam,
                                          const double* __restrict__ mu, long long N, double* __restrict__ part) {
  __shared__ double sh[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps[c * N + i];
    const double ltr = lam[i] * (e[0] + e[1] + e[2]), m2 = 2.0 * mu[i];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += m2 * e[c] + (c < 3 ? ltr : 0.0);
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}


// ---- batched solves: per-slot bookkeeping between the FP64 outer pass and the FP32 inner window
struct BatchAcc {
  int inner;  // inner iterations accumulated over the windows
  int outer;  // FP64 outer passes
};

// Parameters of one batched solve, read by the slots' kernels on the device (so that one instantiated
// graph serves any tolerance and iteration budget).
struct BatchCtl {
  double tol;
  int max_windows;
};

// First kernel of a slot's window: on the slot's first window the initial state (eps = E_J for the
// Voigt unit load J, zero FP32 correction, fresh outer and inner states); a no-op afterwards.
__global__ void batch_init_kernel(double* __restrict__ eps, float* __restrict__ eps32, long long N, int load,
                                  SolveState* __restrict__ st, SolveState* __restrict__ st_in, BatchAcc* acc,
                                  double* __restrict__ cmean, const int* __restrict__ windows,
                                  const BatchCtl* __restrict__ ctl) {
  if (*windows != 0) return;
  const double e = load < 3 ? 1.0 : 0.5;  // tensor component of the Voigt unit strain
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 6 * N; i += stride) {
    eps[i] = (i / N == load) ? e : 0.0;
    eps32[i] = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SolveState s0;
    memset(&s0, 0, sizeof(s0));
    s0.maxit = 1 << 30;
    s0.tol = ctl->tol;
    s0.eta = INFINITY;
    s0.eta_min = INFINITY;
    *st = s0;
    *st_in = s0;
    acc->inner = 0;
    acc->outer = 0;
    for (int c = 0; c < 6; ++c) cmean[c] = 0.0;
  }
}

// Start of a slot's window: if its inner iterations stopped at the window cap (state 2) they continue
// for another window and the FP64 outer pass is held (DONE_HELD makes its kernels no-ops); otherwise
// (first window, inner target reached, inner divergence) the outer pass runs.
__global__ void batch_gate_kernel(SolveState* __restrict__ st, SolveState* __restrict__ st_in, int window) {
  if (threadIdx.x != 0 || st->done) return;
  if (st_in->done == 2) {
    st->done = DONE_HELD;
    st_in->done = 0;
    st_in->maxit += window;
  }
}

// After the (possibly held) FP64 residual pass: a held slot resumes its inner iterations; otherwise
// count the finished inner solve's iterations and re-arm the inner state from a zero correction with
// the target max(tol/2, ratio eta_64) and the reference stress norm of the outer pass; a converged
// slot leaves its inner state done.
__global__ void batch_arm_kernel(SolveState* __restrict__ st, SolveState* __restrict__ st_in, BatchAcc* acc,
                                 const BatchCtl* __restrict__ ctl, double ratio, int window) {
  if (threadIdx.x != 0) return;
  if (st->done == DONE_HELD) {
    st->done = 0;
    return;
  }
  acc->inner += st_in->it;
  st_in->it = 0;
  if (st->done) {
    st_in->done = 1;
    return;
  }
  acc->outer = st->it;
  st_in->done = 0;
  st_in->growth = 0;
  st_in->maxit = window;
  st_in->eta = INFINITY;
  st_in->eta_min = INFINITY;
  st_in->tol = fmax(0.5 * ctl->tol, ratio * st->eta);
  st_in->restart = 1;
  for (int c = 0; c < 6; ++c) st_in->T0[c] = st->T0[c];
}

// Last kernel of a slot's window: counts the window and sets the slot's loop condition, so that the
// slot's while-node runs another window while its outer state is running and the window budget lasts.
// The count rises by one per window, so every slot's loop ends after at most max_windows windows.
__global__ void batch_loop_kernel(cudaGraphConditionalHandle h, const SolveState* __restrict__ st,
                                  int* __restrict__ windows, const BatchCtl* __restrict__ ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int w = *windows + 1;
  *windows = w;
  cudaGraphSetConditional(h, (st->done == 0 && w < ctl->max_windows) ? 1u : 0u);
}

}  // namespace gfp

// Peak FMA throughput (measurement hook): eight independent FMA chains per thread, values kept bounded
// (x <- a x + b with a < 1 converges), the sum stored only under a condition the values never meet so
// that the chains stay live.
template <typename R>
__global__ void fma_peak_kernel(R* __restrict__ sink, int iters, R a, R b) {
  R x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  R t = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) t += x[c];
  if (t == (R)-1) sink[blockIdx.x] = t;
}

// ------------------------------------------------------------------------------- the grid
struct gfp_grid_s {
  int n1, n2, n3;
  double h;
  cudaStream_t stream;
  Dims d;
  LaunchCfg lc64;
  double* lam = nullptr;
  double* mu = nullptr;
  double lam_h = 0, mu_h = 0;
  bool phases = false;
  int phase_gen = 0;          // incremented by gfp_set_phases and gfp_set_tiles (batch graphs bake both in)
  double* eps = nullptr;
  double2* spec = nullptr;
  double2* tw64[3] = {nullptr, nullptr, nullptr};
  double* tabA[3] = {nullptr, nullptr, nullptr};
  double* tabB[3] = {nullptr, nullptr, nullptr};
  int table_op = -1;
  double* partials = nullptr;
  int np_max = 0;
  SolveState* st = nullptr;
  SolveState* st_host = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  double* scratch = nullptr;  // small device scratch (min/max partials)
  unsigned long long* bad = nullptr;
  double* eps_save = nullptr; // second strain field for gradients
  int state_iters = 0;
  bool resume_pending = false; // gfp_set_state was called: the next solve continues from it
  // mixed precision (allocated on the first mixed solve)
  LaunchCfg lc32;
  float* lam32 = nullptr;
  float* mu32 = nullptr;
  float* eps32 = nullptr;      // FP32 correction state
  float2* vsrc = nullptr;      // FP64 residual vector T kt as the inner source, [3][S]
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  float* tabA32[3] = {nullptr, nullptr, nullptr};
  float* tabB32[3] = {nullptr, nullptr, nullptr};
  SolveState* st_in = nullptr;
  SolveState* st_in_host = nullptr;
  double* cmean = nullptr;     // FP64 mean of the correction (6)
  double* cpart = nullptr;     // its per-block partials
  bool mixed_ready = false;
  bool lam32_valid = false;
  CUtensorMap zmap64, zmap32;  // TMA descriptors of the z-tiles for lc64 / lc32
  double* rpart = nullptr;     // per-CTA sums of the real-space FP64 outer pass, 8 per CTA
  float2* ph32[3] = {nullptr, nullptr, nullptr};  // e^{i th_r / 2} per axis (stencil phase of AHC, AFB/R)
  // discrete Green operator table and the key it was built for
  double* dgo = nullptr;
  double dgo_key[6] = {0, 0, 0, 0, 0, 0};  // lambda_H, mu_H, m, valid, weight power, symmetric range
  double* xpart = nullptr;           // per-CTA partials of the x-pass (DGO residual), n2 n3 entries
  double* estar = nullptr;           // eigenstrain [6][N] while one is set (gfp_set_eigenstrain)
  double2* vprev = nullptr;          // stop_rule 1: previous T kt per point [3][S] (allocated on first use)
  double* cpart64 = nullptr;         // stop_rule 1: per-CTA criterion partials (np_max)
  bool estar_on = false;
  double E_last[6] = {0, 0, 0, 0, 0, 0};  // mean strain of the last solve (displacement output)
  bool have_solution = false;
  long long launches = 0;            // kernels launched by the current gfp_solve call
};


namespace {

const int kMaxN = 1024;

bool factor_ok(int n) {
  if (n < 1 || n > kMaxN) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// Default radix schedule of a length 2^a 3^b: radix-16 stages, then the remaining power of two as one
// stage (2, 4, 8) or as 8 x 4, then the radix-3 stages.
FftPlan make_plan(int n) {
  FftPlan p;
  p.n = n;
  p.nst = 0;
  int a = 0, b = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  int n16 = a / 4;
  const int r = a % 4;
  int tail[2] = {0, 0}, nt = 0;
  if (r == 1 && n16 > 0) { n16 -= 1; tail[nt++] = 8; tail[nt++] = 4; }
  else if (r == 1) tail[nt++] = 2;
  else if (r == 2) tail[nt++] = 4;
  else if (r == 3) tail[nt++] = 8;
  for (int i = 0; i < n16; ++i) p.radix[p.nst++] = 16;
  for (int i = 0; i < nt; ++i) p.radix[p.nst++] = tail[i];
  for (int i = 0; i < b; ++i) p.radix[p.nst++] = 3;
  return p;
}

// A radix schedule is valid when its radices are in {2, 3, 4, 8, 16}, it has at most 12 stages, and
// their product is n.
bool plan_ok(const FftPlan& p, int n) {
  if (p.n != n || p.nst < 0 || p.nst > 12) return false;
  long long prod = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int r = p.radix[s];
    if (r != 2 && r != 3 && r != 4 && r != 8 && r != 16) return false;
    prod *= r;
  }
  return prod == n;
}

// Candidate radix schedules of the shared-memory Stockham passes for the autotuner: the power of two
// split into radices 16, 8 or 4 (the remainder as one smaller stage), the radix-3 stages first or last,
// and the default; duplicates removed.
std::vector<FftPlan> plan_candidates(int n) {
  std::vector<FftPlan> out;
  auto add = [&](const FftPlan& p) {
    if (!plan_ok(p, n)) return;
    for (const FftPlan& q : out)
      if (q.nst == p.nst && std::equal(q.radix, q.radix + q.nst, p.radix)) return;
    out.push_back(p);
  };
  add(make_plan(n));
  int a = 0, b = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  const int bases[3] = {16, 8, 4};
  const int logs[3] = {4, 3, 2};
  for (int k = 0; k < 3; ++k)
    for (int threes_first = 0; threes_first < 2; ++threes_first) {
      FftPlan p;
      p.n = n;
      p.nst = 0;
      const int full = a / logs[k], rem = a % logs[k];
      if (full + (rem ? 1 : 0) + b > 12) continue;
      if (threes_first)
        for (int i = 0; i < b; ++i) p.radix[p.nst++] = 3;
      for (int i = 0; i < full; ++i) p.radix[p.nst++] = bases[k];
      if (rem) p.radix[p.nst++] = 1 << rem;
      if (!threes_first)
        for (int i = 0; i < b; ++i) p.radix[p.nst++] = 3;
      add(p);
    }
  return out;
}

int round32(int x) { return ((x + 31) / 32) * 32; }

// Tile shapes per pass, bounded by the shared memory of one CTA (two ping-pong tile copies plus
// the twiddles) and by 32-byte row segments in the strided y/z passes.
LaunchCfg make_cfg(const Dims& d, int eb) {
  const long long budget = 200 * 1024;
  auto clampt = [](int t) { return std::min(512, std::max(64, round32(t))); };
  LaunchCfg c;
  int L = std::max(1, std::min(16, 2048 / d.n1));
  L = (int)std::min<long long>(L, (long long)d.n2 * d.n3);
  while (L > 1 && (long long)(d.n1 + 6 * L * d.n1) * eb > budget) L /= 2;
  c.x_lines = L;
  c.x_threads = clampt(3 * L * d.n1 / 8);
  int yc = eb == 16 ? 8 : 16;
  while (yc > 1 && (long long)(d.n2 + 2 * yc * d.n2) * eb > budget) yc /= 2;
  c.y_cols = std::max(1, std::min(yc, d.n1h));
  c.y_threads = clampt(c.y_cols * d.n2 / 8);
  int zc = d.n3 >= 512 ? 2 : 4;  // register-FFT z-pass: 6 zc (n3 / 16) threads <= 512
  while (zc > 1 && (long long)(d.n3 + 12 * zc * d.n3) * eb > budget) zc /= 2;
  c.z_cols = std::max(1, std::min(zc, d.n1h));
  c.z_threads = clampt(6 * c.z_cols * d.n3 / 8);
  c.z_blocks = ((d.n1h + c.z_cols - 1) / c.z_cols) * d.n2;
  c.cx_lines = 0;
  c.ztmap = nullptr;
  c.z_tma = 0;
  c.x_async = 0;
  c.plan[0] = make_plan(d.n1);
  c.plan[1] = make_plan(d.n2);
  c.plan[2] = make_plan(d.n3);
  return c;
}

// cuTensorMapEncodeTiled from the driver (looked up once; null if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of a half spectrum (FP32 or FP64 complex) as reals {2P, n2, n3, 6} with z-tiles of
// `cols` columns x min(n3, 256) rows.  FP32 tiles of 8 columns (64-byte rows, the warp-shuffle z-pass)
// use the 64-byte swizzle, all others none.  Returns false if the shape is not TMA-eligible.
bool encode_ztmap(CUtensorMap* m, const void* spec, const Dims& d, int cols, int real_bytes) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || cols < 1 || (2 * cols * real_bytes) % 16 != 0 || ((uintptr_t)spec & 15) != 0) return false;
  const cuuint64_t es = (cuuint64_t)real_bytes;
  cuuint64_t dims[4] = {(cuuint64_t)(2 * d.P), (cuuint64_t)d.n2, (cuuint64_t)d.n3, 6};
  cuuint64_t strides[3] = {2 * (cuuint64_t)d.P * es, (cuuint64_t)d.n2 * 2 * d.P * es, (cuuint64_t)d.S * 2 * es};
  cuuint32_t box[4] = {(cuuint32_t)(2 * cols), 1, (cuuint32_t)std::min(d.n3, 256), 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, real_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                         const_cast<void*>(spec), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         (real_bytes == 4 && cols == 8) ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// (Re)encode the z-tile tensor map of a launch configuration; without TMA the pass falls back to
// the register-FFT kernel with ordinary loads.
void refresh_ztmap(gfp_grid g, bool mixed) {
  LaunchCfg& lc = mixed ? g->lc32 : g->lc64;
  CUtensorMap* m = mixed ? &g->zmap32 : &g->zmap64;
  lc.ztmap = encode_ztmap(m, g->spec, g->d, lc.z_cols, mixed ? 4 : 8) ? m : nullptr;
}

// Recompute the thread counts and partial-sum count after a tile change.
void finalize_cfg(const Dims& d, LaunchCfg& c) {
  auto clampt = [](int t) { return std::min(512, std::max(64, round32(t))); };
  c.x_threads = clampt(3 * c.x_lines * d.n1 / 8);
  c.y_threads = clampt(c.y_cols * d.n2 / 8);
  c.z_threads = clampt(6 * c.z_cols * d.n3 / 8);
  c.z_blocks = ((d.n1h + c.z_cols - 1) / c.z_cols) * d.n2;
}

// Per-axis tables with exact zeros (kappa from the storage index; Nyquist is kappa = -n/2)
void build_tables(int op, int n, double h, std::vector<double>& A, std::vector<double>& B) {
  A.assign(n, 0.0);
  B.assign(n, 1.0);
  const double pi = 3.14159265358979323846;
  auto md = [](long long a, long long m) { long long r = a % m; return r < 0 ? r + m : r; };
  for (int i = 0; i < n; ++i) {
    const long long kap = (i < (n + 1) / 2) ? i : i - n;
    const double th = 2.0 * pi * (double)kap / (double)n;
    switch (op) {
      case OP_F: A[i] = th / h; break;
      case OP_CD: A[i] = md(2 * kap, n) == 0 ? 0.0 : std::sin(th) / h; break;
      case OP_ACD:
        A[i] = md(2 * kap, n) == 0 ? 0.0 : std::sin(th) / h;
        B[i] = md(4 * kap - n, 2LL * n) == 0 ? 0.0 : std::cos(th);
        break;
      case OP_HC: A[i] = md(kap, n) == 0 ? 0.0 : 2.0 * std::sin(0.5 * th) / h; break;
      case OP_AHC:
      case OP_AFB_R:
      default:
        A[i] = md(kap, n) == 0 ? 0.0 : 2.0 * std::sin(0.5 * th) / h;
        B[i] = md(2 * kap - n, 2LL * n) == 0 ? 0.0 : std::cos(0.5 * th);
        break;
    }
  }
}

thread_local char g_detail[256] = "";

void note_error(cudaError_t e, int line) {
  std::snprintf(g_detail, sizeof(g_detail), "%s (%d) at gfp_api.cu:%d", cudaGetErrorString(e), (int)e, line);
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? GFP_OK : (e == cudaErrorMemoryAllocation ? GFP_ERR_OOM : GFP_ERR_CUDA); }

#define GFP_CU(call)                                  \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) {                          \
      note_error(e_, __LINE__);                       \
      return cuda_status(e_);                         \
    }                                                 \
  } while (0)

std::once_flag g_setup_once;
cudaError_t g_setup_err = cudaSuccess;

int global_setup() {
  std::call_once(g_setup_once, [] {
    g_setup_err = Passes<double>::setup();
    if (g_setup_err == cudaSuccess) g_setup_err = Passes<float>::setup();
    if (g_setup_err == cudaSuccess)
      g_setup_err = cudaFuncSetAttribute(rx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (g_setup_err == cudaSuccess)
      g_setup_err = cudaFuncSetAttribute(rz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (g_setup_err != cudaSuccess) note_error(g_setup_err, __LINE__);
  return cuda_status(g_setup_err);
}

void free_grid(gfp_grid g) {
  if (!g) return;
  cudaFree(g->lam); cudaFree(g->mu); cudaFree(g->eps); cudaFree(g->spec);
  for (int r = 0; r < 3; ++r) { cudaFree(g->tw64[r]); cudaFree(g->tabA[r]); cudaFree(g->tabB[r]); }
  cudaFree(g->partials); cudaFree(g->st); cudaFree(g->hist); cudaFree(g->scratch); cudaFree(g->bad);
  cudaFree(g->eps_save);
  cudaFree(g->lam32); cudaFree(g->mu32); cudaFree(g->eps32); cudaFree(g->vsrc);
  for (int r = 0; r < 3; ++r) { cudaFree(g->tw32[r]); cudaFree(g->tabA32[r]); cudaFree(g->tabB32[r]); }
  cudaFree(g->st_in); cudaFree(g->cmean); cudaFree(g->cpart); cudaFree(g->rpart);
  for (int r = 0; r < 3; ++r) cudaFree(g->ph32[r]);
  cudaFree(g->dgo); cudaFree(g->xpart); cudaFree(g->estar); cudaFree(g->vprev); cudaFree(g->cpart64);
  if (g->st_host) cudaFreeHost(g->st_host);
  if (g->st_in_host) cudaFreeHost(g->st_in_host);
  delete g;
}

int ensure_tables(gfp_grid g, int op) {
  if (g->table_op == op) return GFP_OK;
  const int ns[3] = {g->n1, g->n2, g->n3};
  for (int r = 0; r < 3; ++r) {
    std::vector<double> A, B;
    build_tables(op, ns[r], g->h, A, B);
    GFP_CU(cudaMemcpyAsync(g->tabA[r], A.data(), sizeof(double) * ns[r], cudaMemcpyHostToDevice, g->stream));
    GFP_CU(cudaMemcpyAsync(g->tabB[r], B.data(), sizeof(double) * ns[r], cudaMemcpyHostToDevice, g->stream));
    if (g->tabA32[r]) {
      std::vector<float> Af(A.begin(), A.end()), Bf(B.begin(), B.end());
      GFP_CU(cudaMemcpyAsync(g->tabA32[r], Af.data(), sizeof(float) * ns[r], cudaMemcpyHostToDevice, g->stream));
      GFP_CU(cudaMemcpyAsync(g->tabB32[r], Bf.data(), sizeof(float) * ns[r], cudaMemcpyHostToDevice, g->stream));
      GFP_CU(cudaStreamSynchronize(g->stream));
    }
  }
  GFP_CU(cudaStreamSynchronize(g->stream));
  g->table_op = op;
  return GFP_OK;
}

int ensure_hist(gfp_grid g, int cap) {
  if (cap <= g->hist_cap) return GFP_OK;
  cudaFree(g->hist);
  g->hist = nullptr;
  g->hist_cap = 0;
  GFP_CU(cudaMalloc(&g->hist, sizeof(double) * cap));
  g->hist_cap = cap;
  return GFP_OK;
}

// x-pass parameters of the FP64 passes: the eigenstrain while one is set
PolarParams fp64_xparams(gfp_grid g) {
  PolarParams pp;
  for (int c = 0; c < 6; ++c) pp.E[c] = 0;
  pp.lam_h = pp.mu_h = 0;
  pp.partials = nullptr;
  pp.estar = g->estar_on ? g->estar : nullptr;
  return pp;
}

void one_iteration64(gfp_grid g, const GammaParams<double>& gp, int have_delta, const LaunchCfg* lc_override = nullptr) {
  const Dims& d = g->d;
  const LaunchCfg& lc = lc_override ? *lc_override : g->lc64;
  g->launches += 5;
  const PolarParams pp = fp64_xparams(g);
  Passes<double>::pass_x(g->stream, lc, g->spec, g->eps, g->lam, g->mu, g->tw64[0], lc.plan[0], d,
                         have_delta ? PX_DELTA : 0, nullptr, nullptr, g->st, &pp);
  Passes<double>::pass_y(g->stream, lc, false, g->spec, g->tw64[1], lc.plan[1], d, g->st);
  Passes<double>::pass_z(g->stream, lc, g->spec, g->tw64[2], lc.plan[2], d, gp, g->partials, g->st, PZ_GAMMA,
                         nullptr);
  if (gp.vprev)
    reduce_crit_kernel<<<1, 1024, 0, g->stream>>>(g->partials, gp.cpart, lc.z_blocks, 1.0 / std::sqrt((double)d.N),
                                                  g->st, g->hist, g->hist_cap);
  else
    launch_reduce_eta(g->stream, g->partials, lc.z_blocks, g->st, g->hist, g->hist_cap);
  Passes<double>::pass_y(g->stream, lc, true, g->spec, g->tw64[1], lc.plan[1], d, g->st);
}

// resume: continue from the strain set by gfp_set_state; its iteration count K is taken as the
// count before the stress evaluation of that strain, so a resumed solve re-evaluates iteration K
// and then follows exactly the iterates (and counts) of an uninterrupted solve.
int solve_fp64(gfp_grid g, const gfp_scheme* sc, const double E[6], double tol, int maxit, gfp_result* out,
               bool resume) {
  int rc = ensure_tables(g, sc->op);
  if (rc) return rc;
  rc = ensure_hist(g, std::max(maxit, 1));
  if (rc) return rc;
  GammaParams<double> gp;
  for (int r = 0; r < 3; ++r) { gp.A[r] = g->tabA[r]; gp.B[r] = g->tabB[r]; }
  gp.c_mu = 1.0 / (2.0 * g->mu_h);
  gp.c_lm = (g->lam_h + g->mu_h) / (g->mu_h * (g->lam_h + 2.0 * g->mu_h));
  gp.invN = 1.0 / (double)g->d.N;
  gp.nyq_avg = (sc->op == OP_F || sc->op == OP_HC) ? 1 : 0;
  gp.half_shift = 0;
  gp.dgo = nullptr;
  // the paper's increment rule: the previous iteration's T kt per point and the criterion partials
  // (the TMA z-pass has no criterion: the register or generic kernel runs with these tiles)
  LaunchCfg lc_rule = g->lc64;
  lc_rule.z_tma = 0;
  const bool rule1 = sc->stop_rule == 1;
  if (rule1) {
    if (resume) return GFP_ERR_UNSUPPORTED;
    if (!g->vprev) GFP_CU(cudaMalloc(&g->vprev, sizeof(double2) * 3 * (size_t)g->d.S));
    if (!g->cpart64) GFP_CU(cudaMalloc(&g->cpart64, sizeof(double) * (size_t)g->np_max));
    GFP_CU(cudaMemsetAsync(g->vprev, 0, sizeof(double2) * 3 * (size_t)g->d.S, g->stream));
    gp.vprev = g->vprev;
    gp.cpart = g->cpart64;
    gp.inv_mu = 1.0 / g->mu_h;
    gp.c_g = (g->lam_h + g->mu_h) / (g->lam_h + 2.0 * g->mu_h);
  }
  SolveState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.maxit = maxit;
  s0.tol = tol;
  s0.eta = INFINITY;
  s0.eta_min = INFINITY;
  const int start_it = resume ? std::max(0, g->state_iters - 1) : 0;
  s0.it = start_it;
  if (start_it >= maxit) return GFP_ERR_ARG;
  if (!resume) {
    fill_eps_kernel<<<std::min<long long>(4096, (g->d.N + 255) / 256), 256, 0, g->stream>>>(g->eps, g->d.N, E[0], E[1],
                                                                                            E[2], E[3], E[4], E[5]);
    g->launches += 1;
  }
  *g->st_host = s0;
  GFP_CU(cudaMemcpyAsync(g->st, g->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
  int launched = 0;
  int chunk = 2;
  const int budget = maxit - start_it;
  while (launched < budget) {
    const int nb = std::min(chunk, budget - launched);
    for (int b = 0; b < nb; ++b) one_iteration64(g, gp, (launched + b) > 0 ? 1 : 0, rule1 ? &lc_rule : nullptr);
    launched += nb;
    GFP_CU(cudaGetLastError());
    GFP_CU(cudaMemcpyAsync(g->st_host, g->st, sizeof(SolveState), cudaMemcpyDeviceToHost, g->stream));
    GFP_CU(cudaStreamSynchronize(g->stream));
    if (g->st_host->done) break;
    chunk = std::min(chunk * 2, 64);
  }
  // the mean stress of the final strain by a compensated real-space sum (the k = 0 value of the
  // transform rounds at about 1e-16 of it)
  if (g->st_host->done != DONE_TIMEOUT) {
    const int mb = 512;
    double* mpart = g->scratch;  // 8 K doubles: 12 per block
    mean_stress64_kernel<<<mb, 256, 0, g->stream>>>(g->eps, g->lam, g->mu, g->estar_on ? g->estar : nullptr,
                                                    g->d.N, mpart);
    mean_stress64_final_kernel<<<1, 32, 0, g->stream>>>(mpart, mb, g->st);
    g->launches += 2;
    GFP_CU(cudaGetLastError());
    GFP_CU(cudaMemcpyAsync(g->st_host->T0, g->st->T0, sizeof(double) * 6, cudaMemcpyDeviceToHost, g->stream));
    GFP_CU(cudaStreamSynchronize(g->stream));
  }
  const SolveState& s = *g->st_host;
  g->state_iters = s.it;
  int status = GFP_OK;
  if (s.done == 2 || s.done == 0) status = GFP_ERR_NOT_CONVERGED;
  if (s.done == 3) status = GFP_ERR_DIVERGED;
  if (s.done == DONE_TIMEOUT) status = GFP_ERR_DEVICE_TIMEOUT;
  if (out) {
    out->iters = s.it;
    out->outer = 0;
    out->launches = (int)g->launches;
    out->residual = rule1 ? s.crit : s.eta;
    for (int c = 0; c < 6; ++c) out->sigma_mean[c] = s.T0[c] / (double)g->d.N;
    out->status = status;
    if (out->residual_history && out->history_cap > 0) {
      const int nh = std::min(out->history_cap, std::min(s.it, g->hist_cap));
      if (nh > 0)
        GFP_CU(cudaMemcpy(out->residual_history, g->hist, sizeof(double) * nh, cudaMemcpyDeviceToHost));
    }
  }
  return status;
}

// Real-space outer pass: stencil family of a scheme, CTA grid and count, z-transform tile width.
int res_stencil(int op) { return op == OP_CD ? RS_CD : (op == OP_ACD ? RS_ACD : RS_AFD); }
dim3 res64_grid(const Dims& d) {
  return dim3((d.n1 + kResTX - 1) / kResTX, (d.n2 + kResTY - 1) / kResTY, (d.n3 + kResTZ - 1) / kResTZ);
}
int res64_blocks(const Dims& d) {
  const dim3 g = res64_grid(d);
  return (int)(g.x * g.y * g.z);
}
int rz_cols(int n3) {
  int c = 16;
  while (c > 1 && sizeof(float2) * 2 * (size_t)c * (n3 + 1) > 200 * 1024) c /= 2;
  return c;
}
// th = 2 pi kappa / n for storage index j (kappa = j below the middle, j - n from it on: the Nyquist
// index of an even axis is kappa = -n/2), as in the wave-vector tables
double stencil_angle(int n, int j) {
  const long long kap = (j < (n + 1) / 2) ? j : (long long)j - n;
  return 2.0 * 3.14159265358979323846 * (double)kap / (double)n;
}

int ensure_mixed(gfp_grid g) {
  if (g->mixed_ready) return GFP_OK;
  const Dims& d = g->d;
  const int ns[3] = {g->n1, g->n2, g->n3};
  g->lc32 = make_cfg(d, 8);
  refresh_ztmap(g, true);
  GFP_CU(cudaMalloc(&g->lam32, sizeof(float) * d.N));
  GFP_CU(cudaMalloc(&g->mu32, sizeof(float) * d.N));
  GFP_CU(cudaMalloc(&g->eps32, sizeof(float) * 6 * d.N));
  GFP_CU(cudaMalloc(&g->vsrc, sizeof(float2) * 3 * d.S));
  for (int r = 0; r < 3; ++r) {
    GFP_CU(cudaMalloc(&g->tw32[r], sizeof(float2) * ns[r]));
    GFP_CU(cudaMalloc(&g->tabA32[r], sizeof(float) * ns[r]));
    GFP_CU(cudaMalloc(&g->tabB32[r], sizeof(float) * ns[r]));
    std::vector<double2> tw(ns[r]);
    GFP_CU(cudaMemcpy(tw.data(), g->tw64[r], sizeof(double2) * ns[r], cudaMemcpyDeviceToHost));
    std::vector<float2> twf(ns[r]);
    for (int j = 0; j < ns[r]; ++j) { twf[j].x = (float)tw[j].x; twf[j].y = (float)tw[j].y; }
    GFP_CU(cudaMemcpy(g->tw32[r], twf.data(), sizeof(float2) * ns[r], cudaMemcpyHostToDevice));
  }
  GFP_CU(cudaMalloc(&g->st_in, sizeof(SolveState)));
  GFP_CU(cudaMallocHost((void**)&g->st_in_host, sizeof(SolveState)));
  GFP_CU(cudaMalloc(&g->cmean, sizeof(double) * 6));
  GFP_CU(cudaMalloc(&g->cpart, sizeof(double) * 6 * 1024));
  GFP_CU(cudaMalloc(&g->rpart, sizeof(double) * 8 * (size_t)res64_blocks(d)));
  for (int r = 0; r < 3; ++r) {
    std::vector<float2> ph(ns[r]);
    for (int j = 0; j < ns[r]; ++j) {
      const double th = stencil_angle(ns[r], j);
      ph[j].x = (float)std::cos(0.5 * th);
      ph[j].y = (float)std::sin(0.5 * th);
    }
    GFP_CU(cudaMalloc(&g->ph32[r], sizeof(float2) * ns[r]));
    GFP_CU(cudaMemcpy(g->ph32[r], ph.data(), sizeof(float2) * ns[r], cudaMemcpyHostToDevice));
  }
  const int pz32 = g->lc32.z_blocks;
  if (pz32 > g->np_max) {
    cudaFree(g->partials);
    g->partials = nullptr;
    GFP_CU(cudaMalloc(&g->partials, sizeof(double) * pz32));
    g->np_max = pz32;
  }
  g->table_op = -1;  // refill tables, now including the FP32 copies
  g->mixed_ready = true;
  return GFP_OK;
}

template <typename R>
GammaParams<R> gamma_params(gfp_grid g, int op, const R* const* A, const R* const* B) {
  GammaParams<R> gp;
  for (int r = 0; r < 3; ++r) { gp.A[r] = A[r]; gp.B[r] = B[r]; }
  gp.c_mu = (R)(1.0 / (2.0 * g->mu_h));
  gp.c_lm = (R)((g->lam_h + g->mu_h) / (g->mu_h * (g->lam_h + 2.0 * g->mu_h)));
  gp.invN = (R)(1.0 / (double)g->d.N);
  gp.nyq_avg = (op == OP_F || op == OP_HC) ? 1 : 0;
  gp.half_shift = (op == OP_AFB_R) ? 1 : 0;
  gp.dgo = nullptr;
  return gp;
}

// Real-space FP64 outer pass (gfp_outer.cuh) on explicit buffers, for single and batched solves:
// eps += corr - mean(corr) (if corr), r = D^b C : (eps - estar), the FP64 residual and mean stress
// into st (reduce_eta decides convergence).  r (FP32 [3][N]) goes to rbuf.  Every kernel is a no-op
// while st is done (held batch slots).
void outer_pass64(cudaStream_t s, const Dims& d, double h, int op, double* eps, const double* lam, const double* mu,
                  const double* estar, const float* corr, const double* cmean, float* rbuf, double* rpart,
                  double* partials, SolveState* st, long long& launches) {
  if (corr) {
    const int cvb = (int)std::min<long long>(1024, (d.N + 255) / 256);
    apply_corr64_kernel<<<cvb, 256, 0, s>>>(eps, corr, cmean, d.N, st);
    ++launches;
  }
  const dim3 grid = res64_grid(d);
  const double inv_h = 1.0 / h;
  switch (res_stencil(op)) {
    case RS_CD: residual64_kernel<RS_CD><<<grid, kResTX * kResTY, 0, s>>>(eps, lam, mu, estar, d, inv_h, rbuf, rpart, st); break;
    case RS_ACD: residual64_kernel<RS_ACD><<<grid, kResTX * kResTY, 0, s>>>(eps, lam, mu, estar, d, inv_h, rbuf, rpart, st); break;
    default: residual64_afd_kernel<<<grid, kResTX * kResTY, 0, s>>>(eps, lam, mu, estar, d, inv_h, rbuf, rpart, st); break;
  }
  res64_sum_kernel<<<1, 256, 0, s>>>(rpart, res64_blocks(d), d.N, st, partials);
  launch_reduce_eta(s, partials, 1, st, nullptr, 0);
  launches += 3;
}

// The inner iterations' source v = T_check kt from the residual field r: FP32 transforms along x1
// (rx_kernel), x2 (the y-pass on three components) and x3 with the stencil phase (rz_kernel).
void outer_source32(cudaStream_t s, const LaunchCfg& lc32, const Dims& d, int op, const float* rbuf, float2* vsrc,
                    float2* const* tw32, float2* const* ph, const SolveState* st, long long& launches) {
  const long long nlines = (long long)d.n2 * d.n3;
  const int L = 4;
  const size_t smx = sizeof(float2) * 2 * (3 * L / 2) * (size_t)d.n1;
  rx_kernel<<<(unsigned)((nlines + L - 1) / L), 256, smx, s>>>(rbuf, vsrc, tw32[0], lc32.plan[0], d, L, st);
  Passes<float>::pass_y(s, lc32, false, vsrc, tw32[1], lc32.plan[1], d, st, 3);
  const int zc = rz_cols(d.n3);
  const size_t smz = sizeof(float2) * 2 * (size_t)zc * (d.n3 + 1);
  const bool phase = res_stencil(op) == RS_AFD;
  rz_kernel<<<dim3((d.n1h + zc - 1) / zc, d.n2, 3), 256, smz, s>>>(vsrc, tw32[2], lc32.plan[2], d, zc,
                                                                   phase ? ph[0] : nullptr, phase ? ph[1] : nullptr,
                                                                   phase ? ph[2] : nullptr, st);
  launches += 3;
}

void residual_pass64(gfp_grid g, int op, bool with_corr) {
  outer_pass64(g->stream, g->d, g->h, op, g->eps, g->lam, g->mu, g->estar_on ? g->estar : nullptr,
               with_corr ? g->eps32 : nullptr, g->cmean, reinterpret_cast<float*>(g->spec), g->rpart, g->partials,
               g->st, g->launches);
}

void inner_source32(gfp_grid g, int op) {
  outer_source32(g->stream, g->lc32, g->d, op, reinterpret_cast<const float*>(g->spec), g->vsrc, g->tw32,
                 g->ph32, g->st, g->launches);
}

// One FP32 inner iteration on the correction: delta += d_delta, sigma = C32 : delta, forward,
// v = T kt + v64, Delta = -Gamma0(v) / N, inverse.
void inner_iteration32(gfp_grid g, const GammaParams<float>& gp, int flags) {
  const Dims& d = g->d;
  g->launches += 5;
  float2* spec32 = reinterpret_cast<float2*>(g->spec);
  Passes<float>::pass_x(g->stream, g->lc32, spec32, g->eps32, g->lam32, g->mu32, g->tw32[0], g->lc32.plan[0], d, flags,
                        nullptr, nullptr, g->st_in);
  Passes<float>::pass_y(g->stream, g->lc32, false, spec32, g->tw32[1], g->lc32.plan[1], d, g->st_in);
  Passes<float>::pass_z(g->stream, g->lc32, spec32, g->tw32[2], g->lc32.plan[2], d, gp, g->partials, g->st_in, PZ_INNER,
                        g->vsrc);
  launch_reduce_eta(g->stream, g->partials, g->lc32.z_blocks, g->st_in, nullptr, 0);
  Passes<float>::pass_y(g->stream, g->lc32, true, spec32, g->tw32[1], g->lc32.plan[1], d, g->st_in);
}

const double kInnerReduction = 1e-4;  // target of one inner solve relative to the FP64 residual

// Mixed precision: FP64 outer loop (exact residual, mean strain, refinement) around FP32 inner
// iterations of the same Green-operator scheme on the correction.
int solve_mixed(gfp_grid g, const gfp_scheme* sc, const double E[6], double tol, int maxit, gfp_result* out) {
  if (sc->op == OP_F || sc->op == OP_HC || sc->op == OP_DGO) return GFP_ERR_UNSUPPORTED;
  int rc = ensure_mixed(g);
  if (rc) return rc;
  rc = ensure_tables(g, sc->op);
  if (rc) return rc;
  const Dims& d = g->d;
  const int cvb = (int)std::min<long long>(1024, (d.N + 255) / 256);
  if (!g->lam32_valid) {
    to_float_kernel<<<cvb, 256, 0, g->stream>>>(g->lam, g->lam32, d.N);
    to_float_kernel<<<cvb, 256, 0, g->stream>>>(g->mu, g->mu32, d.N);
    g->lam32_valid = true;
    g->launches += 2;
  }
  const GammaParams<float> gp32 = gamma_params<float>(g, sc->op, g->tabA32, g->tabB32);
  fill_eps_kernel<<<std::min<long long>(4096, (d.N + 255) / 256), 256, 0, g->stream>>>(g->eps, d.N, E[0], E[1], E[2],
                                                                                       E[3], E[4], E[5]);
  g->launches += 1;
  SolveState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.maxit = 1 << 30;
  s0.tol = tol;
  s0.eta = INFINITY;
  s0.eta_min = INFINITY;
  *g->st_host = s0;
  GFP_CU(cudaMemcpyAsync(g->st, g->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
  int inner_total = 0, outer = 0;
  bool with_corr = false;
  int status = GFP_ERR_NOT_CONVERGED;
  while (true) {
    residual_pass64(g, sc->op, with_corr);
    ++outer;
    GFP_CU(cudaGetLastError());
    GFP_CU(cudaMemcpyAsync(g->st_host, g->st, sizeof(SolveState), cudaMemcpyDeviceToHost, g->stream));
    GFP_CU(cudaStreamSynchronize(g->stream));
    const SolveState so = *g->st_host;
    if (so.done == 1) { status = GFP_OK; break; }
    if (so.done == 3) { status = GFP_ERR_DIVERGED; break; }
    if (so.done == DONE_TIMEOUT) { status = GFP_ERR_DEVICE_TIMEOUT; break; }
    if (inner_total >= maxit) { status = GFP_ERR_NOT_CONVERGED; break; }
    // inner solve of the correction equation from a zero correction, with the source of this residual
    inner_source32(g, sc->op);
    SolveState si = s0;
    si.maxit = maxit - inner_total;
    si.tol = std::max(0.5 * tol, kInnerReduction * so.eta);
    for (int c = 0; c < 6; ++c) si.T0[c] = so.T0[c];
    *g->st_in_host = si;
    GFP_CU(cudaMemcpyAsync(g->st_in, g->st_in_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
    int launched = 0, chunk = 4;
    while (launched < si.maxit) {
      const int nb = std::min(chunk, si.maxit - launched);
      for (int b = 0; b < nb; ++b) inner_iteration32(g, gp32, (launched + b) == 0 ? PX_ZERO : PX_DELTA);
      launched += nb;
      GFP_CU(cudaGetLastError());
      GFP_CU(cudaMemcpyAsync(g->st_in_host, g->st_in, sizeof(SolveState), cudaMemcpyDeviceToHost, g->stream));
      GFP_CU(cudaStreamSynchronize(g->stream));
      if (g->st_in_host->done) break;
      chunk = std::min(chunk * 2, 64);
    }
    inner_total += g->st_in_host->it;
    if (g->st_in_host->done == 3) { status = GFP_ERR_DIVERGED; break; }
    if (g->st_in_host->done == DONE_TIMEOUT) { status = GFP_ERR_DEVICE_TIMEOUT; break; }
    corr_mean_partial_kernel<<<cvb, 256, 0, g->stream>>>(g->eps32, d.N, g->cpart, nullptr);
    corr_mean_final_kernel<<<1, 32, 0, g->stream>>>(g->cpart, cvb, d.N, g->cmean, nullptr);
    g->launches += 2;
    // the next outer pass re-arms the FP64 state (it counts outer passes; never stops on maxit)
    g->st_host->done = 0;
    GFP_CU(cudaMemcpyAsync(g->st, g->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
    with_corr = true;
  }
  const SolveState& s = *g->st_host;
  g->state_iters = inner_total;
  if (out) {
    out->iters = inner_total;
    out->outer = outer;
    out->launches = (int)g->launches;
    out->residual = s.eta;
    for (int c = 0; c < 6; ++c) out->sigma_mean[c] = s.T0[c] / (double)d.N;
    out->status = status;
    if (out->residual_history && out->history_cap > 0) out->residual_history[0] = s.eta;
  }
  return status;
}

// Sinc weights s_j = sinc(pi j / n) of axis r raised to `power`, for omega in [0, n) (rows) and
// nu in [lo, lo + W) (columns); exact zeros where j = 0 mod n, j != 0.
void dgo_weights(int n, int lo, int W, int power, std::vector<double>& w) {
  const double pi = 3.14159265358979323846;
  w.assign((size_t)n * W, 0.0);
  for (int o = 0; o < n; ++o)
    for (int v = lo; v < lo + W; ++v) {
      const long long j = (long long)v * n + o;
      double s;
      if (j == 0) s = 1.0;
      else if (j % n == 0) s = 0.0;
      else { const double x = pi * (double)j / (double)n; s = std::sin(x) / x; }
      w[(size_t)o * W + (v - lo)] = power == 2 ? s * s : s;
    }
}

std::once_flag g_mono_once;

int ensure_dgo(gfp_grid g, int dgo_m, int power, int sym) {
  const Dims& d = g->d;
  const int ns[3] = {g->n1, g->n2, g->n3};
  int ms[3];
  for (int r = 0; r < 3; ++r) ms[r] = std::max(1, dgo_m > 0 ? dgo_m : ns[r] / 2);
  if (g->dgo && g->dgo_key[3] == 1.0 && g->dgo_key[0] == g->lam_h && g->dgo_key[1] == g->mu_h &&
      g->dgo_key[2] == (double)dgo_m && g->dgo_key[4] == (double)power && g->dgo_key[5] == (double)sym)
    return GFP_OK;
  static int mono_err = 0;
  std::call_once(g_mono_once, [] {
    int m4[3][3][3][3], m2[3][3];
    int q = 0, idx4[3][3][3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j)
        for (int p = j; p < 3; ++p)
          for (int r = p; r < 3; ++r) idx4[i][j][p][r] = q++;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int p = 0; p < 3; ++p)
          for (int r = 0; r < 3; ++r) {
            int v[4] = {i, j, p, r};
            std::sort(v, v + 4);
            m4[i][j][p][r] = idx4[v[0]][v[1]][v[2]][v[3]];
          }
    const int s2map[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) m2[a][b] = s2map[a][b];
    if (cudaMemcpyToSymbol(c_mono4, m4, sizeof(m4)) != cudaSuccess) mono_err = 1;
    if (cudaMemcpyToSymbol(c_mono2, m2, sizeof(m2)) != cudaSuccess) mono_err = 1;
  });
  if (mono_err) return GFP_ERR_CUDA;
  if (!g->dgo) GFP_CU(cudaMalloc(&g->dgo, sizeof(double) * 21 * (size_t)d.S));
  double* w[3] = {nullptr, nullptr, nullptr};
  for (int r = 0; r < 3; ++r) {
    std::vector<double> hw;
    dgo_weights(ns[r], sym ? -ms[r] - 1 : -ms[r], sym ? 2 * ms[r] + 2 : 2 * ms[r], power, hw);
    GFP_CU(cudaMalloc(&w[r], sizeof(double) * hw.size()));
    GFP_CU(cudaMemcpy(w[r], hw.data(), sizeof(double) * hw.size(), cudaMemcpyHostToDevice));
  }
  GFP_CU(cudaMemsetAsync(g->dgo, 0, sizeof(double) * 21 * (size_t)d.S, g->stream));
  // representatives: every axis folded to [0, n_r/2] and, on a cubic grid, sorted ascending (printed
  // range); every half-spectrum point (symmetric range, whose sum is even only in all axes at once)
  const bool fold = !sym;
  const bool cubic = fold && ns[0] == ns[1] && ns[1] == ns[2] && ms[0] == ms[1] && ms[1] == ms[2];
  const int F[3] = {ns[0] / 2 + 1, fold ? ns[1] / 2 + 1 : ns[1], fold ? ns[2] / 2 + 1 : ns[2]};
  std::vector<int> pts;
  for (int o3 = 0; o3 < F[2]; ++o3)
    for (int o2 = 0; o2 < F[1]; ++o2)
      for (int o1 = 0; o1 < F[0]; ++o1)
        if (!cubic || (o1 <= o2 && o2 <= o3)) pts.push_back(o1 | (o2 << 11) | (o3 << 22));
  double* rep = nullptr;
  int* dpts = nullptr;
  cudaError_t e = cudaMalloc(&rep, sizeof(double) * 21 * (size_t)F[0] * F[1] * F[2]);
  if (e == cudaSuccess) e = cudaMalloc(&dpts, sizeof(int) * pts.size());
  if (e == cudaSuccess) e = cudaMemcpy(dpts, pts.data(), sizeof(int) * pts.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int nrep = (int)pts.size();
    dgo_table_kernel<<<std::max(1, std::min(4096, (nrep + 63) / 64)), 64, 0, g->stream>>>(
        rep, dpts, nrep, d, F[0], F[1], F[2], w[0], w[1], w[2], ms[0], ms[1], ms[2], sym, g->h, g->lam_h, g->mu_h);
    const long long npts = (long long)d.n1h * d.n2 * d.n3;
    dgo_expand_kernel<<<(int)std::min<long long>(4096, (npts + 255) / 256), 256, 0, g->stream>>>(
        g->dgo, rep, d, F[0], F[1], F[2], fold ? 1 : 0, cubic ? 1 : 0);
    g->launches += 2;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  cudaFree(rep);
  cudaFree(dpts);
  for (int r = 0; r < 3; ++r) cudaFree(w[r]);
  if (e != cudaSuccess) { note_error(e, __LINE__); return cuda_status(e); }
  g->dgo_key[0] = g->lam_h;
  g->dgo_key[1] = g->mu_h;
  g->dgo_key[2] = (double)dgo_m;
  g->dgo_key[3] = 1.0;
  g->dgo_key[4] = (double)power;
  g->dgo_key[5] = (double)sym;
  return GFP_OK;
}

// Algorithm D-3D.  Polarization form (default): eps = E_bar + F+ Gamma^c F- [(C - C_H) eps]; stress form
// (as printed): eps += F+ Gamma^c F- [C : eps].  Iteration `it` forms eps^(it) in the x-pass of the next
// launch, and the residual ||eps^(it) - eps^(it-1)|| / (sqrt(N) ||E_bar||_F) is reduced right after it;
// the returned strain includes the last increment (Algorithm D-3D adds it inside the loop body).
int solve_dgo(gfp_grid g, const gfp_scheme* sc, const double E[6], double tol, int maxit, gfp_result* out) {
  const int power = sc->dgo_power == 1 ? 1 : 2;
  const bool stress_form = sc->dgo_form == 1;
  int rc = ensure_dgo(g, sc->dgo_m, power, sc->dgo_range == 1 ? 1 : 0);
  if (rc) return rc;
  rc = ensure_tables(g, OP_AFB_R);  // the DGO path does not read k-tables; keep them valid
  if (rc) return rc;
  rc = ensure_hist(g, std::max(maxit, 1));
  if (rc) return rc;
  const Dims& d = g->d;
  if (!g->xpart) GFP_CU(cudaMalloc(&g->xpart, sizeof(double) * (size_t)d.n2 * d.n3));
  GFP_CU(cudaMemsetAsync(g->xpart, 0, sizeof(double) * (size_t)d.n2 * d.n3, g->stream));
  GammaParams<double> gp = gamma_params<double>(g, OP_AFB_R, g->tabA, g->tabB);
  gp.dgo = g->dgo;
  PolarParams pp;
  for (int c = 0; c < 6; ++c) pp.E[c] = E[c];
  pp.lam_h = g->lam_h;
  pp.mu_h = g->mu_h;
  pp.partials = g->xpart;
  pp.estar = nullptr;
  const double en2 = E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + 2.0 * (E[3] * E[3] + E[4] * E[4] + E[5] * E[5]);
  const double enorm = std::sqrt(en2) * std::sqrt((double)d.N);
  fill_eps_kernel<<<(int)std::min<long long>(4096, (d.N + 255) / 256), 256, 0, g->stream>>>(g->eps, d.N, E[0], E[1],
                                                                                          E[2], E[3], E[4], E[5]);
  g->launches += 1;
  SolveState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.maxit = maxit;
  s0.tol = tol;
  s0.eta = INFINITY;
  s0.eta_min = INFINITY;
  *g->st_host = s0;
  GFP_CU(cudaMemcpyAsync(g->st, g->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
  const int np = d.n2 * d.n3;
  int launched = 0, chunk = 2;
  while (launched < maxit + 1) {
    const int nb = std::min(chunk, maxit + 1 - launched);
    for (int b = 0; b < nb; ++b) {
      const int j = launched + b;
      Passes<double>::pass_x(g->stream, g->lc64, g->spec, g->eps, g->lam, g->mu, g->tw64[0], g->lc64.plan[0], d,
                             (stress_form ? PX_DRES : PX_POLAR) | (j > 0 ? PX_DELTA : 0), nullptr, nullptr, g->st,
                             &pp);
      if (j > 0) reduce_dgo_kernel<<<1, 256, 0, g->stream>>>(g->xpart, np, enorm, g->st, g->hist, g->hist_cap);
      g->launches += j > 0 ? 5 : 4;
      Passes<double>::pass_y(g->stream, g->lc64, false, g->spec, g->tw64[1], g->lc64.plan[1], d, g->st);
      Passes<double>::pass_z(g->stream, g->lc64, g->spec, g->tw64[2], g->lc64.plan[2], d, gp, g->partials, g->st, PZ_DGO,
                             nullptr);
      Passes<double>::pass_y(g->stream, g->lc64, true, g->spec, g->tw64[1], g->lc64.plan[1], d, g->st);
    }
    launched += nb;
    GFP_CU(cudaGetLastError());
    GFP_CU(cudaMemcpyAsync(g->st_host, g->st, sizeof(SolveState), cudaMemcpyDeviceToHost, g->stream));
    GFP_CU(cudaStreamSynchronize(g->stream));
    if (g->st_host->done) break;
    chunk = std::min(chunk * 2, 64);
  }
  const SolveState s = *g->st_host;
  // mean stress of the final strain
  const int sb = (int)std::min<long long>(1024, (d.N + 255) / 256);
  stress_sum_partial_kernel<<<sb, 256, 0, g->stream>>>(g->eps, g->lam, g->mu, d.N, g->scratch);
  g->launches += 1;
  std::vector<double> part(6 * (size_t)sb);
  GFP_CU(cudaMemcpyAsync(part.data(), g->scratch, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, g->stream));
  GFP_CU(cudaStreamSynchronize(g->stream));
  g->state_iters = s.it;
  int status = GFP_OK;
  if (s.done == 2 || s.done == 0) status = GFP_ERR_NOT_CONVERGED;
  if (s.done == 3) status = GFP_ERR_DIVERGED;
  if (s.done == DONE_TIMEOUT) status = GFP_ERR_DEVICE_TIMEOUT;
  if (out) {
    out->iters = s.it;
    out->outer = 0;
    out->launches = (int)g->launches;
    out->residual = s.eta;
    for (int c = 0; c < 6; ++c) {
      double acc = 0.0;
      for (int b = 0; b < sb; ++b) acc += part[(size_t)b * 6 + c];
      out->sigma_mean[c] = acc / (double)d.N;
    }
    out->status = status;
    if (out->residual_history && out->history_cap > 0) {
      const int nh = std::min(out->history_cap, std::min(s.it, g->hist_cap));
      if (nh > 0) GFP_CU(cudaMemcpy(out->residual_history, g->hist, sizeof(double) * nh, cudaMemcpyDeviceToHost));
    }
  }
  return status;
}

bool scheme_ok(const gfp_scheme* sc) {
  return sc && sc->op >= 0 && sc->op <= OP_DGO && (sc->disc == GFP_TD || sc->disc == GFP_PCD) &&
         (sc->prec == GFP_FP64 || sc->prec == GFP_MIXED) && sc->dgo_power >= 0 && sc->dgo_power <= 2 &&
         (sc->dgo_form == 0 || sc->dgo_form == 1) && (sc->dgo_range == 0 || sc->dgo_range == 1);
}

}  // namespace

// ------------------------------------------------------------------------------- allocation-free solve
// Scratch of gfp_solve_noalloc.  It is a file-scope device array, so every GPU that loads this
// library holds it until the process exits, and every call of the entry point shares it.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

const int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

// Device address of the scratch on the current device (looked up once per device).  In host code
// g_noalloc_scratch only names a host-side stand-in, so kernels must be given this address instead.
int noalloc_scratch(void** out) {
  int dev = 0;
  GFP_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return GFP_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    GFP_CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GFP_OK;
}

// One entry of the per-axis tables (same values as build_tables).
void table_entry(int op, int n, int i, double h, double* A, double* B) {
  const double pi = 3.14159265358979323846;
  auto md = [](long long a, long long m) { long long q = a % m; return q < 0 ? q + m : q; };
  const long long kap = (i < (n + 1) / 2) ? i : i - n;
  const double th = 2.0 * pi * (double)kap / (double)n;
  *A = 0.0;
  *B = 1.0;
  switch (op) {
    case OP_F: *A = th / h; break;
    case OP_CD: *A = md(2 * kap, n) == 0 ? 0.0 : std::sin(th) / h; break;
    case OP_ACD:
      *A = md(2 * kap, n) == 0 ? 0.0 : std::sin(th) / h;
      *B = md(4 * kap - n, 2LL * n) == 0 ? 0.0 : std::cos(th);
      break;
    case OP_HC: *A = md(kap, n) == 0 ? 0.0 : 2.0 * std::sin(0.5 * th) / h; break;
    default:
      *A = md(kap, n) == 0 ? 0.0 : 2.0 * std::sin(0.5 * th) / h;
      *B = md(2 * kap - n, 2LL * n) == 0 ? 0.0 : std::cos(0.5 * th);
      break;
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// ------------------------------------------------------------------------------- C ABI
extern "C" {

const char* gfp_last_error_detail(void) { return g_detail; }

int gfp_set_fault_injection(int kind, int value) {
  if (kind != 1 || value < 0 || value > 1) return GFP_ERR_ARG;
  g_inject_tma_timeout = (unsigned)value;
  return GFP_OK;
}

const char* gfp_error_string(int status) {
  switch (status) {
    case GFP_OK: return "ok";
    case GFP_ERR_ARG: return "bad argument";
    case GFP_ERR_UNSUPPORTED_SIZE: return "unsupported grid size (each n must be 2^a 3^b and <= 1024)";
    case GFP_ERR_OOM: return "device out of memory";
    case GFP_ERR_NOT_CONVERGED: return "not converged within maxit iterations";
    case GFP_ERR_DIVERGED: return "iteration diverged";
    case GFP_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case GFP_ERR_CUDA: return "CUDA runtime error";
    case GFP_ERR_UNSUPPORTED: return "unsupported scheme/precision combination";
    default: return "unknown status";
  }
}

int gfp_create_grid(int n1, int n2, int n3, double h, void* cuda_stream, gfp_grid* out) {
  if (!out) return GFP_ERR_ARG;
  *out = nullptr;
  if (!(h > 0.0) || !std::isfinite(h)) return GFP_ERR_ARG;
  if (n1 < 1 || n2 < 1 || n3 < 1) return GFP_ERR_ARG;
  if (!factor_ok(n1) || !factor_ok(n2) || !factor_ok(n3)) return GFP_ERR_UNSUPPORTED_SIZE;
  int rc = global_setup();
  if (rc) return rc;
  gfp_grid g = new (std::nothrow) gfp_grid_s();
  if (!g) return GFP_ERR_OOM;
  g->n1 = n1; g->n2 = n2; g->n3 = n3; g->h = h;
  g->stream = (cudaStream_t)cuda_stream;
  Dims& d = g->d;
  d.n1 = n1; d.n2 = n2; d.n3 = n3;
  d.n1h = n1 / 2 + 1;
  d.P = ((d.n1h + 3) / 4) * 4;
  d.N = (long long)n1 * n2 * n3;
  d.S = (long long)n3 * n2 * d.P;
  const int ns[3] = {n1, n2, n3};
  g->lc64 = make_cfg(d, 16);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void**)&g->lam, sizeof(double) * d.N);
  A((void**)&g->mu, sizeof(double) * d.N);
  A((void**)&g->eps, sizeof(double) * 6 * d.N);
  A((void**)&g->spec, sizeof(double2) * 6 * d.S);
  for (int r = 0; r < 3; ++r) {
    A((void**)&g->tw64[r], sizeof(double2) * ns[r]);
    A((void**)&g->tabA[r], sizeof(double) * ns[r]);
    A((void**)&g->tabB[r], sizeof(double) * ns[r]);
  }
  g->np_max = d.n1h * d.n2;  // enough for any z-tile width (one column per CTA)
  A((void**)&g->partials, sizeof(double) * g->np_max);
  A((void**)&g->st, sizeof(SolveState));
  A((void**)&g->scratch, sizeof(double) * 8 * 1024);
  A((void**)&g->bad, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&g->st_host, sizeof(SolveState));
  if (e != cudaSuccess) { note_error(e, __LINE__); free_grid(g); return cuda_status(e); }
  // twiddles w_n^j = e^{-2 pi i j / n}
  const double pi = 3.14159265358979323846;
  for (int r = 0; r < 3; ++r) {
    std::vector<double2> tw(ns[r]);
    for (int j = 0; j < ns[r]; ++j) {
      const double a = -2.0 * pi * (double)j / (double)ns[r];
      tw[j].x = std::cos(a);
      tw[j].y = std::sin(a);
    }
    e = cudaMemcpy(g->tw64[r], tw.data(), sizeof(double2) * ns[r], cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_grid(g); return cuda_status(e); }
  }
  e = cudaMemsetAsync(g->spec, 0, sizeof(double2) * 6 * d.S, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) { free_grid(g); return cuda_status(e); }
  refresh_ztmap(g, false);
  *out = g;
  return GFP_OK;
}

int gfp_destroy_grid(gfp_grid g) {
  if (!g) return GFP_ERR_ARG;
  cudaStreamSynchronize(g->stream);
  free_grid(g);
  return GFP_OK;
}

int gfp_set_phases(gfp_grid g, const double* lambda, const double* mu, int where, const double* ref) {
  if (!g || !lambda || !mu || (where != 0 && where != 1)) return GFP_ERR_ARG;
  const long long N = g->d.N;
  const cudaMemcpyKind k = where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  GFP_CU(cudaMemcpyAsync(g->lam, lambda, sizeof(double) * N, k, g->stream));
  GFP_CU(cudaMemcpyAsync(g->mu, mu, sizeof(double) * N, k, g->stream));
  const int blocks = (int)std::min<long long>(1024, (N + 255) / 256);
  GFP_CU(cudaMemsetAsync(g->bad, 0, sizeof(unsigned long long), g->stream));
  phase_stats_kernel<<<blocks, 256, 0, g->stream>>>(g->lam, g->mu, N, g->scratch, g->bad);
  GFP_CU(cudaGetLastError());
  std::vector<double> mm(4 * blocks);
  unsigned long long bad = 0;
  GFP_CU(cudaMemcpyAsync(mm.data(), g->scratch, sizeof(double) * 4 * blocks, cudaMemcpyDeviceToHost, g->stream));
  GFP_CU(cudaMemcpyAsync(&bad, g->bad, sizeof(bad), cudaMemcpyDeviceToHost, g->stream));
  GFP_CU(cudaStreamSynchronize(g->stream));
  if (bad) return GFP_ERR_ARG;
  double q[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  for (int b = 0; b < blocks; ++b)
    for (int j = 0; j < 4; ++j) q[j] = std::min(q[j], mm[4 * b + j]);
  if (ref) {
    if (!std::isfinite(ref[0]) || !std::isfinite(ref[1]) || !(ref[1] > 0.0) || !(ref[0] + 2.0 * ref[1] > 0.0))
      return GFP_ERR_ARG;
    g->lam_h = ref[0];
    g->mu_h = ref[1];
  } else {
    g->lam_h = 0.5 * (q[0] + (-q[1]));
    g->mu_h = 0.5 * (q[2] + (-q[3]));
  }
  g->phases = true;
  ++g->phase_gen;
  g->lam32_valid = false;
  return GFP_OK;
}

int gfp_solve(gfp_grid g, const gfp_scheme* sc, const double E[6], double tol, int maxit, gfp_result* out) {
  if (!g || !scheme_ok(sc) || !E || !(tol >= 0.0) || maxit < 1) return GFP_ERR_ARG;
  for (int c = 0; c < 6; ++c) if (!std::isfinite(E[c])) return GFP_ERR_ARG;
  if (!g->phases) return GFP_ERR_ARG;
  // the paper's increment rule runs in FP64 for the pairings with a single real wave vector per mode
  if (sc->stop_rule != 0 && (sc->stop_rule != 1 || sc->prec != GFP_FP64 || sc->op == OP_F || sc->op == OP_HC ||
                             sc->op == OP_DGO))
    return GFP_ERR_UNSUPPORTED;
  if (g->estar_on && sc->op == OP_DGO) return GFP_ERR_UNSUPPORTED;
  for (int c = 0; c < 6; ++c) g->E_last[c] = E[c];
  g->have_solution = true;
  g->launches = 0;
  if (sc->prec == GFP_MIXED) {
    g->resume_pending = false;
    return solve_mixed(g, sc, E, tol, maxit, out);
  }
  if (sc->op == OP_DGO) {
    g->resume_pending = false;
    return solve_dgo(g, sc, E, tol, maxit, out);
  }
  const bool resume = g->resume_pending;
  g->resume_pending = false;
  return solve_fp64(g, sc, E, tol, maxit, out, resume);
}

int gfp_set_eigenstrain(gfp_grid g, const double* estar, int where) {
  if (!g || (where != 0 && where != 1)) return GFP_ERR_ARG;
  if (!estar) {
    g->estar_on = false;
    return GFP_OK;
  }
  const size_t bytes = sizeof(double) * 6 * (size_t)g->d.N;
  if (!g->estar) GFP_CU(cudaMalloc(&g->estar, bytes));
  GFP_CU(cudaMemcpyAsync(g->estar, estar, bytes, where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                         g->stream));
  GFP_CU(cudaStreamSynchronize(g->stream));
  g->estar_on = true;
  return GFP_OK;
}

int gfp_get_displacement(gfp_grid g, const gfp_scheme* sc, double* dst, int where) {
  if (!g || !scheme_ok(sc) || !dst || (where != 0 && where != 1)) return GFP_ERR_ARG;
  if (!g->have_solution) return GFP_ERR_ARG;
  if (sc->op == OP_DGO) return GFP_ERR_UNSUPPORTED;
  int rc = ensure_tables(g, sc->op);
  if (rc) return rc;
  const Dims& d = g->d;
  const size_t bytes = sizeof(double) * 3 * (size_t)d.N;
  double* out = reinterpret_cast<double*>(dst);
  if (where == 0) {
    if (!g->eps_save) GFP_CU(cudaMalloc(&g->eps_save, sizeof(double) * 6 * (size_t)d.N));
    out = g->eps_save;
  }
  const GammaParams<double> gp = gamma_params<double>(g, sc->op, g->tabA, g->tabB);
  PolarParams pp = fp64_xparams(g);
  pp.estar = nullptr;
  for (int c = 0; c < 6; ++c) pp.E[c] = g->E_last[c];
  SolveState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.maxit = 1 << 30;
  *g->st_host = s0;
  GFP_CU(cudaMemcpyAsync(g->st, g->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
  // forward transform of eps - E_bar, u^ per mode, inverse transform of its 3 components
  Passes<double>::pass_x(g->stream, g->lc64, g->spec, g->eps, g->lam, g->mu, g->tw64[0], g->lc64.plan[0], d, PX_STRAIN,
                         nullptr, nullptr, g->st, &pp);
  Passes<double>::pass_y(g->stream, g->lc64, false, g->spec, g->tw64[1], g->lc64.plan[1], d, g->st);
  Passes<double>::pass_z(g->stream, g->lc64, g->spec, g->tw64[2], g->lc64.plan[2], d, gp, g->partials, g->st, PZ_DISP,
                         nullptr);
  Passes<double>::pass_y(g->stream, g->lc64, true, g->spec, g->tw64[1], g->lc64.plan[1], d, g->st);
  Passes<double>::pass_x(g->stream, g->lc64, g->spec, out, g->lam, g->mu, g->tw64[0], g->lc64.plan[0], d,
                         PX_DELTA | PX_OUTPUT, nullptr, nullptr, g->st, &pp);
  GFP_CU(cudaGetLastError());
  if (where == 0) GFP_CU(cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, g->stream));
  GFP_CU(cudaStreamSynchronize(g->stream));
  return GFP_OK;
}

int gfp_get_strain(gfp_grid g, double* dst, int where) {
  if (!g || !dst || (where != 0 && where != 1)) return GFP_ERR_ARG;
  GFP_CU(cudaMemcpyAsync(dst, g->eps, sizeof(double) * 6 * g->d.N,
                         where == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream));
  GFP_CU(cudaStreamSynchronize(g->stream));
  return GFP_OK;
}

int gfp_effective_stiffness(gfp_grid g, const gfp_scheme* sc, double tol, int maxit, double C_eff[36], int iters[6]) {
  if (!g || !scheme_ok(sc) || !C_eff || maxit < 1) return GFP_ERR_ARG;
  if (g->estar_on) return GFP_ERR_UNSUPPORTED;
  int worst = GFP_OK;
  for (int J = 0; J < 6; ++J) {
    double E[6] = {0, 0, 0, 0, 0, 0};
    E[J] = J < 3 ? 1.0 : 0.5;
    gfp_result r;
    std::memset(&r, 0, sizeof(r));
    const int rc = gfp_solve(g, sc, E, tol, maxit, &r);
    if (rc != GFP_OK && rc != GFP_ERR_NOT_CONVERGED) return rc;
    if (rc != GFP_OK) worst = rc;
    for (int I = 0; I < 6; ++I) C_eff[I * 6 + J] = r.sigma_mean[I];
    if (iters) iters[J] = r.iters;
  }
  return worst;
}

int gfp_grad(gfp_grid g, const gfp_scheme* sc, int I, int J, double tol, int maxit, double* dl, double* dm, int where) {
  if (!g || !scheme_ok(sc) || I < 0 || I > 5 || J < 0 || J > 5 || !dl || !dm || (where != 0 && where != 1))
    return GFP_ERR_ARG;
  if (g->estar_on) return GFP_ERR_UNSUPPORTED;
  const long long N = g->d.N;
  if (!g->eps_save) GFP_CU(cudaMalloc(&g->eps_save, sizeof(double) * 6 * N));
  double E[6] = {0, 0, 0, 0, 0, 0};
  E[I] = I < 3 ? 1.0 : 0.5;
  gfp_result r;
  std::memset(&r, 0, sizeof(r));
  int rc = gfp_solve(g, sc, E, tol, maxit, &r);
  if (rc != GFP_OK) return rc;
  GFP_CU(cudaMemcpyAsync(g->eps_save, g->eps, sizeof(double) * 6 * N, cudaMemcpyDeviceToDevice, g->stream));
  // adjoint field: the transposed Gamma-iteration equals the forward one (Gamma real and symmetric),
  // so the adjoint state for C_eff,IJ is the forward solution of load J
  double EJ[6] = {0, 0, 0, 0, 0, 0};
  EJ[J] = J < 3 ? 1.0 : 0.5;
  rc = gfp_solve(g, sc, EJ, tol, maxit, &r);
  if (rc != GFP_OK) return rc;
  double *odl = dl, *odm = dm;
  double* tmp = nullptr;
  if (where == 0) {
    GFP_CU(cudaMalloc(&tmp, sizeof(double) * 2 * N));
    odl = tmp;
    odm = tmp + N;
  }
  grad_contract_kernel<<<(int)std::min<long long>(4096, (N + 255) / 256), 256, 0, g->stream>>>(g->eps_save, g->eps, N,
                                                                                             odl, odm);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && where == 0) {
    e = cudaMemcpyAsync(dl, odl, sizeof(double) * N, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dm, odm, sizeof(double) * N, cudaMemcpyDeviceToHost, g->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (tmp) cudaFree(tmp);
  return cuda_status(e);
}

int gfp_get_state(gfp_grid g, double* eps_dst, int* iters) {
  if (!g || !eps_dst) return GFP_ERR_ARG;
  int rc = gfp_get_strain(g, eps_dst, 0);
  if (rc) return rc;
  if (iters) *iters = g->state_iters;
  return GFP_OK;
}

int gfp_set_state(gfp_grid g, const double* eps_src, int iters) {
  if (!g || !eps_src || iters < 0) return GFP_ERR_ARG;
  GFP_CU(cudaMemcpyAsync(g->eps, eps_src, sizeof(double) * 6 * g->d.N, cudaMemcpyHostToDevice, g->stream));
  GFP_CU(cudaStreamSynchronize(g->stream));
  g->state_iters = iters;
  g->resume_pending = true;
  return GFP_OK;
}

int gfp_time_passes(gfp_grid g, const gfp_scheme* sc, int iters, double pass_ms[5]) {
  if (!g || !scheme_ok(sc) || iters < 1 || !pass_ms || !g->phases) return GFP_ERR_ARG;
  if (sc->op == OP_DGO) return GFP_ERR_UNSUPPORTED;
  const bool mixed = sc->prec == GFP_MIXED;
  if (mixed && (sc->op == OP_F || sc->op == OP_HC)) return GFP_ERR_UNSUPPORTED;
  int rc = mixed ? ensure_mixed(g) : GFP_OK;
  if (rc) return rc;
  rc = ensure_tables(g, sc->op);
  if (rc) return rc;
  const Dims& d = g->d;
  const GammaParams<double> gp = gamma_params<double>(g, sc->op, g->tabA, g->tabB);
  SolveState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.maxit = iters + 2;
  s0.tol = -1.0;  // never converges: every pass runs
  s0.eta = INFINITY;
  s0.eta_min = INFINITY;
  *g->st_host = s0;
  GFP_CU(cudaMemcpyAsync(g->st, g->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
  GammaParams<float> gp32;
  float2* spec32 = reinterpret_cast<float2*>(g->spec);
  if (mixed) {
    const int cvb = (int)std::min<long long>(1024, (d.N + 255) / 256);
    if (!g->lam32_valid) {
      to_float_kernel<<<cvb, 256, 0, g->stream>>>(g->lam, g->lam32, d.N);
      to_float_kernel<<<cvb, 256, 0, g->stream>>>(g->mu, g->mu32, d.N);
      g->lam32_valid = true;
    }
    gp32 = gamma_params<float>(g, sc->op, g->tabA32, g->tabB32);
    residual_pass64(g, sc->op, false);  // the FP64 residual, T(0) and the inner source
    inner_source32(g, sc->op);
    GFP_CU(cudaMemcpyAsync(g->st_host, g->st, sizeof(SolveState), cudaMemcpyDeviceToHost, g->stream));
    GFP_CU(cudaStreamSynchronize(g->stream));
    SolveState si = s0;
    for (int c = 0; c < 6; ++c) si.T0[c] = g->st_host->T0[c];
    *g->st_in_host = si;
    GFP_CU(cudaMemcpyAsync(g->st_in, g->st_in_host, sizeof(SolveState), cudaMemcpyHostToDevice, g->stream));
    inner_iteration32(g, gp32, PX_ZERO);
  }
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) GFP_CU(cudaEventCreate(&ev[i]));
  double acc[5] = {0, 0, 0, 0, 0};
  for (int it = 0; it < iters; ++it) {
    GFP_CU(cudaEventRecord(ev[0], g->stream));
    if (mixed)
      Passes<float>::pass_x(g->stream, g->lc32, spec32, g->eps32, g->lam32, g->mu32, g->tw32[0], g->lc32.plan[0], d,
                            PX_DELTA, nullptr, nullptr, g->st_in);
    else
      Passes<double>::pass_x(g->stream, g->lc64, g->spec, g->eps, g->lam, g->mu, g->tw64[0], g->lc64.plan[0], d, PX_DELTA,
                             nullptr, nullptr, g->st);
    GFP_CU(cudaEventRecord(ev[1], g->stream));
    if (mixed) Passes<float>::pass_y(g->stream, g->lc32, false, spec32, g->tw32[1], g->lc32.plan[1], d, g->st_in);
    else Passes<double>::pass_y(g->stream, g->lc64, false, g->spec, g->tw64[1], g->lc64.plan[1], d, g->st);
    GFP_CU(cudaEventRecord(ev[2], g->stream));
    if (mixed)
      Passes<float>::pass_z(g->stream, g->lc32, spec32, g->tw32[2], g->lc32.plan[2], d, gp32, g->partials, g->st_in,
                            PZ_INNER, g->vsrc);
    else
      Passes<double>::pass_z(g->stream, g->lc64, g->spec, g->tw64[2], g->lc64.plan[2], d, gp, g->partials, g->st, PZ_GAMMA,
                             nullptr);
    GFP_CU(cudaEventRecord(ev[3], g->stream));
    if (mixed) launch_reduce_eta(g->stream, g->partials, g->lc32.z_blocks, g->st_in, nullptr, 0);
    else launch_reduce_eta(g->stream, g->partials, g->lc64.z_blocks, g->st, nullptr, 0);
    GFP_CU(cudaEventRecord(ev[4], g->stream));
    if (mixed) Passes<float>::pass_y(g->stream, g->lc32, true, spec32, g->tw32[1], g->lc32.plan[1], d, g->st_in);
    else Passes<double>::pass_y(g->stream, g->lc64, true, g->spec, g->tw64[1], g->lc64.plan[1], d, g->st);
    GFP_CU(cudaEventRecord(ev[5], g->stream));
    GFP_CU(cudaEventSynchronize(ev[5]));
    for (int k = 0; k < 5; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      acc[k] += ms;
    }
  }
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  for (int k = 0; k < 5; ++k) pass_ms[k] = acc[k] / iters;
  GFP_CU(cudaGetLastError());
  return GFP_OK;
}

// Peak FMA rate of this GPU in TFLOP/s (see include/gfp.h).
int gfp_measure_fma_peak(int dtype, double* tflops) {
  if (!tflops || (dtype != 0 && dtype != 1)) return GFP_ERR_ARG;
  int dev = 0, sms = 0;
  GFP_CU(cudaGetDevice(&dev));
  GFP_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const int iters = dtype == 0 ? 4000 : 200000;
  void* sink = nullptr;
  GFP_CU(cudaMalloc(&sink, sizeof(double) * blocks));
  cudaEvent_t e0, e1;
  GFP_CU(cudaEventCreate(&e0));
  GFP_CU(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first run warms up
    cudaEventRecord(e0, 0);
    if (dtype == 0) fma_peak_kernel<double><<<blocks, threads>>>((double*)sink, iters, 0.999999, 1e-6);
    else fma_peak_kernel<float><<<blocks, threads>>>((float*)sink, iters, 0.999f, 1e-3f);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  GFP_CU(e);
  *tflops = 2.0 * 8.0 * (double)blocks * threads * (double)iters / (best * 1e-3) / 1e12;
  return GFP_OK;
}

// Allocation-free FP64 solve (see include/gfp.h).
int gfp_solve_noalloc(int n1, int n2, int n3, double h, const double* lambda, const double* mu,
                      const double* ref_lambda_mu, const gfp_scheme* sc, const double E[6], double tol, int maxit,
                      double* eps, gfp_result* out, void* cuda_stream) {
  if (!lambda || !mu || !eps || !E || !scheme_ok(sc) || !(tol >= 0.0) || maxit < 1) return GFP_ERR_ARG;
  if (!(h > 0.0) || !std::isfinite(h) || n1 < 1 || n2 < 1 || n3 < 1) return GFP_ERR_ARG;
  for (int c = 0; c < 6; ++c) if (!std::isfinite(E[c])) return GFP_ERR_ARG;
  if (sc->op == OP_DGO || sc->prec != GFP_FP64 || sc->stop_rule != 0) return GFP_ERR_UNSUPPORTED;
  if (!factor_ok(n1) || !factor_ok(n2) || !factor_ok(n3)) return GFP_ERR_UNSUPPORTED_SIZE;
  Dims d;
  d.n1 = n1; d.n2 = n2; d.n3 = n3;
  d.n1h = n1 / 2 + 1;
  d.P = ((d.n1h + 3) / 4) * 4;
  d.N = (long long)n1 * n2 * n3;
  d.S = (long long)n3 * n2 * d.P;
  const LaunchCfg lc = make_cfg(d, 16);
  const int ns[3] = {n1, n2, n3};
  const int sblocks = 256;  // phase statistics partials
  // scratch layout: spectrum, twiddles, tables, residual partials, state, phase statistics
  size_t off = 0;
  const size_t o_spec = off; off = align256(off + sizeof(double2) * 6 * (size_t)d.S);
  size_t o_tw[3], o_A[3], o_B[3];
  for (int r = 0; r < 3; ++r) { o_tw[r] = off; off = align256(off + sizeof(double2) * ns[r]); }
  for (int r = 0; r < 3; ++r) { o_A[r] = off; off = align256(off + sizeof(double) * ns[r]); }
  for (int r = 0; r < 3; ++r) { o_B[r] = off; off = align256(off + sizeof(double) * ns[r]); }
  const size_t o_part = off; off = align256(off + sizeof(double) * (size_t)lc.z_blocks);
  const size_t o_st = off; off = align256(off + sizeof(SolveState));
  const size_t o_mm = off; off = align256(off + sizeof(double) * 4 * sblocks);
  const size_t o_bad = off; off = align256(off + sizeof(unsigned long long));
  if (off > kNoAllocScratchBytes) {
    std::snprintf(g_detail, sizeof(g_detail),
                  "grid %dx%dx%d needs %zu bytes of scratch; the allocation-free entry point holds %zu", n1, n2, n3,
                  off, kNoAllocScratchBytes);
    return GFP_ERR_UNSUPPORTED_SIZE;
  }
  int rc = global_setup();
  if (rc) return rc;
  void* base = nullptr;
  rc = noalloc_scratch(&base);
  if (rc) return rc;
  unsigned char* sb = static_cast<unsigned char*>(base);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  double2* spec = reinterpret_cast<double2*>(sb + o_spec);
  double* partials = reinterpret_cast<double*>(sb + o_part);
  SolveState* st = reinterpret_cast<SolveState*>(sb + o_st);
  double2* tw[3];
  GammaParams<double> gp;
  // twiddles and wave-vector tables, staged through a small host buffer
  const double pi = 3.14159265358979323846;
  for (int r = 0; r < 3; ++r) {
    tw[r] = reinterpret_cast<double2*>(sb + o_tw[r]);
    double* A = reinterpret_cast<double*>(sb + o_A[r]);
    double* B = reinterpret_cast<double*>(sb + o_B[r]);
    gp.A[r] = A;
    gp.B[r] = B;
    for (int j0 = 0; j0 < ns[r]; j0 += 64) {
      double2 t64[64];
      double a64[64], b64[64];
      const int cnt = std::min(64, ns[r] - j0);
      for (int j = 0; j < cnt; ++j) {
        const double ang = -2.0 * pi * (double)(j0 + j) / (double)ns[r];
        t64[j].x = std::cos(ang);
        t64[j].y = std::sin(ang);
        table_entry(sc->op, ns[r], j0 + j, h, &a64[j], &b64[j]);
      }
      GFP_CU(cudaMemcpyAsync(tw[r] + j0, t64, sizeof(double2) * cnt, cudaMemcpyHostToDevice, stream));
      GFP_CU(cudaMemcpyAsync(A + j0, a64, sizeof(double) * cnt, cudaMemcpyHostToDevice, stream));
      GFP_CU(cudaMemcpyAsync(B + j0, b64, sizeof(double) * cnt, cudaMemcpyHostToDevice, stream));
      GFP_CU(cudaStreamSynchronize(stream));
    }
  }
  // reference medium: given, or 1/2 (min + max) of each Lame constant; invalid moduli are rejected
  double lam_h, mu_h;
  {
    double* mm = reinterpret_cast<double*>(sb + o_mm);
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(sb + o_bad);
    GFP_CU(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), stream));
    phase_stats_kernel<<<sblocks, 256, 0, stream>>>(lambda, mu, d.N, mm, bad);
    GFP_CU(cudaGetLastError());
    double mmh[4 * sblocks];
    unsigned long long badh = 0;
    GFP_CU(cudaMemcpyAsync(mmh, mm, sizeof(mmh), cudaMemcpyDeviceToHost, stream));
    GFP_CU(cudaMemcpyAsync(&badh, bad, sizeof(badh), cudaMemcpyDeviceToHost, stream));
    GFP_CU(cudaStreamSynchronize(stream));
    if (badh) return GFP_ERR_ARG;
    double q[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
    for (int b = 0; b < sblocks; ++b)
      for (int j = 0; j < 4; ++j) q[j] = std::min(q[j], mmh[4 * b + j]);
    if (ref_lambda_mu) {
      if (!std::isfinite(ref_lambda_mu[0]) || !std::isfinite(ref_lambda_mu[1]) || !(ref_lambda_mu[1] > 0.0) ||
          !(ref_lambda_mu[0] + 2.0 * ref_lambda_mu[1] > 0.0))
        return GFP_ERR_ARG;
      lam_h = ref_lambda_mu[0];
      mu_h = ref_lambda_mu[1];
    } else {
      lam_h = 0.5 * (q[0] - q[1]);
      mu_h = 0.5 * (q[2] - q[3]);
    }
  }
  gp.c_mu = 1.0 / (2.0 * mu_h);
  gp.c_lm = (lam_h + mu_h) / (mu_h * (lam_h + 2.0 * mu_h));
  gp.invN = 1.0 / (double)d.N;
  gp.nyq_avg = (sc->op == OP_F || sc->op == OP_HC) ? 1 : 0;
  gp.half_shift = 0;
  gp.dgo = nullptr;
  // the shared scratch keeps the previous call's contents: clear the spectrum, reset the state
  GFP_CU(cudaMemsetAsync(spec, 0, sizeof(double2) * 6 * (size_t)d.S, stream));
  fill_eps_kernel<<<(int)std::min<long long>(4096, (d.N + 255) / 256), 256, 0, stream>>>(eps, d.N, E[0], E[1], E[2],
                                                                                        E[3], E[4], E[5]);
  SolveState sh;
  std::memset(&sh, 0, sizeof(sh));
  sh.maxit = maxit;
  sh.tol = tol;
  sh.eta = INFINITY;
  sh.eta_min = INFINITY;
  GFP_CU(cudaMemcpyAsync(st, &sh, sizeof(SolveState), cudaMemcpyHostToDevice, stream));
  GFP_CU(cudaStreamSynchronize(stream));
  int launched = 0, chunk = 2;
  while (launched < maxit) {
    const int nb = std::min(chunk, maxit - launched);
    for (int b = 0; b < nb; ++b) {
      const int flags = (launched + b) > 0 ? PX_DELTA : 0;
      Passes<double>::pass_x(stream, lc, spec, eps, lambda, mu, tw[0], lc.plan[0], d, flags, nullptr, nullptr, st);
      Passes<double>::pass_y(stream, lc, false, spec, tw[1], lc.plan[1], d, st);
      Passes<double>::pass_z(stream, lc, spec, tw[2], lc.plan[2], d, gp, partials, st, PZ_GAMMA, nullptr);
      launch_reduce_eta(stream, partials, lc.z_blocks, st, nullptr, 0);
      Passes<double>::pass_y(stream, lc, true, spec, tw[1], lc.plan[1], d, st);
    }
    launched += nb;
    GFP_CU(cudaGetLastError());
    GFP_CU(cudaMemcpyAsync(&sh, st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream));
    GFP_CU(cudaStreamSynchronize(stream));
    if (sh.done) break;
    chunk = std::min(chunk * 2, 64);
  }
  int status = GFP_OK;
  if (sh.done == 2 || sh.done == 0) status = GFP_ERR_NOT_CONVERGED;
  if (sh.done == 3) status = GFP_ERR_DIVERGED;
  if (out) {
    out->iters = sh.it;
    out->outer = 0;
    out->launches = 2 + 5 * launched;  // phase statistics and strain fill, then five kernels per iteration
    out->residual = sh.eta;
    for (int c = 0; c < 6; ++c) out->sigma_mean[c] = sh.T0[c] / (double)d.N;
    out->status = status;
  }
  return status;
}

// Autotuner: time candidate tile shapes of each pass (register-FFT x-pass lines, y and z tile
// widths) on this grid and keep the fastest; tiles_out receives {x lines, y columns, z columns}.
int gfp_tune(gfp_grid g, const gfp_scheme* sc, int iters, int tiles_out[3]) {
  if (!g || !scheme_ok(sc) || iters < 1 || !g->phases) return GFP_ERR_ARG;
  if (sc->op == OP_DGO) return GFP_ERR_UNSUPPORTED;
  const bool mixed = sc->prec == GFP_MIXED;
  if (mixed && (sc->op == OP_F || sc->op == OP_HC)) return GFP_ERR_UNSUPPORTED;
  double dummy[5];
  int rc = gfp_time_passes(g, sc, 1, dummy);  // prepares state, tables and (mixed) the inner source
  if (rc) return rc;
  const Dims& d = g->d;
  const GammaParams<double> gp = gamma_params<double>(g, sc->op, g->tabA, g->tabB);
  GammaParams<float> gp32;
  if (mixed) gp32 = gamma_params<float>(g, sc->op, g->tabA32, g->tabB32);
  float2* spec32 = reinterpret_cast<float2*>(g->spec);
  LaunchCfg& lc = mixed ? g->lc32 : g->lc64;
  const int eb = mixed ? 8 : 16;
  const long long budget = 200 * 1024;
  cudaEvent_t e0, e1;
  GFP_CU(cudaEventCreate(&e0));
  GFP_CU(cudaEventCreate(&e1));
  auto run = [&](int pass, const LaunchCfg& c) -> float {
    cudaEventRecord(e0, g->stream);
    for (int i = 0; i < iters; ++i) {
      if (pass == 0) {
        if (mixed)
          Passes<float>::pass_x(g->stream, c, spec32, g->eps32, g->lam32, g->mu32, g->tw32[0], c.plan[0], d, PX_DELTA,
                                nullptr, nullptr, g->st_in);
        else
          Passes<double>::pass_x(g->stream, c, g->spec, g->eps, g->lam, g->mu, g->tw64[0], c.plan[0], d, PX_DELTA,
                                 nullptr, nullptr, g->st);
      } else if (pass == 1) {
        if (mixed) Passes<float>::pass_y(g->stream, c, false, spec32, g->tw32[1], c.plan[1], d, g->st_in);
        else Passes<double>::pass_y(g->stream, c, false, g->spec, g->tw64[1], c.plan[1], d, g->st);
      } else {
        if (mixed)
          Passes<float>::pass_z(g->stream, c, spec32, g->tw32[2], c.plan[2], d, gp32, g->partials, g->st_in,
                                PZ_INNER, g->vsrc);
        else
          Passes<double>::pass_z(g->stream, c, g->spec, g->tw64[2], c.plan[2], d, gp, g->partials, g->st, PZ_GAMMA,
                                 nullptr);
      }
    }
    cudaEventRecord(e1, g->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return cudaGetLastError() == cudaSuccess ? ms : 1e30f;
  };
  const int ycmax = mixed ? cy_cols_max<float>(d.n2) : cy_cols_max<double>(d.n2);
  auto zc_ok = [&](int cc) { return mixed ? cz_cols_ok<float>(d.n3, cc) : cz_cols_ok<double>(d.n3, cc); };
  // x-pass lines (register-FFT sizes only)
  {
    const int cands[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
    LaunchCfg best = lc;
    float bt = run(0, lc);
    for (int L : cands) {
      for (int xa = 0; xa < 2; ++xa) {
        LaunchCfg c = lc;
        c.cx_lines = L;
        c.x_async = xa;
        const float t = run(0, c);
        if (t < bt) { bt = t; best = c; }
      }
    }
    lc = best;
  }
  {
    const int cands[] = {2, 4, 8, 16, 32};
    LaunchCfg best = lc;
    float bt = run(1, lc);
    for (int cc : cands) {
      if (cc > ycmax || cc > d.n1h || (long long)(d.n2 + 2 * cc * d.n2) * eb > budget) continue;
      LaunchCfg c = lc;
      c.y_cols = cc;
      finalize_cfg(d, c);
      const float t = run(1, c);
      if (t < bt) { bt = t; best = c; }
    }
    lc = best;
  }
  {
    const int cands[] = {1, 2, 4, 8, 16};
    LaunchCfg best = lc;
    float bt = run(2, lc);
    CUtensorMap cand_map;
    for (int cc : cands) {
      if (!zc_ok(cc) || cc > d.n1h || (long long)(d.n3 + 12 * cc * d.n3) * eb > budget) continue;
      for (int use_tma = 0; use_tma < 2; ++use_tma) {
        LaunchCfg c = lc;
        c.z_cols = cc;
        c.z_tma = use_tma;
        finalize_cfg(d, c);
        c.ztmap = (use_tma && encode_ztmap(&cand_map, g->spec, d, cc, mixed ? 4 : 8)) ? &cand_map : nullptr;
        if (use_tma && !c.ztmap) continue;
        if (use_tma && !(mixed ? cz_tma_ok<float>(d.n3, cc) : cz_tma_ok<double>(d.n3, cc))) continue;
        const float t = run(2, c);
        if (t < bt) { bt = t; best = c; }
      }
    }
    lc = best;
    refresh_ztmap(g, mixed);
  }
  // radix schedules of the shared-memory Stockham passes, on the axes without a register-FFT plan
  {
    const int ns[3] = {d.n1, d.n2, d.n3};
    for (int r = 0; r < 3; ++r) {
      if (has_register_plan(ns[r])) continue;
      const std::vector<FftPlan> cands = plan_candidates(ns[r]);
      if (cands.size() < 2) continue;
      LaunchCfg best = lc;
      float bt = run(r, lc);
      for (const FftPlan& p : cands) {
        LaunchCfg c = lc;
        c.plan[r] = p;
        const float t = run(r, c);
        if (t < bt) { bt = t; best = c; }
      }
      lc = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tiles_out) {
    tiles_out[0] = lc.x_async ? -lc.cx_lines : lc.cx_lines;
    tiles_out[1] = lc.y_cols;
    tiles_out[2] = lc.z_tma ? -lc.z_cols : lc.z_cols;
  }
  GFP_CU(cudaGetLastError());
  return GFP_OK;
}

// Apply tile shapes (e.g. from a tuning cache): {x lines (0 = default), y columns, z columns}.
int gfp_set_tiles(gfp_grid g, int prec, const int tiles[3]) {
  if (!g || !tiles || (prec != GFP_FP64 && prec != GFP_MIXED)) return GFP_ERR_ARG;
  if (prec == GFP_MIXED) {
    int rc = ensure_mixed(g);
    if (rc) return rc;
  }
  const Dims& d = g->d;
  const bool mixed = prec == GFP_MIXED;
  const int eb = mixed ? 8 : 16;
  const long long budget = 200 * 1024;
  const int ycmax = mixed ? cy_cols_max<float>(d.n2) : cy_cols_max<double>(d.n2);
  const int zc = tiles[2] < 0 ? -tiles[2] : tiles[2];
  const bool zc_ok = mixed ? cz_cols_ok<float>(d.n3, zc) : cz_cols_ok<double>(d.n3, zc);
  const int xl = tiles[0] < 0 ? -tiles[0] : tiles[0];
  if (xl > 16 || tiles[1] < 1 || tiles[1] > ycmax || tiles[1] > d.n1h || zc < 1 ||
      !zc_ok || zc > d.n1h || (long long)(d.n2 + 2 * tiles[1] * d.n2) * eb > budget ||
      (long long)(d.n3 + 12 * zc * d.n3) * eb > budget)
    return GFP_ERR_ARG;
  LaunchCfg& lc = mixed ? g->lc32 : g->lc64;
  lc.cx_lines = xl;
  lc.x_async = tiles[0] < 0 ? 1 : 0;
  lc.y_cols = tiles[1];
  lc.z_cols = zc;
  lc.z_tma = tiles[2] < 0 ? 1 : 0;
  finalize_cfg(d, lc);
  refresh_ztmap(g, mixed);
  ++g->phase_gen;
  return GFP_OK;
}

// Radix schedules of the shared-memory Stockham passes (one per axis) for one precision.
int gfp_get_plans(gfp_grid g, int prec, int radix_out[36], int nst_out[3]) {
  if (!g || !radix_out || !nst_out || (prec != GFP_FP64 && prec != GFP_MIXED)) return GFP_ERR_ARG;
  const LaunchCfg& lc = prec == GFP_MIXED ? g->lc32 : g->lc64;
  for (int r = 0; r < 3; ++r) {
    nst_out[r] = lc.plan[r].nst;
    for (int s = 0; s < 12; ++s) radix_out[12 * r + s] = s < lc.plan[r].nst ? lc.plan[r].radix[s] : 0;
  }
  return GFP_OK;
}

int gfp_set_plans(gfp_grid g, int prec, const int radix[36], const int nst[3]) {
  if (!g || !radix || !nst || (prec != GFP_FP64 && prec != GFP_MIXED)) return GFP_ERR_ARG;
  if (prec == GFP_MIXED) {
    int rc = ensure_mixed(g);
    if (rc) return rc;
  }
  const int ns[3] = {g->n1, g->n2, g->n3};
  FftPlan p[3];
  for (int r = 0; r < 3; ++r) {
    if (nst[r] < 0 || nst[r] > 12) return GFP_ERR_ARG;
    p[r].n = ns[r];
    p[r].nst = nst[r];
    for (int s = 0; s < 12; ++s) p[r].radix[s] = s < nst[r] ? radix[12 * r + s] : 0;
    if (!plan_ok(p[r], ns[r])) return GFP_ERR_ARG;
  }
  LaunchCfg& lc = prec == GFP_MIXED ? g->lc32 : g->lc64;
  for (int r = 0; r < 3; ++r) lc.plan[r] = p[r];
  ++g->phase_gen;
  return GFP_OK;
}

}  // extern "C"

// ---- batched homogenization: every (microstructure, Voigt load) pair is a slot with its own state.
// The batch is one CUDA graph of one while-node per slot; a slot's loop body is one window (the FP64
// residual pass when the inner solve has reached its target, then `window` FP32 inner iterations), and
// its last kernel decides on the device whether the slot loops again.  One graph launch solves the
// whole batch: no host round trip between windows, and a finished slot stops launching.
namespace {

struct BatchSlot {
  gfp_grid g;
  int load;
  double* eps = nullptr;
  float* eps32 = nullptr;
  double2* spec = nullptr;
  float2* vsrc = nullptr;
  double* partials = nullptr;
  SolveState* st = nullptr;
  SolveState* st_in = nullptr;
  double* cmean = nullptr;
  double* cpart = nullptr;
  BatchAcc* acc = nullptr;
  cudaStream_t stream = nullptr;
  LaunchCfg lc64, lc32;
  CUtensorMap zm64, zm32;
  double* rpart = nullptr;  // per-CTA sums of the real-space outer pass
};

void free_slot(BatchSlot& s) {
  cudaFree(s.eps); cudaFree(s.eps32); cudaFree(s.spec); cudaFree(s.vsrc); cudaFree(s.partials);
  cudaFree(s.st); cudaFree(s.st_in); cudaFree(s.cmean); cudaFree(s.cpart); cudaFree(s.acc); cudaFree(s.rpart);
  if (s.stream) cudaStreamDestroy(s.stream);
}

constexpr int kBatchWindow = 32;

void slot_window(BatchSlot& s, int op, const GammaParams<float>& gp32, const BatchCtl* ctl, const int* windows,
                 int window) {
  gfp_grid g = s.g;
  const Dims& d = g->d;
  cudaStream_t st = s.stream;
  const int cvb = (int)std::min<long long>(1024, (d.N + 255) / 256);
  batch_init_kernel<<<(int)std::min<long long>(4096, (6 * d.N + 255) / 256), 256, 0, st>>>(
      s.eps, s.eps32, d.N, s.load, s.st, s.st_in, s.acc, s.cmean, windows, ctl);
  batch_gate_kernel<<<1, 32, 0, st>>>(s.st, s.st_in, window);
  // the FP64 outer pass and the inner source: no-ops while the slot's outer state is held or done
  long long launches = 0;
  outer_pass64(st, d, g->h, op, s.eps, g->lam, g->mu, nullptr, s.eps32, s.cmean, reinterpret_cast<float*>(s.spec),
               s.rpart, s.partials, s.st, launches);
  outer_source32(st, s.lc32, d, op, reinterpret_cast<const float*>(s.spec), s.vsrc, g->tw32, g->ph32, s.st,
                 launches);
  batch_arm_kernel<<<1, 32, 0, st>>>(s.st, s.st_in, s.acc, ctl, kInnerReduction, window);
  float2* spec32 = reinterpret_cast<float2*>(s.spec);
  for (int k = 0; k < window; ++k) {
    Passes<float>::pass_x(st, s.lc32, spec32, s.eps32, g->lam32, g->mu32, g->tw32[0], s.lc32.plan[0], d, PX_DELTA,
                          nullptr, nullptr, s.st_in);
    Passes<float>::pass_y(st, s.lc32, false, spec32, g->tw32[1], s.lc32.plan[1], d, s.st_in);
    Passes<float>::pass_z(st, s.lc32, spec32, g->tw32[2], s.lc32.plan[2], d, gp32, s.partials, s.st_in, PZ_INNER, s.vsrc);
    launch_reduce_eta(st, s.partials, s.lc32.z_blocks, s.st_in, nullptr, 0);
    Passes<float>::pass_y(st, s.lc32, true, spec32, g->tw32[1], s.lc32.plan[1], d, s.st_in);
  }
  corr_mean_partial_kernel<<<cvb, 256, 0, st>>>(s.eps32, d.N, s.cpart, s.st_in);
  corr_mean_final_kernel<<<1, 32, 0, st>>>(s.cpart, cvb, d.N, s.cmean, s.st_in);
}

}  // namespace

struct gfp_batch_s {
  std::vector<gfp_grid> grids;
  std::vector<int> gens;          // the grids' phase_gen when the graph was built
  gfp_scheme sc;
  std::vector<BatchSlot> slots;
  BatchCtl* ctl = nullptr;        // device
  int* windows = nullptr;         // device, windows run per slot
  cudaStream_t main = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void batch_free_graph(gfp_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void batch_free(gfp_batch b) {
  batch_free_graph(b);
  if (b->main) cudaStreamDestroy(b->main);
  cudaFree(b->ctl);
  cudaFree(b->windows);
  for (auto& s : b->slots) free_slot(s);
  delete b;
}

// The batch graph: one while-node per slot, its body captured from the slot's stream.
cudaError_t batch_build_graph(gfp_batch b) {
  batch_free_graph(b);
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  for (size_t i = 0; i < b->slots.size() && e == cudaSuccess; ++i) {
    BatchSlot& s = b->slots[i];
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) break;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) break;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    const GammaParams<float> gp32 = gamma_params<float>(s.g, b->sc.op, s.g->tabA32, s.g->tabB32);
    slot_window(s, b->sc.op, gp32, b->ctl, b->windows + i, kBatchWindow);
    batch_loop_kernel<<<1, 32, 0, s.stream>>>(h, s.st, b->windows + i, b->ctl);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(s.stream, &captured);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  for (size_t i = 0; i < b->grids.size(); ++i) b->gens[i] = b->grids[i]->phase_gen;
  return e;
}

// FP32 Lame fields, tables and twiddles of the batch's grids (shared by the grid's six slots).
int batch_prepare_grids(gfp_grid* grids, int count, int op) {
  for (int i = 0; i < count; ++i) {
    gfp_grid g = grids[i];
    int rc = ensure_mixed(g);
    if (rc) return rc;
    rc = ensure_tables(g, op);
    if (rc) return rc;
    const int cvb = (int)std::min<long long>(1024, (g->d.N + 255) / 256);
    if (!g->lam32_valid) {
      to_float_kernel<<<cvb, 256, 0, g->stream>>>(g->lam, g->lam32, g->d.N);
      to_float_kernel<<<cvb, 256, 0, g->stream>>>(g->mu, g->mu32, g->d.N);
      g->lam32_valid = true;
    }
    GFP_CU(cudaStreamSynchronize(g->stream));
  }
  return GFP_OK;
}

}  // namespace

extern "C" {

int gfp_batch_create(int count, gfp_grid* grids, const gfp_scheme* sc, gfp_batch* out) {
  if (!out) return GFP_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !grids || !scheme_ok(sc)) return GFP_ERR_ARG;
  if (sc->prec != GFP_MIXED || sc->op == OP_F || sc->op == OP_HC || sc->op == OP_DGO || sc->stop_rule != 0)
    return GFP_ERR_UNSUPPORTED;
  for (int i = 0; i < count; ++i)
    if (!grids[i] || !grids[i]->phases) return GFP_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (grids[i]->estar_on) return GFP_ERR_UNSUPPORTED;
  int rc = batch_prepare_grids(grids, count, sc->op);
  if (rc) return rc;
  gfp_batch b = new gfp_batch_s();
  b->grids.assign(grids, grids + count);
  b->gens.assign(count, 0);
  b->sc = *sc;
  const int nslots = count * 6;
  b->slots.resize(nslots);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  for (int i = 0; i < count && e == cudaSuccess; ++i)
    for (int J = 0; J < 6; ++J) {
      BatchSlot& s = b->slots[i * 6 + J];
      gfp_grid g = grids[i];
      const Dims& d = g->d;
      s.g = g;
      s.load = J;
      A((void**)&s.eps, sizeof(double) * 6 * d.N);
      A((void**)&s.eps32, sizeof(float) * 6 * d.N);
      A((void**)&s.spec, sizeof(double2) * 6 * d.S);
      A((void**)&s.vsrc, sizeof(float2) * 3 * d.S);
      A((void**)&s.partials, sizeof(double) * (size_t)d.n1h * d.n2);
      A((void**)&s.st, sizeof(SolveState));
      A((void**)&s.st_in, sizeof(SolveState));
      A((void**)&s.cmean, sizeof(double) * 6);
      A((void**)&s.cpart, sizeof(double) * 6 * 1024);
      A((void**)&s.acc, sizeof(BatchAcc));
      A((void**)&s.rpart, sizeof(double) * 8 * (size_t)res64_blocks(d));
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) break;
      s.lc64 = g->lc64;
      s.lc32 = g->lc32;
      s.lc64.ztmap = encode_ztmap(&s.zm64, s.spec, d, s.lc64.z_cols, 8) ? &s.zm64 : nullptr;
      s.lc32.ztmap = encode_ztmap(&s.zm32, s.spec, d, s.lc32.z_cols, 4) ? &s.zm32 : nullptr;
    }
  A((void**)&b->ctl, sizeof(BatchCtl));
  A((void**)&b->windows, sizeof(int) * nslots);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = batch_build_graph(b);
  if (e != cudaSuccess) {
    note_error(e, __LINE__);
    batch_free(b);
    return cuda_status(e);
  }
  *out = b;
  return GFP_OK;
}

int gfp_batch_solve(gfp_batch b, double tol, int maxit, double* C_eff_out, int* iters_out) {
  if (!b || !(tol > 0.0) || maxit < 1 || !C_eff_out) return GFP_ERR_ARG;
  const int count = (int)b->grids.size();
  const int nslots = (int)b->slots.size();
  int rc = batch_prepare_grids(b->grids.data(), count, b->sc.op);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  // phases or tiles changed since the graph was built: its kernels hold the old reference medium and
  // launch shapes, so build it again
  bool stale = false;
  for (int i = 0; i < count; ++i) stale = stale || b->gens[i] != b->grids[i]->phase_gen;
  if (stale) {
    for (auto& s : b->slots) {
      s.lc64 = s.g->lc64;
      s.lc32 = s.g->lc32;
      const Dims& d = s.g->d;
      s.lc64.ztmap = encode_ztmap(&s.zm64, s.spec, d, s.lc64.z_cols, 8) ? &s.zm64 : nullptr;
      s.lc32.ztmap = encode_ztmap(&s.zm32, s.spec, d, s.lc32.z_cols, 4) ? &s.zm32 : nullptr;
    }
    e = batch_build_graph(b);
  }
  const BatchCtl ctl{tol, std::max(1, (maxit + kBatchWindow - 1) / kBatchWindow)};
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, b->main);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->windows, 0, sizeof(int) * nslots, b->main);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->main);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->main);
  rc = GFP_OK;
  if (e == cudaSuccess) {
    for (int i = 0; i < count && e == cudaSuccess; ++i)
      for (int J = 0; J < 6; ++J) {
        BatchSlot& s = b->slots[i * 6 + J];
        SolveState so, si;
        BatchAcc acc;
        e = cudaMemcpy(&so, s.st, sizeof(so), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&si, s.st_in, sizeof(si), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&acc, s.acc, sizeof(acc), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        for (int I = 0; I < 6; ++I) C_eff_out[(size_t)i * 36 + I * 6 + J] = so.T0[I] / (double)s.g->d.N;
        if (iters_out) iters_out[i * 6 + J] = acc.inner + (so.done ? 0 : si.it);
        // slots still running after the budget: the last outer pass holds their best FP64 state
        if (so.done == 0 && rc == GFP_OK) rc = GFP_ERR_NOT_CONVERGED;
        if (so.done == 3 && (rc == GFP_OK || rc == GFP_ERR_NOT_CONVERGED)) rc = GFP_ERR_DIVERGED;
        if (so.done == DONE_TIMEOUT) rc = GFP_ERR_DEVICE_TIMEOUT;
      }
  }
  if (e != cudaSuccess) {
    note_error(e, __LINE__);
    rc = cuda_status(e);
  }
  return rc;
}

int gfp_batch_destroy(gfp_batch b) {
  if (!b) return GFP_ERR_ARG;
  cudaStreamSynchronize(b->main);
  batch_free(b);
  return GFP_OK;
}

int gfp_solve_batch(int count, gfp_grid* grids, const gfp_scheme* sc, double tol, int maxit, double* C_eff_out,
                    int* iters_out) {
  if (!(tol > 0.0) || maxit < 1 || !C_eff_out) return GFP_ERR_ARG;
  gfp_batch b = nullptr;
  int rc = gfp_batch_create(count, grids, sc, &b);
  if (rc) return rc;
  rc = gfp_batch_solve(b, tol, maxit, C_eff_out, iters_out);
  gfp_batch_destroy(b);
  return rc;
}

}  // extern "C"
