// FP64 outer pass of the mixed-precision solve, evaluated in real space.
//
// After each FP32 inner solve the mixed solve needs, for its FP64 strain, the exact residual
// eta = ||T_check q^b|| / ||T_check(0)||_F and the inner iterations' source v = T_check kt (FP32).
// For every scheme the mixed solve runs (CD, ACD, AHC, AFB/R; Sec. 5.3), T_check(k) q^b(k) has the
// modulus of the transform of a difference stencil applied to the stress in real space:
//   CD    D_j f(x) = [f(x + e_j) - f(x - e_j)] / (2h)                     symbol i sin th_j
//   ACD   D_j f(x) = sum_{s,t = +-1} [f(x + e_j + s e_a + t e_b) - f(x - e_j + s e_a + t e_b)] / (8h)
//                                                                          symbol i sin th_j cos th_a cos th_b
//   AHC, AFB/R (averaged forward differences over the unit cube)
//         D_j f(x) = sum_{a,b in {0,1}} [f(x + e_j + a e_s + b e_t) - f(x + a e_s + b e_t)] / (4h)
//                    symbol e^{i phi} i 2 sin(th_j/2) cos(th_s/2) cos(th_t/2), phi = (th_1 + th_2 + th_3)/2
// with th_r = 2 pi kappa_r / n_r (the index map of eq. FieFouAppTra1D, Nyquist kappa = -n/2).  With
// r_i = sum_j D_j sigma_ij the symbol is c(k) i kt(k), |c| = 1 and common to the three components, so
// by Parseval (unnormalised forward transform) sum_k |T_check(k) kt(k)|^2 = N sum_x |r(x)|^2 and
//   eta = sqrt(N sum_x |r(x)|^2) / ||sum_x sigma(x)||_F,      v(k) = -i conj(c(k)) F[r](k).
// The residual and the mean stress are therefore FP64 sums over the stress in real space, without an
// FP64 transform, and the source comes from an FP32 transform of r: v is stored in FP32 and r carries
// its own scale, so the FP32 transform keeps v's relative accuracy.
#pragma once
#include "gfp_kernels.cuh"

namespace gfp {

enum { RS_CD = 0, RS_ACD = 1, RS_AFD = 2 };

// Refinement step of the FP64 strain: eps += corr - mean(corr) (skipped while `gate` is done).
__global__ void apply_corr64_kernel(double* __restrict__ eps, const float* __restrict__ corr,
                                    const double* __restrict__ cmean, long long N, const SolveState* gate) {
  if (gate && gate->done) return;
  double cm[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) cm[c] = cmean[c];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 6; ++c) eps[c * N + i] += (double)corr[c * N + i] - cm[c];
  }
}

// Tile of the real-space residual: RX x RY columns marched over RZ planes, one voxel of halo on each
// side (periodic).  A CTA of RX RY threads keeps the stress of three consecutive halo planes in
// shared memory.
constexpr int kResTX = 32, kResTY = 8, kResTZ = 16;

// sigma = C : (eps - estar) (FP64), r = D^b sigma rounded to FP32 into rout [3][N], and per CTA the
// FP64 sums part[8 b + 0] = sum |r|^2 and part[8 b + 1 + c] = sum sigma_c over the CTA's voxels.
template <int S>
__global__ void __launch_bounds__(kResTX * kResTY) residual64_kernel(const double* __restrict__ eps,
                                                                     const double* __restrict__ lam,
                                                                     const double* __restrict__ mu,
                                                                     const double* __restrict__ estar, Dims d,
                                                                     double inv_h, float* __restrict__ rout,
                                                                     double* __restrict__ part,
                                                                     const SolveState* gate) {
  if (gate && gate->done) return;
  constexpr int HX = kResTX + 2, HY = kResTY + 2, NT = kResTX * kResTY;
  __shared__ double sg[3][6][HY][HX];
  __shared__ double red[NT / 32][8];
  const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
  const long long N = d.N;
  const int x0 = blockIdx.x * kResTX, y0 = blockIdx.y * kResTY, z0 = blockIdx.z * kResTZ;
  const int tx = threadIdx.x % kResTX, ty = threadIdx.x / kResTX;
  const bool col_ok = (x0 + tx < n1) && (y0 + ty < n2);
  const int nz = min(kResTZ, n3 - z0);
  double ss[6] = {0, 0, 0, 0, 0, 0};
  float rr = 0.f;  // eta needs relative accuracy only; r itself is FP64
  // the averaged forward differences need the halo on the high side only
  constexpr int LO = S == RS_AFD ? 1 : 0, RW = HX - LO, RH = HY - LO;
#pragma unroll 1
  for (int p = S == RS_AFD ? 1 : 0; p < nz + 2; ++p) {
    const int zw = ((z0 - 1 + p) % n3 + n3) % n3;
    const int slot = p % 3;
    for (int i = threadIdx.x; i < RW * RH; i += NT) {
      const int hx = LO + i % RW, hy = LO + i / RW;
      const int xg = ((x0 - 1 + hx) % n1 + n1) % n1;
      const int yg = ((y0 - 1 + hy) % n2 + n2) % n2;
      const long long v = ((long long)zw * n2 + yg) * n1 + xg;
      double e[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] = eps[c * N + v];
      if (estar) {
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] -= estar[c * N + v];
      }
      const double m2 = 2.0 * mu[v], ltr = lam[v] * (e[0] + e[1] + e[2]);
      double sgm[6];
      sgm[0] = m2 * e[0] + ltr;
      sgm[1] = m2 * e[1] + ltr;
      sgm[2] = m2 * e[2] + ltr;
      sgm[3] = m2 * e[3];
      sgm[4] = m2 * e[4];
      sgm[5] = m2 * e[5];
#pragma unroll
      for (int c = 0; c < 6; ++c) sg[slot][c][hy][hx] = sgm[c];
      const bool own = hx >= 1 && hx <= kResTX && hy >= 1 && hy <= kResTY && p >= 1 && p <= nz &&
                       x0 - 1 + hx < n1 && y0 - 1 + hy < n2;
      if (own) {
#pragma unroll
        for (int c = 0; c < 6; ++c) ss[c] += sgm[c];
      }
    }
    __syncthreads();
    if (p >= 2 && col_ok) {
      // outputs on plane p - 1 (z = z0 + p - 2); its neighbours below and above are planes p - 2, p
      const int sl[3] = {(p - 2) % 3, (p - 1) % 3, p % 3};
      const int hx = tx + 1, hy = ty + 1;
      // stress component c at offset (dx, dy, dz) from the output voxel
      auto f = [&](int c, int dx, int dy, int dz) -> double { return sg[sl[dz + 1]][c][hy + dy][hx + dx]; };
      // component c at offsets (oj, oa, ob) along (e_j, e_a, e_b), (a, b) the axes after j cyclically
      auto at = [&](int c, int jj, int oj, int oa, int ob) -> double {
        int o[3];
        o[jj] = oj;
        o[(jj + 1) % 3] = oa;
        o[(jj + 2) % 3] = ob;
        return f(c, o[0], o[1], o[2]);
      };
      const double sc = (S == RS_CD ? 0.5 : (S == RS_ACD ? 0.125 : 0.25)) * inv_h;
      double r1, r2, r3;
      if (S == RS_AFD) {
        // over the unit cube, with the pair sums along the third axis shared by a component's two
        // derivatives: D_u f = [p(1,0) + p(1,1)] - [p(0,0) + p(0,1)], p(a,b) = f(a,b,0) + f(a,b,1)
        auto one = [&](int c, int u) -> double {  // single derivative along axis u
          const double hi = (at(c, u, 1, 0, 0) + at(c, u, 1, 0, 1)) + (at(c, u, 1, 1, 0) + at(c, u, 1, 1, 1));
          const double lo = (at(c, u, 0, 0, 0) + at(c, u, 0, 0, 1)) + (at(c, u, 0, 1, 0) + at(c, u, 0, 1, 1));
          return hi - lo;
        };
        // two derivatives along u and v = (u + 1) % 3 of component c, sharing the sums along w
        auto two = [&](int c, int u, double& du, double& dv) {
          double q[2][2];
#pragma unroll
          for (int a = 0; a <= 1; ++a)
#pragma unroll
            for (int b = 0; b <= 1; ++b) q[a][b] = at(c, u, a, b, 0) + at(c, u, a, b, 1);
          du = (q[1][0] + q[1][1]) - (q[0][0] + q[0][1]);
          dv = (q[0][1] + q[1][1]) - (q[0][0] + q[1][0]);
        };
        double d12x, d12y, d23y, d23z, d13z, d13x;
        two(5, 0, d12x, d12y);  // sigma_12: D_1, D_2
        two(3, 1, d23y, d23z);  // sigma_23: D_2, D_3
        two(4, 2, d13z, d13x);  // sigma_13: D_3, D_1
        r1 = sc * (one(0, 0) + d12y + d13z);
        r2 = sc * (d12x + one(1, 1) + d23z);
        r3 = sc * (d13x + d23y + one(2, 2));
      } else {
      // D_j of component c, unscaled
      auto D = [&](int c, int jj) -> double {
        double acc = 0.0;
        if (S == RS_CD) {
          acc = at(c, jj, 1, 0, 0) - at(c, jj, -1, 0, 0);
        } else if (S == RS_ACD) {
#pragma unroll
          for (int sa = -1; sa <= 1; sa += 2)
#pragma unroll
            for (int sb = -1; sb <= 1; sb += 2) acc += at(c, jj, 1, sa, sb) - at(c, jj, -1, sa, sb);
        } else {
#pragma unroll
          for (int oa = 0; oa <= 1; ++oa)
#pragma unroll
            for (int ob = 0; ob <= 1; ++ob) acc += at(c, jj, 1, oa, ob) - at(c, jj, 0, oa, ob);
        }
        return acc;
      };
      // components (11, 22, 33, 23, 13, 12) = (0, 1, 2, 3, 4, 5)
      r1 = sc * (D(0, 0) + D(5, 1) + D(4, 2));
      r2 = sc * (D(5, 0) + D(1, 1) + D(3, 2));
      r3 = sc * (D(4, 0) + D(3, 1) + D(2, 2));
      }
      const long long v = ((long long)(z0 + p - 2) * n2 + (y0 + ty)) * n1 + (x0 + tx);
      const float f1 = (float)r1, f2 = (float)r2, f3 = (float)r3;
      rout[v] = f1;
      rout[N + v] = f2;
      rout[2 * N + v] = f3;
      rr += f1 * f1 + f2 * f2 + f3 * f3;
    }
    __syncthreads();
  }
  // per-CTA sums, fixed order
  double q[7] = {(double)rr, ss[0], ss[1], ss[2], ss[3], ss[4], ss[5]};
#pragma unroll
  for (int k = 0; k < 7; ++k)
    for (int off = 16; off > 0; off >>= 1) q[k] += __shfl_down_sync(0xffffffffu, q[k], off);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 7; ++k) red[threadIdx.x >> 5][k] = q[k];
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
    const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[8 * b + threadIdx.x] = s;
  }
}

// The averaged-forward-difference case (AHC, AFB/R) of residual64_kernel with the work shared between
// planes.  In the 2x2 window of a thread on plane z, with g_ab = f(x + a, y + b, z):
//   Qx f = (g10 - g00) + (g11 - g01),  Qy f = (g01 - g00) + (g11 - g10),  P f = g00 + g01 + g10 + g11,
// and D_x f(z) = Qx f(z) + Qx f(z+1), D_y f(z) = Qy f(z) + Qy f(z+1), D_z f(z) = P f(z+1) - P f(z).  So
// r_1(z) = M_1(z) + S_1(z+1) with S_1 = Qx s11 + Qy s12 + P s13 and M_1 = Qx s11 + Qy s12 - P s13 (and
// likewise r_2 from s12, s22, s23 and r_3 from s13, s23, s33): each plane is visited once, and only M
// is carried to the next plane.  Same outputs and partial sums as residual64_kernel<RS_AFD>.
__global__ void __launch_bounds__(kResTX * kResTY) residual64_afd_kernel(const double* __restrict__ eps,
                                                                         const double* __restrict__ lam,
                                                                         const double* __restrict__ mu,
                                                                         const double* __restrict__ estar, Dims d,
                                                                         double inv_h, float* __restrict__ rout,
                                                                         double* __restrict__ part,
                                                                         const SolveState* gate) {
  if (gate && gate->done) return;
  constexpr int HX = kResTX + 1, HY = kResTY + 1, NT = kResTX * kResTY;
  __shared__ double sg[6][HY][HX];
  __shared__ double red[NT / 32][8];
  const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
  const long long N = d.N;
  const int x0 = blockIdx.x * kResTX, y0 = blockIdx.y * kResTY, z0 = blockIdx.z * kResTZ;
  const int tx = threadIdx.x % kResTX, ty = threadIdx.x / kResTX;
  const bool col_ok = (x0 + tx < n1) && (y0 + ty < n2);
  const int nz = min(kResTZ, n3 - z0);
  const double sc = 0.25 * inv_h;
  double ss[6] = {0, 0, 0, 0, 0, 0};
  float rr = 0.f;
  double M1 = 0.0, M2 = 0.0, M3 = 0.0;
#pragma unroll 1
  for (int p = 0; p <= nz; ++p) {  // planes z0 .. z0 + nz
    const int zw = (z0 + p) % n3;
    for (int i = threadIdx.x; i < HX * HY; i += NT) {
      const int hx = i % HX, hy = i / HX;
      const int xg = (x0 + hx) % n1, yg = (y0 + hy) % n2;
      const long long v = ((long long)zw * n2 + yg) * n1 + xg;
      double e[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] = eps[c * N + v];
      if (estar) {
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] -= estar[c * N + v];
      }
      const double m2 = 2.0 * mu[v], ltr = lam[v] * (e[0] + e[1] + e[2]);
      double sgm[6];
      sgm[0] = m2 * e[0] + ltr;
      sgm[1] = m2 * e[1] + ltr;
      sgm[2] = m2 * e[2] + ltr;
      sgm[3] = m2 * e[3];
      sgm[4] = m2 * e[4];
      sgm[5] = m2 * e[5];
#pragma unroll
      for (int c = 0; c < 6; ++c) sg[c][hy][hx] = sgm[c];
      if (hx < kResTX && hy < kResTY && p < nz && x0 + hx < n1 && y0 + hy < n2) {
#pragma unroll
        for (int c = 0; c < 6; ++c) ss[c] += sgm[c];
      }
    }
    __syncthreads();
    if (col_ok) {
      auto g = [&](int c, int a, int b) -> double { return sg[c][ty + b][tx + a]; };
      // components (11, 22, 33, 23, 13, 12) = (0, 1, 2, 3, 4, 5)
      const double qx11 = (g(0, 1, 0) - g(0, 0, 0)) + (g(0, 1, 1) - g(0, 0, 1));
      const double qy22 = (g(1, 0, 1) - g(1, 0, 0)) + (g(1, 1, 1) - g(1, 1, 0));
      const double p33 = (g(2, 0, 0) + g(2, 0, 1)) + (g(2, 1, 0) + g(2, 1, 1));
      const double a12 = g(5, 1, 1) - g(5, 0, 0), b12 = g(5, 1, 0) - g(5, 0, 1);
      const double qx12 = a12 + b12, qy12 = a12 - b12;
      const double u13 = g(4, 1, 0) + g(4, 1, 1), w13 = g(4, 0, 0) + g(4, 0, 1);
      const double qx13 = u13 - w13, p13 = u13 + w13;
      const double u23 = g(3, 0, 1) + g(3, 1, 1), w23 = g(3, 0, 0) + g(3, 1, 0);
      const double qy23 = u23 - w23, p23 = u23 + w23;
      const double t1 = qx11 + qy12, t2 = qx12 + qy22, t3 = qx13 + qy23;
      if (p >= 1) {  // outputs on plane z0 + p - 1
        const double r1 = sc * (M1 + (t1 + p13));
        const double r2 = sc * (M2 + (t2 + p23));
        const double r3 = sc * (M3 + (t3 + p33));
        const long long v = ((long long)(z0 + p - 1) * n2 + (y0 + ty)) * n1 + (x0 + tx);
        const float f1 = (float)r1, f2 = (float)r2, f3 = (float)r3;
        rout[v] = f1;
        rout[N + v] = f2;
        rout[2 * N + v] = f3;
        rr += f1 * f1 + f2 * f2 + f3 * f3;
      }
      M1 = t1 - p13;
      M2 = t2 - p23;
      M3 = t3 - p33;
    }
    __syncthreads();
  }
  double q[7] = {(double)rr, ss[0], ss[1], ss[2], ss[3], ss[4], ss[5]};
#pragma unroll
  for (int k = 0; k < 7; ++k)
    for (int off = 16; off > 0; off >>= 1) q[k] += __shfl_down_sync(0xffffffffu, q[k], off);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 7; ++k) red[threadIdx.x >> 5][k] = q[k];
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double sm = 0.0;
    for (int w = 0; w < NT / 32; ++w) sm += red[w][threadIdx.x];
    const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[8 * b + threadIdx.x] = sm;
  }
}

// Mean stress of an FP64 strain field with compensated summation: sigma = C : (eps - estar) per voxel,
// summed per thread and per CTA in Neumaier's form (running sum plus the accumulated rounding
// errors), per-CTA (sum, compensation) pairs into part[12 b + 2 c], then combined in a fixed order by
// mean_stress64_final_kernel.  The sum the transform forms at k = 0 rounds at about 1e-16 of the mean
// stress, which is the size of the change one voxel's modulus makes in the effective stiffness of a
// 128^3 cell; this sum keeps the rounding well below it.
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

__global__ void __launch_bounds__(256) mean_stress64_kernel(const double* __restrict__ eps, const double* __restrict__ lam,
                                                          const double* __restrict__ mu, const double* __restrict__ estar,
                                                          long long N, double* __restrict__ part) {
  __shared__ double sh[256][12];
  double s[6] = {0, 0, 0, 0, 0, 0}, cp[6] = {0, 0, 0, 0, 0, 0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
    double e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps[c * N + v] - (estar ? estar[c * N + v] : 0.0);
    const double m2 = 2.0 * mu[v], ltr = lam[v] * (e[0] + e[1] + e[2]);
    neumaier_add(s[0], cp[0], m2 * e[0] + ltr);
    neumaier_add(s[1], cp[1], m2 * e[1] + ltr);
    neumaier_add(s[2], cp[2], m2 * e[2] + ltr);
    neumaier_add(s[3], cp[3], m2 * e[3]);
    neumaier_add(s[4], cp[4], m2 * e[4]);
    neumaier_add(s[5], cp[5], m2 * e[5]);
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) { sh[threadIdx.x][2 * c] = s[c]; sh[threadIdx.x][2 * c + 1] = cp[c]; }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    double ss = 0.0, cc = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      neumaier_add(ss, cc, sh[i][2 * c]);
      cc += sh[i][2 * c + 1];
    }
    part[12 * blockIdx.x + 2 * c] = ss;
    part[12 * blockIdx.x + 2 * c + 1] = cc;
  }
}

// Fixed-order combination of the per-CTA pairs: st->T0[c] = sum sigma_c (the transform at k = 0).
__global__ void mean_stress64_final_kernel(const double* __restrict__ part, int nb, SolveState* st) {
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    double ss = 0.0, cc = 0.0;
    for (int b = 0; b < nb; ++b) {
      neumaier_add(ss, cc, part[12 * b + 2 * c]);
      cc += part[12 * b + 2 * c + 1];
    }
    st->T0[c] = ss + cc;
  }
}

// Sum of the per-CTA residual sums in a fixed order: st->T0 = sum sigma (the transform at k = 0) and
// out[0] = N sum |r|^2, the spectral residual sum that reduce_eta turns into eta and the decision.
__global__ void res64_sum_kernel(const double* __restrict__ part, int np, long long N, SolveState* st,
                                 double* __restrict__ out) {
  if (st->done) return;
  __shared__ double sh[7][256];
  double q[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < np; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 7; ++k) q[k] += part[8 * b + k];
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] = q[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = (double)N * sh[0][0];
    for (int c = 0; c < 6; ++c) st->T0[c] = sh[1 + c][0];
  }
}

// Forward real-to-complex transform along x1 of the three residual components r [3][N] (FP32) into
// the half spectra v [3][k3][k2][P]: `lines` consecutive x-lines per CTA (even), the same component
// of two neighbouring lines sharing one complex line (a + i b), split after the transform.
__global__ void __launch_bounds__(256) rx_kernel(const float* __restrict__ r, float2* __restrict__ v,
                                                 const float2* __restrict__ tw, FftPlan plan, Dims d, int lines,
                                                 const SolveState* gate) {
  if (gate && gate->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = d.n1, NH = n / 2 + 1, hp = lines / 2, nl = 3 * hp;
  float2* a = reinterpret_cast<float2*>(smem_raw);
  float2* b = a + nl * n;
  const long long nlines = (long long)d.n2 * d.n3;
  const long long line0 = (long long)blockIdx.x * lines;
  for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
    const int e = i % n, q = i / n;
    const int c = q / hp, p2 = q % hp;
    const long long la = line0 + 2 * p2, lb = la + 1;
    float2 z;
    z.x = la < nlines ? r[c * d.N + la * n + e] : 0.f;
    z.y = lb < nlines ? r[c * d.N + lb * n + e] : 0.f;
    a[i] = z;
  }
  __syncthreads();
  LineLayout L{nl, 1, n, false};
  const float2* Z = fft_lines<false>(a, b, tw, plan, L);
  for (int i = threadIdx.x; i < nl * NH; i += blockDim.x) {
    const int k = i % NH, q = i / NH;
    const int c = q / hp, p2 = q % hp;
    const long long la = line0 + 2 * p2, lb = la + 1;
    if (la >= nlines) continue;
    const float2 zk = Z[q * n + k], zn = Z[q * n + (n - k) % n];
    float2 A, B;
    A.x = 0.5f * (zk.x + zn.x); A.y = 0.5f * (zk.y - zn.y);
    B.x = 0.5f * (zk.y + zn.y); B.y = -0.5f * (zk.x - zn.x);
    v[c * d.S + d.xrow(la) * d.P + k] = A;
    if (lb < nlines) v[c * d.S + d.xrow(lb) * d.P + k] = B;
  }
}

// Forward transform along x3 of the three half spectra v, in place, then v <- -i conj(c(k)) v with
// c(k) = ph1[k1] ph2[k2] ph3[k3] the common phase of the stencil symbol (null tables: c = 1).  CTA =
// `cols` k1 columns of one component at fixed k2.
__global__ void __launch_bounds__(256) rz_kernel(float2* __restrict__ v, const float2* __restrict__ tw, FftPlan plan,
                                                 Dims d, int cols, const float2* __restrict__ ph1,
                                                 const float2* __restrict__ ph2, const float2* __restrict__ ph3,
                                                 const SolveState* gate) {
  if (gate && gate->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = d.n3, ls = n + 1;
  float2* a = reinterpret_cast<float2*>(smem_raw);
  float2* b = a + cols * ls;
  const int k10 = blockIdx.x * cols, k2 = blockIdx.y, c = blockIdx.z;
  float2* g = v + c * d.S + d.row(0, k2) * d.P;
  const long long zs = d.zstride();
  for (int i = threadIdx.x; i < cols * n; i += blockDim.x) {
    const int l = i % cols, e = i / cols;
    float2 z; z.x = 0.f; z.y = 0.f;
    if (k10 + l < d.n1h) z = g[e * zs + k10 + l];
    a[l * ls + e] = z;
  }
  __syncthreads();
  LineLayout L{cols, 1, ls, false};
  const float2* Z = fft_lines<false>(a, b, tw, plan, L);
  float2 p2; p2.x = 1.f; p2.y = 0.f;
  if (ph2) p2 = ph2[k2];
  for (int i = threadIdx.x; i < cols * n; i += blockDim.x) {
    const int l = i % cols, e = i / cols;
    const int k1 = k10 + l;
    if (k1 >= d.n1h) continue;
    float2 z = Z[l * ls + e];
    if (ph1) {
      float2 ph = cmul(cmul(ph1[k1], p2), ph3[e]);
      ph.y = -ph.y;  // conj(c)
      z = cmul(z, ph);
    }
    float2 o; o.x = z.y; o.y = -z.x;  // -i z
    g[e * zs + k1] = o;
  }
}

}  // namespace gfp
