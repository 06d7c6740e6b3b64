// Register-resident line FFTs with compile-time lengths (sm_103a), and the hot-path passes built on
// them.  Same transform as gfp_fft.cuh (Stockham stages, forward e^{-2 pi i jk/n}, unnormalised), but
// each thread keeps E elements of a line in registers: the first stage reads global memory directly,
// the last stage writes global memory directly, and consecutive stages exchange through shared
// memory once.  All index arithmetic is compile-time except the thread's position in the line.
#pragma once
#include "gfp_kernels.cuh"

namespace gfp {

// Stage radices per length: E elements per thread, T = N / E threads per line; every radix divides E.
template <int N> struct CPlan { static constexpr bool ok = false; };
#define GFP_CPLAN(N_, E_, NST_, R0, R1, R2)                                                   \
  template <> struct CPlan<N_> {                                                               \
    static constexpr bool ok = true;                                                           \
    static constexpr int N = N_, E = E_, T = N_ / E_, NST = NST_;                              \
    __host__ __device__ static constexpr int R(int s) { return s == 0 ? R0 : (s == 1 ? R1 : R2); } \
    __host__ __device__ static constexpr int Ns(int s) { return s == 0 ? 1 : (s == 1 ? R0 : R0 * R1); } \
  };
GFP_CPLAN(32, 8, 2, 8, 4, 1)
GFP_CPLAN(64, 8, 2, 8, 8, 1)
GFP_CPLAN(96, 24, 3, 8, 4, 3)
GFP_CPLAN(128, 16, 2, 16, 8, 1)
GFP_CPLAN(192, 24, 3, 8, 8, 3)
GFP_CPLAN(256, 16, 2, 16, 16, 1)
GFP_CPLAN(512, 32, 3, 16, 16, 2)
#undef GFP_CPLAN

// Element index read by input r of butterfly b at stage S (thread position t): j + r N / R, j = t + b T.
template <int N, int S> __device__ __forceinline__ int cin_idx(int t, int b, int r) {
  typedef CPlan<N> P;
  return t + b * P::T + r * (N / P::R(S));
}
// Element index written by output r of butterfly b at stage S: (j / Ns) Ns R + j % Ns + r Ns.
template <int N, int S> __device__ __forceinline__ int cout_idx(int t, int b, int r) {
  typedef CPlan<N> P;
  constexpr int R = P::R(S), Ns = P::Ns(S);
  const int j = t + b * P::T;
  return (j / Ns) * Ns * R + (j % Ns) + r * Ns;
}

// Twiddle and butterflies of stage S for the thread's E / R butterflies.
template <int N, int S, bool INV, typename T>
__device__ __forceinline__ void cstage(T* v, int t, const T* __restrict__ tw) {
  typedef CPlan<N> P;
  constexpr int R = P::R(S), Ns = P::Ns(S), NB = P::E / R, stride = N / (Ns * R);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (S > 0) {
      const int k = (t + b * P::T) % Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        T w = tw[r * k * stride];
        if (INV) w.y = -w.y;
        v[b * R + r] = cmul(v[b * R + r], w);
      }
    }
    Dft<R, INV, T>::run(v + b * R);
  }
}

// 16-byte asynchronous global -> shared copies (L2 only) and a full wait.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Line buffer in shared memory with an element stride and an optional pad of one element per 16
// (line-major buffers, to spread the strided Stockham writes over the banks).
template <typename T, bool PAD>
struct SLine {
  T* base;
  int es;
  __device__ __forceinline__ T& operator[](int e) const { return base[(PAD ? e + (e >> 4) : e) * es]; }
};

// Line L of the 8-column z tile (rows of 48 elements: component c, column cc at 8 c + cc) with the
// columns of odd rows XOR-swizzled by 8, i.e. one component further: the Green step's half-warps
// (2 rows x 8 columns of one component) then touch every bank once, while the line transforms'
// access patterns keep their bank spread.
template <typename T>
struct SLineX {
  T* base;
  int L;
  __device__ __forceinline__ T& operator[](int e) const { return base[e * 48 + (L ^ ((e & 1) << 3))]; }
};

template <int N, int S, bool INV, typename T, typename SL>
__device__ __forceinline__ void cexchange(T* v, SL sm, int t) {
  typedef CPlan<N> P;
  constexpr int R = P::R(S), R1 = P::R(S + 1);
#pragma unroll
  for (int b = 0; b < P::E / R; ++b)
#pragma unroll
    for (int r = 0; r < R; ++r) sm[cout_idx<N, S>(t, b, r)] = v[b * R + r];
  __syncthreads();
#pragma unroll
  for (int b = 0; b < P::E / R1; ++b)
#pragma unroll
    for (int r = 0; r < R1; ++r) v[b * R1 + r] = sm[cin_idx<N, S + 1>(t, b, r)];
  __syncthreads();
}

// Full transform of one line held as v[b R0 + r] = x[cin_idx<N,0>(t,b,r)]; on return
// v[b RL + r] = X[cout_idx<N,NST-1>(t,b,r)] = X[t + b T + r N / RL].  Every thread of the block
// must call it (it synchronises).
template <int N, bool INV, typename T, typename SL>
__device__ __forceinline__ void cfft(T* v, SL sm, int t, const T* __restrict__ tw) {
  typedef CPlan<N> P;
  cstage<N, 0, INV>(v, t, tw);
  if constexpr (P::NST > 1) {
    cexchange<N, 0, INV>(v, sm, t);
    cstage<N, 1, INV>(v, t, tw);
  }
  if constexpr (P::NST > 2) {
    cexchange<N, 1, INV>(v, sm, t);
    cstage<N, 2, INV>(v, t, tw);
  }
}

// ------------------------------------------------------------------------------------------------
// pass_y: CTA = C columns of k1 x all n2 rows of one component at fixed k3; thread = (column, t).
// ------------------------------------------------------------------------------------------------
template <typename R, int N, bool INV, int COLS>
__global__ void __launch_bounds__(512) pass_y_c_kernel(typename C<R>::T* __restrict__ spec,
                                                       const typename C<R>::T* __restrict__ tw, Dims d, int cols_arg,
                                                       const SolveState* __restrict__ st) {
  typedef typename C<R>::T T;
  typedef CPlan<N> P;
  const int cols = COLS > 0 ? COLS : cols_arg;
  // the inverse pass runs after the residual reduction of its iteration: it still completes an
  // iteration stopped by the iteration cap (state 2), so that a batched solve resumes from a fully
  // transformed increment
  if (st->done && !(INV && st->done == 2)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* twl = reinterpret_cast<T*>(smem_raw);
  T* buf = twl + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) twl[i] = tw[i];
  const int col = threadIdx.x % cols, t = threadIdx.x / cols;
  const int k1 = blockIdx.x * cols + col;
  const bool live = k1 < d.n1h;
  T* g = spec + blockIdx.z * d.S + d.row(blockIdx.y, 0) * d.P + k1;
  const int ys = d.ystride();
  T v[P::E];
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) {
      T x; x.x = 0; x.y = 0;
      if (live) x = g[cin_idx<N, 0>(t, b, r) * ys];
      v[b * P::R(0) + r] = x;
    }
  __syncthreads();
  cfft<N, INV>(v, SLine<T, false>{buf + col, cols}, t, twl);
  constexpr int RL = P::R(P::NST - 1);
  if (live) {
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) g[cout_idx<N, P::NST - 1>(t, b, r) * ys] = v[b * RL + r];
  }
}

// ------------------------------------------------------------------------------------------------
// pass_z_gamma: CTA = C columns x 6 components x all n3 rows at fixed k2; line = (comp, col).
// Same modes as the generic kernel (PZ_GAMMA, PZ_RESIDUAL, PZ_INNER).
// ------------------------------------------------------------------------------------------------
// FP32 register FFTs of up to 16 elements per thread fit two 384-thread CTAs per SM.
template <typename R, int N> struct ZBound {
  static constexpr bool small = sizeof(R) == 4 && CPlan<N>::E <= 16;
  static constexpr int threads = small ? 384 : 512;
  static constexpr int blocks = small ? 2 : 1;
};

// Green step on a z-tile in shared memory: rows [k3][ZS] holding 6 components x cols columns
// (component c, column cc at c cols + cc, XOR swz on odd rows).  Residual partial of the thread
// (returned), T(0), and, by mode, the increment written back in place (PZ_GAMMA, PZ_INNER, PZ_DGO) or
// the inner-iteration source stored (PZ_RESIDUAL).  vs: the tile's inner source staged as
// [3][N][cols], or null to read it from global memory.  blockDim.x is a multiple of cols: every
// thread keeps one column.
template <typename R, int N>
__device__ __forceinline__ R green_tile(typename C<R>::T* __restrict__ buf, int ZS, int cols, int swz,
                                        const typename C<R>::T* __restrict__ ab3, const float2* vs, const Dims& d,
                                        int k10, int k2, const GammaParams<R>& gp, SolveState* __restrict__ st,
                                        int mode, float2* __restrict__ vsrc, R* acc2 = nullptr) {
  typedef typename C<R>::T T;
  R acc = 0;
  const bool ny2 = ((d.n2 & 1) == 0) && (2 * k2 == d.n2);
  const R b2 = gp.B[1][k2], a2 = gp.A[1][k2];
  const int cc = threadIdx.x % cols;
  const int k1 = k10 + cc;
  if (k1 < d.n1h) {
    const R a1 = gp.A[0][k1], b1 = gp.B[0][k1];
    const bool ny1 = ((d.n1 & 1) == 0) && (2 * k1 == d.n1);
    const bool self1 = (k1 == 0) || ny1;
    const int zstep = blockDim.x / cols;
    // inner source of point z: staged tile or global memory
    auto source = [&](int z, float2& s1, float2& s2, float2& s3) {
      if (vs) { s1 = vs[z * cols + cc]; s2 = vs[(N + z) * cols + cc]; s3 = vs[(2 * N + z) * cols + cc]; }
      else {
        const long long vi = d.row(z, k2) * d.P + k1;
        s1 = vsrc[vi]; s2 = vsrc[d.S + vi]; s3 = vsrc[2 * d.S + vi];
      }
    };
    // the next point's source is loaded one point ahead, so its latency overlaps this point's arithmetic
    float2 p1, p2, p3;
    const int z0 = threadIdx.x / cols;
    if (mode == PZ_INNER && z0 < N) source(z0, p1, p2, p3);
    for (int z = z0; z < N; z += zstep) {
      float2 s1, s2, s3;
      if (mode == PZ_INNER) {
        s1 = p1; s2 = p2; s3 = p3;
        if (z + zstep < N) source(z + zstep, p1, p2, p3);
      }
      T* rowz = buf + z * ZS;
      const int sw = (z & 1) ? swz : 0;
      T tt[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) tt[c] = rowz[(c * cols + cc) ^ sw];
      const T ab = ab3[z];
      const R a3 = ab.x, b3 = ab.y;
      const R kt1 = a1 * b2 * b3, kt2 = a2 * b3 * b1, kt3 = a3 * b1 * b2;
      const bool ny3 = (2 * z == N);
      const long long vi = d.row(z, k2) * d.P + k1;
      if (sizeof(R) == 8 && mode == PZ_DISP) {  // FP64 only (folded out of the FP32 kernels' registers)
        T o[6];
        disp_point<R>(tt, kt1, kt2, kt3, gp.half_shift, d, k1, k2, z, gp.invN, o);
#pragma unroll
        for (int c = 0; c < 6; ++c) rowz[(c * cols + cc) ^ sw] = o[c];
        continue;
      }
      if (mode != PZ_INNER && k1 == 0 && k2 == 0 && z == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) st->T0[c] = (double)tt[c].x;
      }
      T v1, v2, v3;
      tk_vec<R>(tt, kt1, kt2, kt3, v1, v2, v3);
      if (mode == PZ_INNER) {
        v1.x += (R)s1.x; v1.y += (R)s1.y; v2.x += (R)s2.x; v2.y += (R)s2.y; v3.x += (R)s3.x; v3.y += (R)s3.y;
      }
      R r2 = vnorm2(v1, v2, v3);
      if (!self1) {
        if (gp.nyq_avg && (ny2 || ny3)) r2 += tk_norm2<R>(tt, kt1, ny2 ? -kt2 : kt2, ny3 ? -kt3 : kt3);
        else r2 *= (R)2;
      }
      acc += r2;
      if (sizeof(R) == 8 && mode == PZ_GAMMA && acc2 && gp.vprev) {  // FP64 only (the paper's stop rule)
        const R c = incr_point<R>(v1, v2, v3, kt1, kt2, kt3, gp, vi, d.S);
        *acc2 += self1 ? c : (R)2 * c;
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
        dgo_apply_point<R>(tt, gp.dgo, vi, d.S, gp.invN, o);
#pragma unroll
        for (int c = 0; c < 6; ++c) rowz[(c * cols + cc) ^ sw] = o[c];
        continue;
      }
      gamma0_from_v<R>(v1, v2, v3, kt1, kt2, kt3, gp.c_mu, gp.c_lm, gp.invN, o);
      if (gp.nyq_avg && (ny1 || ny2 || ny3)) {
        T o2[6];
        gamma0_apply<R>(tt, ny1 ? -kt1 : kt1, ny2 ? -kt2 : kt2, ny3 ? -kt3 : kt3, gp.c_mu, gp.c_lm, gp.invN, o2);
#pragma unroll
        for (int c = 0; c < 6; ++c) { o[c].x = (R)0.5 * (o[c].x + o2[c].x); o[c].y = (R)0.5 * (o[c].y + o2[c].y); }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) rowz[(c * cols + cc) ^ sw] = o[c];
    }
  }
  return acc;
}

// COLS > 0 fixes the tile width at compile time (index arithmetic folds); COLS = 0 reads cols_arg.
template <typename R, int N, int COLS>
__global__ void __launch_bounds__(ZBound<R, N>::threads, ZBound<R, N>::blocks) pass_z_c_kernel(typename C<R>::T* __restrict__ spec,
                                                       const typename C<R>::T* __restrict__ tw, Dims d, int cols_arg,
                                                       GammaParams<R> gp, double* __restrict__ partials,
                                                       SolveState* __restrict__ st, int mode, float2* __restrict__ vsrc) {
  typedef typename C<R>::T T;
  typedef CPlan<N> P;
  const int cols = COLS > 0 ? COLS : cols_arg;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* twl = reinterpret_cast<T*>(smem_raw);
  T* ab3 = twl + N;                          // (A_3, B_3) per k3
  T* buf = ab3 + N;                          // [k3][ZS]: 6 components x cols, then cols of padding
  // Row pitch 7 cols: with 8-byte elements each half-warp of the Green step (4 or 8 rows x cols
  // columns of one component) then touches every bank once.
  const int ZS = 7 * cols;
  __shared__ double red[32];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    twl[i] = tw[i];
    T ab;
    ab.x = gp.A[2][i];
    ab.y = gp.B[2][i];
    ab3[i] = ab;
  }
  const int w6 = 6 * cols;
  const int l = threadIdx.x % w6, t = threadIdx.x / w6;
  const int comp = l / cols, col = l % cols;
  const int k10 = blockIdx.x * cols;
  const int k2 = blockIdx.y;
  const bool live = k10 + col < d.n1h;
  T* g = spec + comp * d.S + d.row(0, k2) * d.P + k10 + col;
  const int zs = (int)d.zstride();  // N zs < 2^31 for every supported grid
  // inner iterations: stage this tile's FP64-residual source [3][N][cols] while the transform runs
  float2* vs = reinterpret_cast<float2*>(buf + ZS * N);
  // (2, 4 or 8 columns in 16-byte granules of two columns.  The row pitch P is a multiple of 4, so a
  // granule lies wholly inside or wholly beyond the row; granules at or beyond P are not copied (an
  // 8-column tile can reach past P, and past the end of the buffer on its last row), and the
  // columns they would hold are never read.)
  const bool stage_v = (mode == PZ_INNER) && (cols == 2 || cols == 4 || cols == 8);
  if (stage_v) {
    const int per_row = cols / 2;  // 16-byte granules per row
    for (int i = threadIdx.x; i < 3 * N * per_row; i += blockDim.x) {
      const int gr = i % per_row, rz = i / per_row;
      const int z = rz % N, c = rz / N;
      if (k10 + 2 * gr >= d.P) continue;
      cp_async16(vs + (c * N + z) * cols + 2 * gr, vsrc + c * d.S + d.row(z, k2) * d.P + k10 + 2 * gr);
    }
  }
  T v[P::E];
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) {
      T x; x.x = 0; x.y = 0;
      if (live) x = g[cin_idx<N, 0>(t, b, r) * zs];
      v[b * P::R(0) + r] = x;
    }
  __syncthreads();
  const SLine<T, false> sl{buf + l, ZS};
  cfft<N, false>(v, sl, t, twl);
  constexpr int RL = P::R(P::NST - 1);
#pragma unroll
  for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) sl[cout_idx<N, P::NST - 1>(t, b, r)] = v[b * RL + r];
  if (stage_v) cp_async_wait_all();
  __syncthreads();
  // Green operator, residual and T(0) per (k3, column)
  R acc2 = 0;
  const R acc = green_tile<R, N>(buf, ZS, cols, 0, ab3, stage_v ? vs : nullptr, d, k10, k2, gp, st, mode, vsrc,
                                 &acc2);
  if (sizeof(R) == 8 && mode == PZ_GAMMA && gp.vprev) {
    const double s2 = block_sum((double)acc2, red);
    if (threadIdx.x == 0) gp.cpart[blockIdx.y * gridDim.x + blockIdx.x] = s2;
    __syncthreads();
  }
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
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) v[b * P::R(0) + r] = sl[cin_idx<N, 0>(t, b, r)];
  __syncthreads();
  cfft<N, true>(v, sl, t, twl);
  if (live) {
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) g[cout_idx<N, P::NST - 1>(t, b, r) * zs] = v[b * RL + r];
  }
}

// ------------------------------------------------------------------------------------------------
// pass_z_gamma with 8-column tiles and two lines per thread (FP32, E <= 16): thread (l, t), l < 24,
// transforms line l (components 0-2) from registers and line l + 24 (components 3-5), which cp.async
// brings into the tile while line l is transformed.  The 6-component z-columns are read in 64-byte
// row segments, which the DRAM serves about twice as fast as the 32-byte segments of 4-column tiles,
// at the occupancy of the 4-column kernel (two CTAs of 24 T threads per SM; the unpadded tile is
// 48 N elements).  The inner-iteration source is read from global memory in the Green step.
// ------------------------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(24 * CPlan<N>::T, 2) pass_z_c2_kernel(typename C<R>::T* __restrict__ spec,
                                                       const typename C<R>::T* __restrict__ tw, Dims d,
                                                       GammaParams<R> gp, double* __restrict__ partials,
                                                       SolveState* __restrict__ st, int mode, float2* __restrict__ vsrc) {
  typedef typename C<R>::T T;
  typedef CPlan<N> P;
  constexpr int COLS = 8, ZS = 6 * COLS;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* twl = reinterpret_cast<T*>(smem_raw);
  T* ab3 = twl + N;
  T* buf = ab3 + N;                          // [k3][48]: component c, column cc at 8 c + cc
  __shared__ double red[32];
  const int k10 = blockIdx.x * COLS;
  const int k2 = blockIdx.y;
  // components 3-5 into the tile: 16-byte granules of two columns; the row pitch P is a multiple of
  // 4, so granules at or beyond P (dead columns of the last tile) are skipped and never read
  for (int i = threadIdx.x; i < 3 * N * (COLS / 2); i += blockDim.x) {
    const int gr = i % (COLS / 2), rz = i / (COLS / 2);
    const int z = rz % N, c = 3 + rz / N;
    if (k10 + 2 * gr >= d.P) continue;
    const int sw = (z & 1) ? 8 : 0;
    cp_async16(buf + z * ZS + ((c * COLS + 2 * gr) ^ sw), spec + c * d.S + d.row(z, k2) * d.P + k10 + 2 * gr);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    twl[i] = tw[i];
    T ab;
    ab.x = gp.A[2][i];
    ab.y = gp.B[2][i];
    ab3[i] = ab;
  }
  const int l = threadIdx.x % 24, t = threadIdx.x / 24;
  const int col = l % COLS;
  const bool live = k10 + col < d.n1h;
  const int zs = (int)d.zstride();  // N zs < 2^31 for every supported grid
  T* gA = spec + (l / COLS) * d.S + d.row(0, k2) * d.P + k10 + col;
  T* gB = gA + 3 * d.S;
  const SLineX<T> slA{buf, l}, slB{buf, l + 24};
  constexpr int RL = P::R(P::NST - 1);
  T v[P::E];
  // line A: global -> registers -> forward transform -> tile
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) {
      T x; x.x = 0; x.y = 0;
      if (live) x = gA[cin_idx<N, 0>(t, b, r) * zs];
      v[b * P::R(0) + r] = x;
    }
  __syncthreads();
  cfft<N, false>(v, slA, t, twl);
#pragma unroll
  for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) slA[cout_idx<N, P::NST - 1>(t, b, r)] = v[b * RL + r];
  // line B: tile -> registers -> forward transform -> tile
  cp_async_wait_all();
  __syncthreads();
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) {
      T x = slB[cin_idx<N, 0>(t, b, r)];
      if (!live) { x.x = 0; x.y = 0; }
      v[b * P::R(0) + r] = x;
    }
  __syncthreads();
  cfft<N, false>(v, slB, t, twl);
#pragma unroll
  for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) slB[cout_idx<N, P::NST - 1>(t, b, r)] = v[b * RL + r];
  __syncthreads();
  const R acc = green_tile<R, N>(buf, ZS, COLS, 8, ab3, nullptr, d, k10, k2, gp, st, mode, vsrc);
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
  // inverse transforms: tile -> registers -> global, line A then line B
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) v[b * P::R(0) + r] = slA[cin_idx<N, 0>(t, b, r)];
  __syncthreads();
  cfft<N, true>(v, slA, t, twl);
  if (live) {
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) gA[cout_idx<N, P::NST - 1>(t, b, r) * zs] = v[b * RL + r];
  }
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) v[b * P::R(0) + r] = slB[cin_idx<N, 0>(t, b, r)];
  __syncthreads();
  cfft<N, true>(v, slB, t, twl);
  if (live) {
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) gB[cout_idx<N, P::NST - 1>(t, b, r) * zs] = v[b * RL + r];
  }
}

// ------------------------------------------------------------------------------------------------
// pass_x: CTA = `lines` x1-lines (consecutive i2 at fixed i3) x 3 component pairs; thread = (pair
// line, t).  Same flags and correction as the generic kernel.
// ------------------------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(512) pass_x_c_kernel(typename C<R>::T* __restrict__ spec, R* __restrict__ eps,
                                                       const R* __restrict__ lam, const R* __restrict__ mu,
                                                       const typename C<R>::T* __restrict__ tw, Dims d, int lines,
                                                       int flags, const float* __restrict__ corr,
                                                       const double* __restrict__ corr_mean, PolarParams pp,
                                                       const SolveState* __restrict__ st) {
  typedef typename C<R>::T T;
  typedef CPlan<N> P;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  T* twl = reinterpret_cast<T*>(smem_raw);
  T* buf = twl + N;                          // [3 lines][N + N/16] (padded line-major)
  constexpr int LP = N + N / 16;
  constexpr int NH = N / 2 + 1;
  for (int i = threadIdx.x; i < N; i += blockDim.x) twl[i] = tw[i];
  const long long nlines = (long long)d.n2 * d.n3;
  const long long line0 = (long long)blockIdx.x * lines;
  const int t = threadIdx.x % P::T, fl = threadIdx.x / P::T;   // fl = pair * lines + l
  const int p = fl / lines, l = fl % lines;
  const long long li = line0 + l;
  const bool live = (fl < 3 * lines) && (li < nlines);
  const bool zero = (flags & PX_ZERO) != 0 || st->restart;
  const bool have_delta = (flags & PX_DELTA) != 0 && !st->restart;
  // eigenstrain and displacement output are FP64 features: compiled out of the FP32 instance, whose
  // registers (64) set its occupancy
  constexpr bool F64 = sizeof(R) == 8;
  const bool outmode = F64 && (flags & PX_OUTPUT) != 0, strainmode = F64 && (flags & PX_STRAIN) != 0;
  const bool dres = F64 && (flags & PX_DRES) != 0;
  const SLine<T, true> sl{buf + fl * LP, 1};
  T v[P::E];
  if (have_delta) {
    const T* A = spec + (2 * p) * d.S + d.xrow(li) * d.P;
    const T* B = spec + (2 * p + 1) * d.S + d.xrow(li) * d.P;
#pragma unroll
    for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
      for (int r = 0; r < P::R(0); ++r) {
        const int x = cin_idx<N, 0>(t, b, r);
        T z; z.x = 0; z.y = 0;
        if (live) {
          const int k = x < NH ? x : N - x;
          T a = A[k], bb = B[k];
          if (k == 0 || 2 * k == N) { a.y = 0; bb.y = 0; }
          if (x < NH) { z.x = a.x - bb.y; z.y = a.y + bb.x; }      // A + iB
          else { z.x = a.x + bb.y; z.y = -a.y + bb.x; }            // conj(A) + i conj(B)
        }
        v[b * P::R(0) + r] = z;
      }
    __syncthreads();
    cfft<N, true>(v, sl, t, twl);
    constexpr int RL = P::R(P::NST - 1);
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) sl[cout_idx<N, P::NST - 1>(t, b, r)] = v[b * RL + r];
  }
  __syncthreads();
  const bool polar = (flags & PX_POLAR) != 0;
  double dacc = 0.0;
  double cm[6];
  if (corr) {
#pragma unroll
    for (int c = 0; c < 6; ++c) cm[c] = corr_mean[c];
  }
  // XU voxels per step, all their loads issued before any store: a plain loop waits one DRAM latency
  // per voxel, since its strain loads are ordered after the previous voxel's stores to the same array
  // (FP32: 2 voxels at 64 registers; FP64 keeps 1, its registers are already at the launch bound)
  constexpr int XU = sizeof(R) == 4 ? 2 : 1;
  const int nvox = lines * N;
  for (int i0 = threadIdx.x; i0 < nvox; i0 += XU * blockDim.x) {
    R eu[XU][6], lu[XU], mu_[XU];
#pragma unroll
    for (int u = 0; u < XU; ++u) {
      const int i = i0 + u * blockDim.x;
      const long long lj = line0 + i / N;
      const bool ok = i < nvox && lj < nlines;
      const long long vv = lj * N + i % N;
#pragma unroll
      for (int c = 0; c < 6; ++c) eu[u][c] = (ok && !zero && !outmode) ? eps[c * d.N + vv] : (R)0;
      lu[u] = ok ? lam[vv] : (R)0;
      mu_[u] = ok ? mu[vv] : (R)0;
    }
#pragma unroll
    for (int u = 0; u < XU; ++u) {
    const int i = i0 + u * blockDim.x;
    const int x = i % N, ll = i / N;
    const long long lj = line0 + ll;
    if (i >= nvox || lj >= nlines) continue;
    const long long vv = lj * N + x;
    const int px = x + (x >> 4);
    R e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eu[u][c];
    if (have_delta) {
      R dd[6];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const T z = buf[(q * lines + ll) * LP + px];
        dd[2 * q] = z.x;
        dd[2 * q + 1] = z.y;
      }
      if (outmode) {
#pragma unroll
        for (int c = 0; c < 3; ++c) eps[c * d.N + vv] = dd[c];
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
      for (int c = 0; c < 6; ++c) e[c] += (R)((double)corr[c * d.N + vv] - cm[c]);
    }
    if (have_delta || zero || corr) {
#pragma unroll
      for (int c = 0; c < 6; ++c) eps[c * d.N + vv] = e[c];
    }
    T zz[3];
    if (strainmode) {
      zz[0].x = e[0] - (R)pp.E[0]; zz[0].y = e[1] - (R)pp.E[1];
      zz[1].x = e[2] - (R)pp.E[2]; zz[1].y = e[3] - (R)pp.E[3];
      zz[2].x = e[4] - (R)pp.E[4]; zz[2].y = e[5] - (R)pp.E[5];
    } else if (polar) pack_stress<R>(e, lu[u] - (R)pp.lam_h, mu_[u] - (R)pp.mu_h, zz);
    else if (F64 && pp.estar) {
      R es[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) es[c] = e[c] - (R)pp.estar[c * d.N + vv];
      pack_stress<R>(es, lu[u], mu_[u], zz);
    } else pack_stress<R>(e, lu[u], mu_[u], zz);
#pragma unroll
    for (int q = 0; q < 3; ++q) buf[(q * lines + ll) * LP + px] = zz[q];
    }
  }
  if (outmode) return;
  if ((polar || dres) && have_delta) {
    const double sum = block_sum(dacc, red);
    if (threadIdx.x == 0) pp.partials[blockIdx.x] = sum;
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) v[b * P::R(0) + r] = sl[cin_idx<N, 0>(t, b, r)];
  __syncthreads();
  cfft<N, false>(v, sl, t, twl);
  {
    constexpr int RL = P::R(P::NST - 1);
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) sl[cout_idx<N, P::NST - 1>(t, b, r)] = v[b * RL + r];
  }
  __syncthreads();
  // split Z = FFT(a + i b) into the half spectra of a and b
  for (int i = threadIdx.x; i < 3 * lines * NH; i += blockDim.x) {
    const int k = i % NH, f = i / NH;
    const int q = f / lines, ll = f % lines;
    const long long lj = line0 + ll;
    if (lj >= nlines) continue;
    const T* line = buf + f * LP;
    const int kn = (N - k) % N;
    const T zk = line[k + (k >> 4)];
    const T zn = line[kn + (kn >> 4)];
    T A, B;
    A.x = (R)0.5 * (zk.x + zn.x); A.y = (R)0.5 * (zk.y - zn.y);
    B.x = (R)0.5 * (zk.y + zn.y); B.y = (R)-0.5 * (zk.x - zn.x);
    const long long row = d.xrow(lj) * d.P;
    spec[(2 * q) * d.S + row + k] = A;
    spec[(2 * q + 1) * d.S + row + k] = B;
  }
}

// ------------------------------------------------------------------------------------------------
// pass_x with asynchronous staging: the CTA first copies its spectrum rows, strain rows and Lame
// rows into shared memory with cp.async (16-byte granules, L2 only), so that all loads are in flight
// at once, then runs the same transform / update / stress / transform sequence as pass_x_c_kernel
// from shared memory.  Meant for small CTAs (few lines), several resident per SM.
// ------------------------------------------------------------------------------------------------

template <typename R, int N>
__host__ __device__ constexpr int xa_spec_pitch() {  // complex elements per staged spectrum row (16-byte multiple)
  return ((N / 2 + 1) * (int)sizeof(typename C<R>::T) + 15) / 16 * 16 / (int)sizeof(typename C<R>::T);
}

template <typename R, int N>
__host__ __device__ constexpr size_t xa_smem_bytes(int lines) {
  typedef typename C<R>::T T;
  return sizeof(T) * (size_t)(N + 3 * lines * (N + N / 16) + 6 * lines * xa_spec_pitch<R, N>()) +
         sizeof(R) * (size_t)(8 * lines * N);
}

template <typename R, int N>
__global__ void __launch_bounds__(512) pass_x_a_kernel(typename C<R>::T* __restrict__ spec, R* __restrict__ eps,
                                                       const R* __restrict__ lam, const R* __restrict__ mu,
                                                       const typename C<R>::T* __restrict__ tw, Dims d, int lines,
                                                       int flags, const float* __restrict__ corr,
                                                       const double* __restrict__ corr_mean,
                                                       const SolveState* __restrict__ st) {
  typedef typename C<R>::T T;
  typedef CPlan<N> P;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LP = N + N / 16;
  constexpr int NH = N / 2 + 1;
  constexpr int SP = xa_spec_pitch<R, N>();
  T* sspec = reinterpret_cast<T*>(smem_raw);                 // [6][lines][SP]
  T* twl = sspec + 6 * lines * SP;                           // [N]
  T* buf = twl + N;                                          // [3 lines][LP]
  R* sst = reinterpret_cast<R*>(buf + 3 * lines * LP);       // [8][lines][N]: eps 0..5, lambda, mu
  const long long nlines = (long long)d.n2 * d.n3;
  const long long line0 = (long long)blockIdx.x * lines;
  const bool zero = (flags & PX_ZERO) != 0 || st->restart;
  const bool have_delta = (flags & PX_DELTA) != 0 && !st->restart;
  // ---- stage everything this CTA reads
  {
    constexpr int spec_chunks = SP * (int)sizeof(T) / 16;     // 16-byte granules per spectrum row
    constexpr int row_chunks = N * (int)sizeof(R) / 16;      // per real row
    const int nsp = have_delta ? 6 * lines * spec_chunks : 0;
    const int nre = (zero ? 2 : 8) * lines * row_chunks;
    for (int i = threadIdx.x; i < nsp + nre; i += blockDim.x) {
      if (i < nsp) {
        const int ch = i % spec_chunks, cl = i / spec_chunks;
        const int l = cl % lines, c = cl / lines;
        const long long li = line0 + l;
        if (li >= nlines) continue;
        cp_async16(reinterpret_cast<unsigned char*>(sspec + (c * lines + l) * SP) + 16 * ch,
                   reinterpret_cast<const unsigned char*>(spec + c * d.S + d.xrow(li) * d.P) + 16 * ch);
      } else {
        const int j = i - nsp;
        const int ch = j % row_chunks, ql = j / row_chunks;
        const int l = ql % lines, q0 = ql / lines;
        const int q = zero ? 6 + q0 : q0;
        const long long li = line0 + l;
        if (li >= nlines) continue;
        const R* src = q < 6 ? eps + q * d.N + li * N : (q == 6 ? lam + li * N : mu + li * N);
        cp_async16(reinterpret_cast<unsigned char*>(sst + (q * lines + l) * N) + 16 * ch,
                   reinterpret_cast<const unsigned char*>(src) + 16 * ch);
      }
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) twl[i] = tw[i];
  cp_async_wait_all();
  __syncthreads();
  const int t = threadIdx.x % P::T, fl = threadIdx.x / P::T;   // fl = pair * lines + l
  const int p = fl / lines, l = fl % lines;
  const SLine<T, true> sl{buf + fl * LP, 1};
  T v[P::E];
  if (have_delta) {
    const T* A = sspec + (2 * p * lines + l) * SP;
    const T* B = sspec + ((2 * p + 1) * lines + l) * SP;
#pragma unroll
    for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
      for (int r = 0; r < P::R(0); ++r) {
        const int x = cin_idx<N, 0>(t, b, r);
        const int k = x < NH ? x : N - x;
        T a = A[k], bb = B[k];
        if (k == 0 || 2 * k == N) { a.y = 0; bb.y = 0; }
        T z;
        if (x < NH) { z.x = a.x - bb.y; z.y = a.y + bb.x; }      // A + iB
        else { z.x = a.x + bb.y; z.y = -a.y + bb.x; }            // conj(A) + i conj(B)
        v[b * P::R(0) + r] = z;
      }
    cfft<N, true>(v, sl, t, twl);
    constexpr int RL = P::R(P::NST - 1);
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) sl[cout_idx<N, P::NST - 1>(t, b, r)] = v[b * RL + r];
  }
  __syncthreads();
  double cm[6];
  if (corr) {
#pragma unroll
    for (int c = 0; c < 6; ++c) cm[c] = corr_mean[c];
  }
  for (int i = threadIdx.x; i < lines * N; i += blockDim.x) {
    const int x = i % N, ll = i / N;
    const long long lj = line0 + ll;
    if (lj >= nlines) continue;
    const long long vv = lj * N + x;
    const int px = x + (x >> 4);
    R e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = zero ? (R)0 : sst[(c * lines + ll) * N + x];
    if (have_delta) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const T z = buf[(q * lines + ll) * LP + px];
        e[2 * q] += z.x;
        e[2 * q + 1] += z.y;
      }
    }
    if (corr) {
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] += (R)((double)corr[c * d.N + vv] - cm[c]);
    }
    if (have_delta || zero || corr) {
#pragma unroll
      for (int c = 0; c < 6; ++c) eps[c * d.N + vv] = e[c];
    }
    const R la = sst[(6 * lines + ll) * N + x], m2 = (R)2 * sst[(7 * lines + ll) * N + x];
    const R ltr = la * (e[0] + e[1] + e[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T z;
      z.x = m2 * e[2 * q] + (q < 2 ? ltr : (R)0);        // 11, 33, 13
      z.y = m2 * e[2 * q + 1] + (q == 0 ? ltr : (R)0);   // 22, 23, 12
      buf[(q * lines + ll) * LP + px] = z;
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < P::E / P::R(0); ++b)
#pragma unroll
    for (int r = 0; r < P::R(0); ++r) v[b * P::R(0) + r] = sl[cin_idx<N, 0>(t, b, r)];
  __syncthreads();
  cfft<N, false>(v, sl, t, twl);
  {
    constexpr int RL = P::R(P::NST - 1);
#pragma unroll
    for (int b = 0; b < P::E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) sl[cout_idx<N, P::NST - 1>(t, b, r)] = v[b * RL + r];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * lines * NH; i += blockDim.x) {
    const int k = i % NH, f = i / NH;
    const int q = f / lines, ll = f % lines;
    const long long lj = line0 + ll;
    if (lj >= nlines) continue;
    const T* line = buf + f * LP;
    const int kn = (N - k) % N;
    const T zk = line[k + (k >> 4)];
    const T zn = line[kn + (kn >> 4)];
    T A, B;
    A.x = (R)0.5 * (zk.x + zn.x); A.y = (R)0.5 * (zk.y - zn.y);
    B.x = (R)0.5 * (zk.y + zn.y); B.y = (R)-0.5 * (zk.x - zn.x);
    const long long row = d.xrow(lj) * d.P;
    spec[(2 * q) * d.S + row + k] = A;
    spec[(2 * q + 1) * d.S + row + k] = B;
  }
}

}  // namespace gfp
