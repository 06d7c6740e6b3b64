// TMA-fed, software-pipelined z-pass (sm_103a).
//
// Persistent CTAs walk the (k2, k1-chunk) tiles.  One elected thread loads each tile -- 6 components
// x n3 rows x C columns of the half spectrum -- with cp.async.bulk.tensor into one of two shared-memory
// buffers, signalling an mbarrier, while the CTA transforms, applies the Green operator to, and
// inverse-transforms the previous tile.  Every wait on an mbarrier is bounded: after about a second it
// marks the solve as timed out (SolveState::done = 4) and the CTA stops issuing work.
//
// The 8-column variant (pass_z_s_kernel, FP32 inner iterations, square plans N = T^2) loads its
// whole tile with TMA in the 64-byte swizzle, transforms each line with T lanes of one warp that
// exchange through __shfl_sync instead of shared memory, and stores the tile back with a TMA store.
#pragma once
#include <cuda.h>

#include "gfp_fftc.cuh"

namespace gfp {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false after `budget` cycles of polling (default 2^31,
// about a second).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  long long budget = (1LL << 31)) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// Tensor map of the half spectrum seen as a 4D array of reals: {2 P (re/im interleaved), n2, n3, 6};
// the box is {2 C, 1, min(n3, 256), 1}, so one load brings C columns x up to 256 rows of one component.
template <typename R, int N>
__global__ void __launch_bounds__(384, ZBound<R, N>::blocks) pass_z_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                            typename C<R>::T* __restrict__ spec,
                                                            const typename C<R>::T* __restrict__ tw, Dims d, int cols,
                                                            int ntx, GammaParams<R> gp, double* __restrict__ partials,
                                                            SolveState* __restrict__ st, int mode,
                                                            float2* __restrict__ vsrc, unsigned inject_timeout) {
  typedef typename C<R>::T T;
  typedef CPlan<N> P;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned: align the dynamic region by hand (the launch adds
  // 128 bytes for this)
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int tile_elems = 6 * N * cols;
  T* tiles[2];
  tiles[0] = reinterpret_cast<T*>(base);
  tiles[1] = tiles[0] + tile_elems;
  T* twl = tiles[1] + tile_elems;
  __shared__ __align__(8) unsigned long long bars[3];  // two tile buffers; [2] is never arrived at
  __shared__ double red[32];
  __shared__ int abort_flag;
  if ((smem_u32(tiles[0]) & 127u) != 0 || (smem_u32(tiles[1]) & 127u) != 0) {  // never issue a misaligned TMA
    if (threadIdx.x == 0) atomicExch(&st->done, (int)DONE_TIMEOUT);
    return;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) twl[i] = tw[i];
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  __syncthreads();
  const int ntiles = ntx * d.n2;
  const int w6 = 6 * cols;
  const int l = threadIdx.x % w6, t = threadIdx.x / w6;
  const int comp = l / cols, col = l % cols;
  const unsigned tile_bytes = (unsigned)(tile_elems * sizeof(T));
  constexpr int ZB = N < 256 ? N : 256;
  auto issue = [&](int tile, int b) {
    const int k2 = tile / ntx, k10 = (tile % ntx) * cols;
    mbar_expect_tx(&bars[b], tile_bytes);
    for (int c = 0; c < 6; ++c)
      for (int z0 = 0; z0 < N; z0 += ZB)
        tma_load_4d(tiles[b] + (c * N + z0) * cols, &tmap, &bars[b], 2 * k10, k2, z0, c);
  };
  if (threadIdx.x == 0 && blockIdx.x < ntiles) issue(blockIdx.x, 0);
  int k = 0;
  int inflight_next = 0;  // the load of the next tile was issued in this iteration
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int b = k & 1;
    T* buf = tiles[b];
    const int next = tile + gridDim.x;
    inflight_next = 0;
    if (threadIdx.x == 0 && next < ntiles) {
      issue(next, b ^ 1);
      inflight_next = 1;
    }
    if (threadIdx.x == 0) {
      // inject_timeout (tests of failure detection): wait instead, with a budget of 2^22 cycles, on
      // bars[2], which nothing arrives at, so the wait runs out; the tile loads keep their true byte
      // counts, so the drain below confirms that they have landed
      const bool ok = inject_timeout ? mbar_wait_bounded(&bars[2], 0, 1LL << 22)
                                     : mbar_wait_bounded(&bars[b], (k >> 1) & 1);
      if (!ok) abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag) {
      if (threadIdx.x == 0) {
        atomicExch(&st->done, (int)DONE_TIMEOUT);
        // loads still in flight land in this CTA's shared memory: wait for them (bounded) first
        mbar_wait_bounded(&bars[b], (k >> 1) & 1);
        if (inflight_next) mbar_wait_bounded(&bars[b ^ 1], ((k + 1) >> 1) & 1);
      }
      return;
    }
    const int k2 = tile / ntx, k10 = (tile % ntx) * cols;
    const bool live = k10 + col < d.n1h;
    const SLine<T, false> sl{buf + comp * N * cols + col, cols};
    T v[P::E];
#pragma unroll
    for (int bb = 0; bb < P::E / P::R(0); ++bb)
#pragma unroll
      for (int r = 0; r < P::R(0); ++r) v[bb * P::R(0) + r] = sl[cin_idx<N, 0>(t, bb, r)];
    __syncthreads();
    cfft<N, false>(v, sl, t, twl);
    constexpr int RL = P::R(P::NST - 1);
#pragma unroll
    for (int bb = 0; bb < P::E / RL; ++bb)
#pragma unroll
      for (int r = 0; r < RL; ++r) sl[cout_idx<N, P::NST - 1>(t, bb, r)] = v[bb * RL + r];
    __syncthreads();
    // Green operator, residual and T(0) per (k3, column)
    R tacc = 0;
    const bool ny2 = ((d.n2 & 1) == 0) && (2 * k2 == d.n2);
    const R b2 = gp.B[1][k2], a2 = gp.A[1][k2];
    for (int i = threadIdx.x; i < N * cols; i += blockDim.x) {
      const int cc = i % cols, z = i / cols;
      const int k1 = k10 + cc;
      if (k1 >= d.n1h) continue;
      T tt[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) tt[c] = buf[(c * N + z) * cols + cc];
      const R a1 = gp.A[0][k1], b1 = gp.B[0][k1];
      const R a3 = gp.A[2][z], b3 = gp.B[2][z];
      const R kt1 = a1 * b2 * b3, kt2 = a2 * b3 * b1, kt3 = a3 * b1 * b2;
      const bool ny1 = ((d.n1 & 1) == 0) && (2 * k1 == d.n1);
      const bool ny3 = (2 * z == N);
      const bool self1 = (k1 == 0) || ny1;
      const long long vi = d.row(z, k2) * d.P + k1;
      if (mode != PZ_INNER && k1 == 0 && k2 == 0 && z == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) st->T0[c] = (double)tt[c].x;
      }
      T v1, v2, v3;
      tk_vec<R>(tt, kt1, kt2, kt3, v1, v2, v3);
      if (mode == PZ_INNER) {
        const float2 s1 = vsrc[vi], s2 = vsrc[d.S + vi], s3 = vsrc[2 * d.S + vi];
        v1.x += (R)s1.x; v1.y += (R)s1.y; v2.x += (R)s2.x; v2.y += (R)s2.y; v3.x += (R)s3.x; v3.y += (R)s3.y;
      }
      R r2 = vnorm2(v1, v2, v3);
      if (!self1) {
        if (gp.nyq_avg && (ny2 || ny3)) r2 += tk_norm2<R>(tt, kt1, ny2 ? -kt2 : kt2, ny3 ? -kt3 : kt3);
        else r2 *= (R)2;
      }
      tacc += r2;
      if (mode == PZ_RESIDUAL) {
        float2 o1, o2, o3;
        o1.x = (float)v1.x; o1.y = (float)v1.y; o2.x = (float)v2.x; o2.y = (float)v2.y;
        o3.x = (float)v3.x; o3.y = (float)v3.y;
        vsrc[vi] = o1; vsrc[d.S + vi] = o2; vsrc[2 * d.S + vi] = o3;
        continue;
      }
      T o[6];
      gamma0_from_v<R>(v1, v2, v3, kt1, kt2, kt3, gp.c_mu, gp.c_lm, gp.invN, o);
      if (gp.nyq_avg && (ny1 || ny2 || ny3)) {
        T o2[6];
        gamma0_apply<R>(tt, ny1 ? -kt1 : kt1, ny2 ? -kt2 : kt2, ny3 ? -kt3 : kt3, gp.c_mu, gp.c_lm, gp.invN, o2);
#pragma unroll
        for (int c = 0; c < 6; ++c) { o[c].x = (R)0.5 * (o[c].x + o2[c].x); o[c].y = (R)0.5 * (o[c].y + o2[c].y); }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) buf[(c * N + z) * cols + cc] = o[c];
    }
    // per-tile residual partial, deterministic order
    double accd = (double)tacc;
    for (int off = 16; off > 0; off >>= 1) accd += __shfl_down_sync(0xffffffffu, accd, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = accd;
    __syncthreads();
    if (threadIdx.x < 32) {
      const int nw = (blockDim.x + 31) >> 5;
      double s = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (threadIdx.x == 0) partials[tile] = s;
    }
    if (mode != PZ_RESIDUAL) {
#pragma unroll
      for (int bb = 0; bb < P::E / P::R(0); ++bb)
#pragma unroll
        for (int r = 0; r < P::R(0); ++r) v[bb * P::R(0) + r] = sl[cin_idx<N, 0>(t, bb, r)];
      __syncthreads();
      cfft<N, true>(v, sl, t, twl);
      if (live) {
        T* g = spec + comp * d.S + d.row(0, k2) * d.P + k10 + col;
        const long long zs = d.zstride();
#pragma unroll
        for (int bb = 0; bb < P::E / RL; ++bb)
#pragma unroll
          for (int r = 0; r < RL; ++r) g[cout_idx<N, P::NST - 1>(t, bb, r) * zs] = v[bb * RL + r];
      }
    }
    fence_proxy_async();  // order this tile's generic shared accesses before the next async load into it
    __syncthreads();      // both the tile buffer and red[] are free for the next tile
  }
}


// TMA store of a 4D box from shared memory (bulk group; the issuing thread waits for its reads).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map), "r"(c0),
      "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait_read() {
  asm volatile("cp.async.bulk.commit_group;\n\tcp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Byte offset inside a 512-byte-aligned region as laid out by the 64-byte TMA swizzle
// (CU_TENSOR_MAP_SWIZZLE_64B): the 16-byte chunk index (bits 4-5) is XORed with bits 7-8.
__device__ __forceinline__ unsigned swz64(unsigned off) { return off ^ (((off >> 7) & 3u) << 4); }

// a[j] <- a[(j - s) mod T] for a lane-dependent s in [0, T): one conditional move per bit of s.
template <int T_, typename V>
__device__ __forceinline__ void rot_right(V* a, int s) {
#pragma unroll
  for (int b = 1; b < T_; b <<= 1) {
    const bool f = (s & b) != 0;
    V tmp[T_];
#pragma unroll
    for (int j = 0; j < T_; ++j) tmp[j] = a[(j - b + T_) % T_];
#pragma unroll
    for (int j = 0; j < T_; ++j) a[j] = f ? tmp[j] : a[j];
  }
}

// Line transform of length N = T^2 on the T lanes of a group (Stockham, two radix-T stages, one
// exchange of T shuffle rounds).  On entry v[r] = x[t + T r]; on return v[k] = X[t + T k].
// Stage 0 gives lane t the values y_k = sum_m x[t + T m] w^{m k} (w = w_T, the transform's sign), of
// which y_k is lane k's stage-1 input t.  The exchange needs them rotated by the lane, u_j = y_{(t - j)
// mod T}, so that round j can send one register j to every lane; instead of moving registers, the
// rotation is computed: y_{t - j} = sum_m (x_m w^{m t}) w^{-m j}, a transform of the opposite sign of
// the inputs scaled by w^{m t}.  After round j lane t holds in register j the stage-1 input from
// position (t + j) mod T (already multiplied by its twiddle w_N^{s t} at the sender), which a register
// rotation by t puts in order.  Tables in shared memory, read by consecutive lanes at compile-time
// offsets: rt[m T + t] = w_T^{m t} and tw3[j T + t] = w_N^{t ((t - j) mod T)} (forward sign).
// Phased forms: without ROT the final rotation is skipped, and since lane t's stage-1 inputs then sit
// at positions (t + j) mod T, output k comes out as w^{-t k} X[t + T k] = conj(rt[t + T k]) X (forward
// sign); without PRE the input scaling by w^{m t} is skipped, i.e. the inputs must arrive already
// multiplied by it -- which is exactly what a phased forward output, passed through a pointwise linear
// step with real coefficients, is for the inverse transform (w_inv^{m t} = conj(w_fwd^{m t})).
template <int N, bool INV, bool PRE = true, bool ROT = true>
__device__ __forceinline__ void sfft(float2* v, int t, int h, const float2* tw3, const float2* rt) {
  constexpr int T_ = CPlan<N>::T, LPW = 32 / T_;
  if (PRE) {
#pragma unroll
    for (int m = 1; m < T_; ++m) {  // x_m w^{m t}
      float2 w = rt[m * T_ + t];
      if (INV) w.y = -w.y;
      v[m] = cmul(v[m], w);
    }
  }
  Dft<T_, !INV, float2>::run(v);  // v[j] = y_{(t - j) mod T}, destined to lane (t - j) mod T
#pragma unroll
  for (int j = 0; j < T_; ++j) {  // its stage-1 twiddle w_N^{t (t - j)}
    float2 w = tw3[j * T_ + t];
    if (INV) w.y = -w.y;
    v[j] = cmul(v[j], w);
  }
#pragma unroll
  for (int j = 1; j < T_; ++j) {  // round j: from position (t + j) mod T, its register j
    const int src = LPW * ((t + j) & (T_ - 1)) + h;
    float2 w;
    w.x = __shfl_sync(0xffffffffu, v[j].x, src);
    w.y = __shfl_sync(0xffffffffu, v[j].y, src);
    v[j] = w;
  }
  if (ROT) rot_right<T_>(v, t);  // v[s] = stage-1 input s
  Dft<T_, INV, float2>::run(v);
}

// ------------------------------------------------------------------------------------------------
// pass_z_gamma with 8-column tiles, TMA in and out, warp-shuffle line transforms (FP32 inner iterations
// of the mixed solve, PZ_INNER; square plans N = T^2 with N <= 256).  CTA = 8 k1 columns x 6 components
// x all n3 rows at fixed k2, 24 T threads: thread (line, t) with line = threadIdx.x / T transforms
// line A = (component line / 8, column line % 8) and line B (component + 3).  The tile is
// [6][N rows][8 columns] of float2 in the 64-byte swizzle, so that the lane pattern of the transforms
// (T rows of two adjacent columns per warp) and that of the Green step (4 rows x 8 columns per warp)
// both touch each bank pair twice per warp access, the minimum for 256 bytes.  The Green step takes
// all its FP64-residual sources from global memory in batches before its arithmetic.
// ------------------------------------------------------------------------------------------------
template <int N> struct SPlanOk {
  static constexpr bool ok = CPlan<N>::ok && CPlan<N>::NST == 2 && CPlan<N>::R(0) == CPlan<N>::T &&
                             CPlan<N>::R(1) == CPlan<N>::T && CPlan<N>::E == CPlan<N>::T && N <= 256;
};
template <int N> constexpr size_t zs_smem_bytes() {
  return (size_t)6 * N * 64 + 1024 + (size_t)3 * N * sizeof(float2);
}

template <int N>
__global__ void __launch_bounds__(24 * CPlan<N>::T, 2) pass_z_s_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                      const float2* __restrict__ tw, Dims d,
                                                                      GammaParams<float> gp,
                                                                      double* __restrict__ partials,
                                                                      SolveState* __restrict__ st,
                                                                      const float2* __restrict__ vsrc) {
  constexpr int T_ = CPlan<N>::T, COLS = 8, NT = 24 * T_;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the swizzle pattern repeats every 512 bytes and TMA destinations with it must be so aligned:
  // align the tile to 1024 bytes by hand (the launch adds 1024 bytes for this)
  unsigned char* tile = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float2* twl = reinterpret_cast<float2*>(tile + 6 * N * 64);
  float2* ab3 = twl + N;
  float2* roots = ab3 + N;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ double red[32];
  __shared__ int abort_flag;
  const int k10 = blockIdx.x * COLS, k2 = blockIdx.y;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, 6u * N * 64u);
    for (int c = 0; c < 6; ++c) tma_load_4d(tile + c * N * 64, &tmap, &bar, 2 * k10, k2, 0, c);
  }
  for (int i = threadIdx.x; i < N; i += NT) {
    const int tt = i % T_, jj = i / T_;
    twl[i] = tw[tt * ((tt - jj + T_) % T_)];        // twl[j T + t] = w_N^{t ((t - j) mod T)}
    roots[i] = tw[T_ * ((tt * jj) % T_)];            // roots[m T + t] = w_T^{m t} = w_N^{T (m t mod T)}
    float2 ab;
    ab.x = gp.A[2][i];
    ab.y = gp.B[2][i];
    ab3[i] = ab;
  }
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0)) abort_flag = 1;
  __syncthreads();
  if (abort_flag) {
    if (threadIdx.x == 0) {
      atomicExch(&st->done, (int)DONE_TIMEOUT);
      mbar_wait_bounded(&bar, 0);  // the loads land in this CTA's shared memory: wait (bounded) for them
    }
    return;
  }
  // lines interleaved in the warp: lane = LPW t + h, line = LPW warp + h
  constexpr int LPW = 32 / T_;
  const int lane = threadIdx.x & 31, h = lane % LPW, t = lane / LPW;
  const int line = (threadIdx.x >> 5) * LPW + h;
  const int col = line % COLS, compA = line / COLS;
  auto el = [&](int c, int z, int cc) -> float2& {
    return *reinterpret_cast<float2*>(tile + swz64((unsigned)(c * N * 64 + z * 64 + cc * 8)));
  };
  // forward transforms of lines A and B, in place (each thread owns rows t + T r of its lines)
#pragma unroll 1
  for (int ab = 0; ab < 2; ++ab) {
    const int c = compA + 3 * ab;
    float2 v[T_];
#pragma unroll
    for (int r = 0; r < T_; ++r) v[r] = el(c, t + T_ * r, col);
    sfft<N, false, true, false>(v, t, h, twl, roots);  // phased output: conj(roots[z]) X[z]
#pragma unroll
    for (int k = 0; k < T_; ++k) el(c, t + T_ * k, col) = v[k];
  }
  __syncthreads();
  // Green step: point p = threadIdx.x + NT q is (row p / 8, column p % 8)
  float acc = 0.f;
  {
    const int cc = threadIdx.x & 7;
    const int k1 = k10 + cc;
    const bool live = k1 < d.n1h;
    const bool ny2 = ((d.n2 & 1) == 0) && (2 * k2 == d.n2);
    (void)ny2;
    const float b2 = gp.B[1][k2], a2 = gp.A[1][k2];
    const float a1 = live ? gp.A[0][k1] : 0.f, b1 = live ? gp.B[0][k1] : 0.f;
    const bool self1 = (k1 == 0) || (((d.n1 & 1) == 0) && (2 * k1 == d.n1));
    constexpr int NQ = (N * COLS + NT - 1) / NT;
    constexpr int GB = NQ < 3 ? NQ : 3;
    float2 src[GB][3];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int z = (threadIdx.x + NT * q) >> 3;
      if (q % GB == 0) {
#pragma unroll
        for (int u = 0; u < GB; ++u) {
          const int zu = (threadIdx.x + NT * (q + u)) >> 3;
          if (q + u < NQ && zu < N && live) {
            const long long vi = d.row(zu, k2) * d.P + k1;
            src[u][0] = vsrc[vi];
            src[u][1] = vsrc[d.S + vi];
            src[u][2] = vsrc[2 * d.S + vi];
          }
        }
      }
      if (z >= N) continue;
      float2 o[6];
      if (live) {
        float2 tt[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) tt[c] = el(c, z, cc);
        const float2 ab = ab3[z];
        const float kt1 = a1 * b2 * ab.y, kt2 = a2 * ab.y * b1, kt3 = ab.x * b1 * b2;
        float2 v1, v2, v3;
        tk_vec<float>(tt, kt1, kt2, kt3, v1, v2, v3);
        // the tile holds conj(roots[z]) X[z] (phased forward transform): the Green step is linear with real
        // coefficients and |v|^2 ignores a common phase, so only the source needs the same phase
        const float2* s3 = src[q % GB];
        float2 ph = roots[z];
        ph.y = -ph.y;
        const float2 p1 = cmul(s3[0], ph), p2 = cmul(s3[1], ph), p3 = cmul(s3[2], ph);
        v1.x += p1.x; v1.y += p1.y; v2.x += p2.x; v2.y += p2.y; v3.x += p3.x; v3.y += p3.y;
        float r2 = vnorm2(v1, v2, v3);
        acc += self1 ? r2 : 2.f * r2;
        gamma0_from_v<float>(v1, v2, v3, kt1, kt2, kt3, gp.c_mu, gp.c_lm, gp.invN, o);
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) { o[c].x = 0.f; o[c].y = 0.f; }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) el(c, z, cc) = o[c];
    }
  }
  double accd = (double)acc;
  for (int off = 16; off > 0; off >>= 1) accd += __shfl_down_sync(0xffffffffu, accd, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = accd;
  __syncthreads();
  if (threadIdx.x < 32) {
    double sm = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) sm += __shfl_down_sync(0xffffffffu, sm, off);
    if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = sm;
  }
  // inverse transforms, in place
#pragma unroll 1
  for (int ab = 0; ab < 2; ++ab) {
    const int c = compA + 3 * ab;
    float2 v[T_];
#pragma unroll
    for (int r = 0; r < T_; ++r) v[r] = el(c, t + T_ * r, col);
    sfft<N, true, false, true>(v, t, h, twl, roots);   // phased input, true output
#pragma unroll
    for (int k = 0; k < T_; ++k) el(c, t + T_ * k, col) = v[k];
  }
  // the tile back to global memory: make the generic-proxy writes visible to the TMA unit first
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 6; ++c) tma_store_4d(&tmap, tile + c * N * 64, 2 * k10, k2, 0, c);
    bulk_commit_and_wait_read();
  }
}

}  // namespace gfp
