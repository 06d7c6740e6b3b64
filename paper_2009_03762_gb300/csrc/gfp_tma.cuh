// TMA-fed, software-pipelined z-pass (sm_103a).
//
// Persistent CTAs walk the (k2, k1-chunk) tiles.  One elected thread loads each tile -- 6 components
// x n3 rows x C columns of the half spectrum -- with cp.async.bulk.tensor into one of two shared-memory
// buffers, signalling an mbarrier, while the CTA transforms, applies the Green operator to, and
// inverse-transforms the previous tile.  Every wait on an mbarrier is bounded: after about a second it
// marks the solve as timed out (SolveState::done = 4) and the CTA stops issuing work.
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

}  // namespace gfp
