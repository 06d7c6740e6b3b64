// Shared-memory Stockham FFT of many lines at once (sm_103a).
//
// The 3D transforms of the solver (eq. DisFouMat3D: a product of 1D transforms along x1, x2, x3)
// are done one axis per pass.  Each pass stages a tile of complete lines in shared memory and runs
// the 1D transform on all of them: radix stages (2, 3, 4, 8, 16) in Stockham autosort order, each
// thread holding its butterflies in registers between one shared-memory read and one write.
//
// Sign and scale: forward uses e^{-2 pi i jk/n}, inverse e^{+2 pi i jk/n}, both unnormalised; the
// solver folds the unitary n^{-3/2} x n^{-3/2} = 1/N into the Green-operator step.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace gfp {

template <typename R> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float> { typedef float2 type; };

template <typename R> struct C {
  typedef typename cplx_t<R>::type T;
};

template <typename T> __device__ __forceinline__ T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename T> __device__ __forceinline__ T cconj(T a) { T r; r.x = a.x; r.y = -a.y; return r; }
template <typename T, typename R> __device__ __forceinline__ T cscale(T a, R s) { T r; r.x = a.x * s; r.y = a.y * s; return r; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename T> __device__ __forceinline__ T mul_mi(T a) {
  T r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// ---------------------------------------------------------------- small DFT kernels (in registers)
template <int RADIX, bool INV, typename T> struct Dft;

template <bool INV, typename T> struct Dft<2, INV, T> {
  __device__ __forceinline__ static void run(T* v) {
    T a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV, typename T> struct Dft<3, INV, T> {
  __device__ __forceinline__ static void run(T* v) {
    typedef decltype(T().x) R;
    const R s3 = (R)0.86602540378443864676;  // sqrt(3)/2
    T t = cadd(v[1], v[2]);
    T d = csub(v[1], v[2]);
    T x0 = cadd(v[0], t);
    T m; m.x = v[0].x - (R)0.5 * t.x; m.y = v[0].y - (R)0.5 * t.y;
    // forward: X1 = m - i s3 d, X2 = m + i s3 d; inverse swaps the sign of i
    T id = mul_mi<INV>(d);  // -i d (fwd) / +i d (inv)
    v[0] = x0;
    v[1].x = m.x + s3 * id.x; v[1].y = m.y + s3 * id.y;
    v[2].x = m.x - s3 * id.x; v[2].y = m.y - s3 * id.y;
  }
};

template <bool INV, typename T> struct Dft<4, INV, T> {
  __device__ __forceinline__ static void run(T* v) {
    T a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    T a2 = cadd(v[1], v[3]), a3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
  }
};

// w8^j for j = 1, 3 (w8 = e^{-+ i pi/4}); j = 2 is -+i
template <bool INV, typename T> __device__ __forceinline__ T w8_1(T a) {
  typedef decltype(T().x) R;
  const R r = (R)0.70710678118654752440;
  T o;
  if (!INV) { o.x = r * (a.x + a.y); o.y = r * (a.y - a.x); }   // a (1 - i)/sqrt2
  else      { o.x = r * (a.x - a.y); o.y = r * (a.y + a.x); }   // a (1 + i)/sqrt2
  return o;
}
template <bool INV, typename T> __device__ __forceinline__ T w8_3(T a) {
  typedef decltype(T().x) R;
  const R r = (R)0.70710678118654752440;
  T o;
  if (!INV) { o.x = r * (a.y - a.x); o.y = -r * (a.x + a.y); }  // a (-1 - i)/sqrt2
  else      { o.x = -r * (a.x + a.y); o.y = r * (a.x - a.y); }  // a (-1 + i)/sqrt2
  return o;
}

template <bool INV, typename T> struct Dft<8, INV, T> {
  __device__ __forceinline__ static void run(T* v) {
    T e[4] = {v[0], v[2], v[4], v[6]};
    T o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV, T>::run(e);
    Dft<4, INV, T>::run(o);
    o[1] = w8_1<INV>(o[1]);
    o[2] = mul_mi<INV>(o[2]);
    o[3] = w8_3<INV>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

template <bool INV, typename T> struct Dft<16, INV, T> {
  __device__ __forceinline__ static void run(T* v) {
    typedef decltype(T().x) R;
    // 16 = 4 x 4: Y_p = DFT4(x[p], x[p+4], x[p+8], x[p+12]); X[k1 + 4 k2] = sum_p w16^{p k1} Y_p[k1] w4^{p k2}
    T y[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      y[p][0] = v[p]; y[p][1] = v[p + 4]; y[p][2] = v[p + 8]; y[p][3] = v[p + 12];
      Dft<4, INV, T>::run(y[p]);
    }
    const R c1 = (R)0.92387953251128675613;  // cos(pi/8)
    const R s1 = (R)0.38268343236508977173;  // sin(pi/8)
    const R r2 = (R)0.70710678118654752440;
    const R sg = INV ? (R)1 : (R)-1;         // twiddle e^{sg i 2 pi j/16}
    // w16^j = cos(2 pi j/16) + sg i sin(2 pi j/16)
    const R cw[10] = {(R)1, c1, r2, s1, (R)0, -s1, -r2, -c1, (R)-1, -c1};
    const R sw[10] = {(R)0, s1, r2, c1, (R)1, c1, r2, s1, (R)0, -s1};
#pragma unroll
    for (int p = 1; p < 4; ++p) {
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) {
        const int j = p * k1;
        T w; w.x = cw[j]; w.y = sg * sw[j];
        y[p][k1] = cmul(y[p][k1], w);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      T z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4, INV, T>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
    }
  }
};

// ---------------------------------------------------------------- FFT plan
struct FftPlan {
  int n;
  int nst;
  int radix[12];
};

// Lines live in shared memory: element e of line l at buf[l * ls + e * es].
// line_fast: consecutive threads take consecutive lines (use when es > 1 and lines are adjacent
// in memory); otherwise consecutive threads take consecutive butterflies of one line (es == 1).
struct LineLayout {
  int lines, es, ls;
  bool line_fast;
};

// One Stockham stage with radix RADIX, out of place (src -> dst): butterfly j of a line reads
// elements j + r n/RADIX, multiplies element r by w_n^{r k n/(Ns RADIX)} (k = j mod Ns), transforms,
// and writes element r to (j / Ns) Ns RADIX + k + r Ns.
template <int RADIX, bool INV, typename T>
__device__ __forceinline__ void fft_stage(const T* __restrict__ src, T* __restrict__ dst, const T* __restrict__ tw,
                                          int n, int Ns, LineLayout L) {
  const int nb = n / RADIX;
  const int total = L.lines * nb;
  const int tstride = n / (Ns * RADIX);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, j;
    if (L.line_fast) { l = t % L.lines; j = t / L.lines; }
    else { j = t % nb; l = t / nb; }
    const T* sb = src + l * L.ls;
    T v[RADIX];
#pragma unroll
    for (int r = 0; r < RADIX; ++r) v[r] = sb[(j + r * nb) * L.es];
    const int k = j % Ns;
    if (k > 0) {
#pragma unroll
      for (int r = 1; r < RADIX; ++r) {
        T w = tw[r * k * tstride];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Dft<RADIX, INV, T>::run(v);
    T* db = dst + l * L.ls;
    const int o = (j / Ns) * Ns * RADIX + k;
#pragma unroll
    for (int r = 0; r < RADIX; ++r) db[(o + r * Ns) * L.es] = v[r];
  }
  __syncthreads();
}

// Full transform of all lines, ping-ponging between a and b (same layout).  The caller
// synchronises before the call; the result is in the returned buffer (a if the number of stages
// is even, else b) and the call returns synchronised.
template <bool INV, typename T>
__device__ __forceinline__ T* fft_lines(T* a, T* b, const T* tw, const FftPlan& P, LineLayout L) {
  int Ns = 1;
  T* src = a;
  T* dst = b;
#pragma unroll 1
  for (int s = 0; s < P.nst; ++s) {
    const int R = P.radix[s];
    switch (R) {
      case 2: fft_stage<2, INV>(src, dst, tw, P.n, Ns, L); break;
      case 3: fft_stage<3, INV>(src, dst, tw, P.n, Ns, L); break;
      case 4: fft_stage<4, INV>(src, dst, tw, P.n, Ns, L); break;
      case 8: fft_stage<8, INV>(src, dst, tw, P.n, Ns, L); break;
      default: fft_stage<16, INV>(src, dst, tw, P.n, Ns, L); break;
    }
    Ns *= R;
    T* t = src; src = dst; dst = t;
  }
  return src;
}

}  // namespace gfp
