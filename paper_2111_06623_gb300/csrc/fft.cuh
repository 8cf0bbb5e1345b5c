// Register-resident 1D FFTs of the grid sides the plane-wave grids use (N = 2^a 3^b <= 48).
//
// One thread transforms one whole line held in registers: a mixed-radix Stockham
// recursion (radices 2, 3, 4) fully unrolled at compile time, so every array index and
// every twiddle index is a constant.  Twiddles come from a per-translation-unit
// __constant__ table (uniform, constant-offset loads); trivial twiddles are skipped at
// compile time.  SIGN = -1: forward, sum_j f_j e^{-2 pi i m j/N};  SIGN = +1: inverse
// without the 1/N.
#pragma once
#include <math.h>

#include "common.cuh"

namespace ll {

// Each translation unit that includes this header owns its copy of the tables and fills
// them with tw_tables_upload() on every device it uses.
static __constant__ double2 c_tw64[kTwTotal];
static __constant__ float2 c_tw32[kTwTotal];

template <typename T> struct TwTab;
template <> struct TwTab<double> {
  static __device__ __forceinline__ cplx<double> get(int i) { double2 w = c_tw64[i]; return mk(w.x, w.y); }
};
template <> struct TwTab<float> {
  static __device__ __forceinline__ cplx<float> get(int i) { float2 w = c_tw32[i]; return mk(w.x, w.y); }
};

// exp(-2 pi i e / N) from the host libm in double (and rounded to float), for every side.
static inline cudaError_t tw_tables_upload(cudaStream_t stream) {
  double2 h64[kTwTotal];
  float2 h32[kTwTotal];
  int off = 0;
  for (int n : kGridSides) {
    for (int e = 0; e < n; ++e) {
      const double ang = -2.0 * 3.14159265358979323846264338327950288 * (double)e / (double)n;
      double c = cos(ang), s = sin(ang);
      if (4 * e == n) { c = 0.0; s = -1.0; }        // exact quarter and half turns
      if (2 * e == n) { c = -1.0; s = 0.0; }
      if (4 * e == 3 * n) { c = 0.0; s = 1.0; }
      h64[off + e] = make_double2(c, s);
      h32[off + e] = make_float2((float)c, (float)s);
    }
    off += n;
  }
  cudaError_t err = cudaMemcpyToSymbolAsync(c_tw64, h64, sizeof(h64), 0, cudaMemcpyHostToDevice, stream);
  if (err != cudaSuccess) return err;
  err = cudaMemcpyToSymbolAsync(c_tw32, h32, sizeof(h32), 0, cudaMemcpyHostToDevice, stream);
  if (err != cudaSuccess) return err;
  return cudaStreamSynchronize(stream);
}

template <typename T, int N, int SIGN>
__device__ __forceinline__ cplx<T> twiddle(int e) {
  cplx<T> w = TwTab<T>::get(TwOff<N>::v + e);
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// R-point DFT in place with exponent sign SIGN.
template <typename T, int R, int SIGN> struct Dft;

template <typename T, int SIGN> struct Dft<T, 2, SIGN> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    cplx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename T, int SIGN> struct Dft<T, 3, SIGN> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    // W_3 = -1/2 + SIGN i sqrt(3)/2
    const T c = T(-0.5);
    const T s = T(SIGN) * T(0.86602540378443864676372317075294);
    cplx<T> a = v[0], b = v[1], d = v[2];
    cplx<T> sum = b + d, dif = b - d;
    v[0] = a + sum;
    cplx<T> m = mk(a.x + c * sum.x, a.y + c * sum.y);
    // i s dif = (-s dif.y, s dif.x)
    v[1] = mk(m.x - s * dif.y, m.y + s * dif.x);
    v[2] = mk(m.x + s * dif.y, m.y - s * dif.x);
  }
};

template <typename T, int SIGN> struct Dft<T, 4, SIGN> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    cplx<T> a0 = v[0] + v[2], a1 = v[0] - v[2];
    cplx<T> b0 = v[1] + v[3], b1 = v[1] - v[3];
    // SIGN i b1
    cplx<T> jb1 = (SIGN > 0) ? mk(-b1.y, b1.x) : mk(b1.y, -b1.x);
    v[0] = a0 + b0;
    v[2] = a0 - b0;
    v[1] = a1 + jb1;
    v[3] = a1 - jb1;
  }
};

// One Stockham pass of radix R after Ns points have been combined.
template <typename T, int N, int R, int Ns, int SIGN>
__device__ __forceinline__ void stockham_pass(const cplx<T>* in, cplx<T>* out) {
#pragma unroll
  for (int j = 0; j < N / R; ++j) {
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = in[j + r * (N / R)];
      const int e = ((j % Ns) * r * (N / (Ns * R))) % N;
      if (e != 0) v[r] = cmul(v[r], twiddle<T, N, SIGN>(e));
    }
    Dft<T, R, SIGN>::run(v);
    const int d = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
    for (int r = 0; r < R; ++r) out[d + r * Ns] = v[r];
  }
}

template <int N> struct Plan;  // radices, first to last
template <> struct Plan<12> { static constexpr int n = 2; static constexpr int r[3] = {4, 3, 1}; };
template <> struct Plan<16> { static constexpr int n = 2; static constexpr int r[3] = {4, 4, 1}; };
template <> struct Plan<18> { static constexpr int n = 3; static constexpr int r[3] = {3, 3, 2}; };
template <> struct Plan<24> { static constexpr int n = 3; static constexpr int r[3] = {4, 3, 2}; };
template <> struct Plan<32> { static constexpr int n = 3; static constexpr int r[3] = {4, 4, 2}; };
template <> struct Plan<36> { static constexpr int n = 3; static constexpr int r[3] = {4, 3, 3}; };
template <> struct Plan<48> { static constexpr int n = 3; static constexpr int r[3] = {4, 4, 3}; };

// In-place FFT of a register line a[0..N-1] (result in a).
template <typename T, int N, int SIGN>
__device__ __forceinline__ void fft_line(cplx<T> (&a)[N]) {
  constexpr int R0 = Plan<N>::r[0], R1 = Plan<N>::r[1], R2 = Plan<N>::r[2];
  cplx<T> b[N];
  stockham_pass<T, N, R0, 1, SIGN>(a, b);
  if constexpr (Plan<N>::n == 2) {
    stockham_pass<T, N, R1, R0, SIGN>(b, a);
  } else {
    stockham_pass<T, N, R1, R0, SIGN>(b, a);
    stockham_pass<T, N, R2, R0 * R1, SIGN>(a, b);
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = b[i];
  }
}

// Input pruning.  A point p of a line whose sphere keeps only |m| <= PR (p <= PR or p >= N - PR)
// is zero on input; the first pass knows these zeros at compile time (a value with a constant
// flag) and skips every add whose operand is such a zero.  The arithmetic on the other values
// is the dense pass's, operation for operation, so the result equals fft_line's (up to the
// sign of exact zeros).
template <typename T>
struct ZC {
  cplx<T> v;
  bool z;   // known zero (compile time once inlined)
};
template <typename T>
__device__ __forceinline__ ZC<T> zadd(ZC<T> a, ZC<T> b) {
  if (a.z) return b;
  if (b.z) return a;
  return {a.v + b.v, false};
}
template <typename T>
__device__ __forceinline__ ZC<T> zsub(ZC<T> a, ZC<T> b) {
  if (b.z) return a;
  if (a.z) return {mk(-b.v.x, -b.v.y), false};
  return {a.v - b.v, false};
}

template <typename T, int R, int SIGN> struct ZDft;
template <typename T, int SIGN> struct ZDft<T, 2, SIGN> {
  static __device__ __forceinline__ void run(ZC<T>* v) {
    const ZC<T> a = v[0], b = v[1];
    v[0] = zadd(a, b);
    v[1] = zsub(a, b);
  }
};
template <typename T, int SIGN> struct ZDft<T, 4, SIGN> {
  static __device__ __forceinline__ void run(ZC<T>* v) {
    const ZC<T> a0 = zadd(v[0], v[2]), a1 = zsub(v[0], v[2]);
    const ZC<T> b0 = zadd(v[1], v[3]), b1 = zsub(v[1], v[3]);
    const ZC<T> jb1 = {(SIGN > 0) ? mk(-b1.v.y, b1.v.x) : mk(b1.v.y, -b1.v.x), b1.z};
    v[0] = zadd(a0, b0);
    v[2] = zsub(a0, b0);
    v[1] = zadd(a1, jb1);
    v[3] = zsub(a1, jb1);
  }
};
template <typename T, int SIGN> struct ZDft<T, 3, SIGN> {   // all zero, or the dense DFT
  static __device__ __forceinline__ void run(ZC<T>* v) {
    if (v[0].z && v[1].z && v[2].z) return;
    cplx<T> d[3] = {v[0].z ? czero<T>() : v[0].v, v[1].z ? czero<T>() : v[1].v, v[2].z ? czero<T>() : v[2].v};
    Dft<T, 3, SIGN>::run(d);
    for (int r = 0; r < 3; ++r) v[r] = {d[r], false};
  }
};

// fft_line<T, N, SIGN> of a line that is zero outside |m| <= PR (PR = 0: fft_line itself).
template <typename T, int N, int SIGN, int PR>
__device__ __forceinline__ void fft_line_in(cplx<T> (&a)[N]) {
  if constexpr (PR == 0) {
    fft_line<T, N, SIGN>(a);
  } else {
    constexpr int R0 = Plan<N>::r[0], R1 = Plan<N>::r[1], R2 = Plan<N>::r[2];
    cplx<T> b[N];
#pragma unroll
    for (int j = 0; j < N / R0; ++j) {   // first Stockham pass (Ns = 1: no twiddles)
      ZC<T> v[R0];
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int i = j + r * (N / R0);
        const bool kept = i <= PR || i >= N - PR;
        v[r] = {kept ? a[i] : czero<T>(), !kept};
      }
      ZDft<T, R0, SIGN>::run(v);
#pragma unroll
      for (int r = 0; r < R0; ++r) b[j * R0 + r] = v[r].z ? czero<T>() : v[r].v;
    }
    if constexpr (Plan<N>::n == 2) {
      stockham_pass<T, N, R1, R0, SIGN>(b, a);
    } else {
      stockham_pass<T, N, R1, R0, SIGN>(b, a);
      stockham_pass<T, N, R2, R0 * R1, SIGN>(a, b);
#pragma unroll
      for (int i = 0; i < N; ++i) a[i] = b[i];
    }
  }
}

// A 2H-point FFT split over a lane pair (lanes l and l ^ 1 of a warp, h = l & 1), each lane
// holding H points, with one radix-2 step exchanged through warp shuffles (mask: the pair).
//   fft_pair_dit: in  a[m] = x[2m + h]    out a[k] = X[H h + k]   (decimation in time)
//   fft_pair_dif: in  a[j] = x[H h + j]   out a[m] = X[2m + h]    (decimation in frequency)
// The transform is fft_line<T, 2H, SIGN>'s, with half the registers per lane.
template <typename T>
__device__ __forceinline__ cplx<T> shfl_pair(cplx<T> v, unsigned mask) {
  return mk(__shfl_xor_sync(mask, v.x, 1), __shfl_xor_sync(mask, v.y, 1));
}

template <typename T, int H, int SIGN>
__device__ __forceinline__ void fft_pair_dit(cplx<T> (&a)[H], int h, unsigned mask) {
  fft_line<T, H, SIGN>(a);               // Y_h[k] = sum_m x[2m + h] W_H^(mk)
  if (h) {
#pragma unroll
    for (int k = 1; k < H; ++k) a[k] = cmul(a[k], twiddle<T, 2 * H, SIGN>(k));   // W_2H^k Y_1[k]
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const cplx<T> o = shfl_pair(a[k], mask);
    a[k] = h ? o - a[k] : a[k] + o;        // X[k] = Y0 + W Y1,  X[k + H] = Y0 - W Y1
  }
}

template <typename T, int H, int SIGN>
__device__ __forceinline__ void fft_pair_dif(cplx<T> (&a)[H], int h, unsigned mask) {
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const cplx<T> o = shfl_pair(a[j], mask);
    if (h) {
      a[j] = o - a[j];                     // x[j] - x[j + H]
      if (j) a[j] = cmul(a[j], twiddle<T, 2 * H, SIGN>(j));
    } else {
      a[j] = a[j] + o;                     // x[j] + x[j + H]
    }
  }
  fft_line<T, H, SIGN>(a);               // even (h = 0) or odd (h = 1) outputs
}

}  // namespace ll
