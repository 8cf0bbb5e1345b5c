// Shared device types for the Liouville-Lanczos kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ll {

template <typename T> struct cplx { T x, y; };

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename T> __host__ __device__ __forceinline__ cplx<T> cjmul(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> czero() { return mk(T(0), T(0)); }

// Offsets of the twiddle table of each supported grid side N in the per-precision table of
// W_N^e = exp(-2 pi i e / N), e = 0..N-1, laid out back to back.
template <int N> struct TwOff;
template <> struct TwOff<12> { static constexpr int v = 0; };
template <> struct TwOff<16> { static constexpr int v = 12; };
template <> struct TwOff<18> { static constexpr int v = 28; };
template <> struct TwOff<24> { static constexpr int v = 46; };
template <> struct TwOff<32> { static constexpr int v = 70; };
template <> struct TwOff<36> { static constexpr int v = 102; };
template <> struct TwOff<48> { static constexpr int v = 138; };
constexpr int kTwTotal = 186;
constexpr int kGridSides[] = {12, 16, 18, 24, 32, 36, 48};

// Division by a divisor fixed at launch, as a multiply-high and a shift (Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI 1994, Sec. 4):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(m, n) + n) >> l
// for every 0 <= n < 2^31 (the sum then cannot overflow 32 bits).
struct FastDiv {
  unsigned d, m, l;
  FastDiv() : d(1), m(1), l(0) {}
  explicit FastDiv(unsigned dv) : d(dv ? dv : 1), m(1), l(0) {  // d = 0 is taken as 1
    while ((1ull << l) < d) ++l;
    m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  }
  __device__ __forceinline__ int div(int n) const { return (int)((__umulhi((unsigned)n, m) + (unsigned)n) >> l); }
  __device__ __forceinline__ int mod(int n) const { return n - div(n) * (int)d; }
};

// Device status word: the kernels never trap; a detected fault sets a code here and the
// host turns it into an ll_status after the call.
enum DevErr : int { DEV_OK = 0, DEV_NOTPD = 1, DEV_BREAKDOWN = 2, DEV_BOUNDS = 3, DEV_TIMEOUT = 4 };

// Bounds-checked build (-DLL_CHECK, libll_check.so): every index the kernels take from a
// sphere or map table is tested before its access; a failing test records the source line
// in g_oob_line (the first one wins), the access is skipped, and the host reports
// LL_EINVAL after the call.  The plain build compiles the tests away.
#ifdef LL_CHECK
static __device__ int g_oob_line;
__device__ __forceinline__ bool ll_inb(bool ok, int line) {
  if (!ok) atomicCAS(&g_oob_line, 0, line);
  return ok;
}
#define LL_INB(cond) ::ll::ll_inb((cond), __LINE__)
#else
#define LL_INB(cond) true
#endif

}  // namespace ll
