// Kernels of one Liouvillian application and of the two Lanczos recursions (sm_103a).
//
// Layouts (all complex interleaved, C order):
//   batch vector      x[vec][k][v][npw_pad]          one orbital per (vec, k, v) on sphere(k+Q)
//   column buffer     cbuf[o][j3][ncol_max]          per orbital o: the sphere's (m1, m2)
//                                                    columns after the 1D FFT along axis 3
//   real-space grids  g[j3][j2][j1]                  (j1 fastest)
//   orbital grids     ur[k][v][j3][j2][j1]           u_{vk}(r) sqrt(Omega), sphere(k)
// A 3D transform of a sphere is split as: 1D FFTs of the occupied columns (axis 3), then for
// every plane j3 a 2D transform over (axis 2, axis 1) restricted to the sphere's rows and
// columns; the full N^3 grid of one orbital is never materialised.
#pragma once
#include "fft.cuh"

namespace ll {

// Plane-wave sphere tables of one family (spheres of k, or of k+Q) on the device.
struct SphereDev {
  int nks, npw_pad, ncol_max, nrow_max;
  const int* npw;       // [nks]
  const int* ncol;      // [nks]
  const int* nrow;      // [nks]
  const int4* col;      // [nks][ncol_max]  (m1, m2, m3 of the first point, point count),
                        //                  ordered by (m2, m1)
  const int* colstart;  // [nks][ncol_max]  first point of the column in the sphere order
  const int4* row;      // [nks][nrow_max]  (m2, first column, m1 of the first column, columns),
                        //                  consecutive m2, each row's m1 consecutive
};

// m mod N for m >= -N (a mask when N is a power of two)
template <int N>
__device__ __forceinline__ int wrapn(int m) { return (int)((unsigned)(m + N) % (unsigned)N); }

// ---------------------------------------------------------------------------------------
// Sphere -> columns: scatter each column's points and inverse-FFT along axis 3.
// grid (nks, nvec, split), block 128; item = (v, column), the k block's items spread over
// the split CTAs.
template <typename T, int N>
__global__ void __launch_bounds__(128) k_zinv(SphereDev s, const cplx<T>* __restrict__ x, int nbnd,
                                              cplx<T>* __restrict__ cbuf, int cb_ncol) {
  const int k = blockIdx.x, vec = blockIdx.y;
  const int nc = s.ncol[k];
  for (int it = blockIdx.z * blockDim.x + threadIdx.x; it < nbnd * nc; it += blockDim.x * gridDim.z) {
    const int v = it / nc, c = it - v * nc;
    const long o = ((long)vec * s.nks + k) * nbnd + v;
    const int4 cl = s.col[k * s.ncol_max + c];
    const int st = s.colstart[k * s.ncol_max + c];
    const cplx<T>* src = x + o * s.npw_pad + st;
    cplx<T> a[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
      const int i = wrapn<N>(p - cl.z);
      a[p] = (i < cl.w && LL_INB(st >= 0 && st + i < s.npw_pad)) ? src[i] : czero<T>();
    }
    fft_line<T, N, +1>(a);
    if (!LL_INB(c < cb_ncol)) continue;
    cplx<T>* dst = cbuf + o * (long)N * cb_ncol + c;
#pragma unroll
    for (int p = 0; p < N; ++p) dst[(long)p * cb_ncol] = a[p];
  }
}

// ---------------------------------------------------------------------------------------
// Bulk prefetch of a contiguous global range into L2 (no data returned to the SM): address
// 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------------------
// Per-plane pass of one operator application.  grid (N planes, groups), block 128.
// The sphere's columns are ordered by (m2, m1) and grouped in rows of equal m2 (consecutive
// m1).  For every orbital of the group (BO at a time), at plane j3 = blockIdx.x:
//   rows     1D FFT along axis 1 (m1 <-> j1) of every sphere row, between the column buffer
//            Cs and the row buffer Ys[row][j1];
//   lines    one thread per (orbital, j1): 1D FFT along axis 2 (m2 <-> j2) of the line
//            x(j2, j1), j2 = 0..N-1, held in registers.  Thread t = s N + j1 (s < S = 128/N)
//            always takes column j1, for the batch's orbitals b = s, s + S, ...; consecutive
//            threads take consecutive j1, so every real-space plane (V, v', u, the density)
//            is read and written with unit stride across a warp straight from HBM.
// Modes:
//   XY_PASS1       inverse 2D FFT of the plane's columns, t(r) = V(r) x(r), forward 2D FFT
//                  back to the columns (in place);
//   XY_PASS1_DENS  the same plus the response-density partial sum_o conj(u_o(r)) x_o(r) of the
//                  orbitals of vector dens_vec, written per (group, plane) to nprt.  Each
//                  thread adds its lines' products into its own column of its slot's plane
//                  Pb[s] (no other thread touches it: no barrier, a fixed order); the S slots
//                  are summed in order once, at the end;
//   XY_PASS2       t(r) = v'(r) u(r) from the orbital grid, forward 2D FFT, added into the
//                  columns (linearity: one axis-3 transform serves both passes);
//   XY_STORE       inverse 2D FFT only, x(r) stored to grid_out (orbital grids at set-up).
enum XYMode { XY_PASS1 = 0, XY_PASS1_DENS = 1, XY_PASS2 = 2, XY_STORE = 3 };

struct XYArgs {
  SphereDev s;
  int nbnd, norb;              // orbitals handled by this launch
  int cb_ncol;
  int per_group;               // orbitals per group
  int o_off;                   // first orbital of this launch (orbital o = o_off + local index)
  int dens_vec;                // vector whose orbitals feed the density (XY_PASS1_DENS)
  int bo;                      // orbitals per batch (as many as shared memory allows, <= the mode's default)
  FastDiv f_ncol, f_nrow;      // divisions by cb_ncol and by the sphere table's nrow_max
  FastDiv f_nbnd, f_nks;       // orbital -> k: (o / nbnd) mod nks
  FastDiv f_pervec;            // orbital -> vector: o / (nks nbnd)
};

// The pruning bounds built besides N/4: 3N/16 at N = 32 (the spheres of a 25 Ry cutoff on the
// two-atom cell reach |m| = 6), none elsewhere.
__host__ __device__ constexpr int tight_prune(int n) { return n == 32 ? 3 * n / 16 : 0; }

// Output pruning of the forward line transforms: with PR > 0 every sphere of the system has
// |m| <= PR on all three axes, so only the points p <= PR and p >= N - PR of a forward line
// are kept; with the stores of the other points gone at compile time, the compiler drops
// the butterflies that only feed them.  PR = 0: every point.
template <int N, int PR>
__device__ __forceinline__ constexpr bool line_kept(int p) {
  return PR == 0 || p <= PR || p >= N - PR;
}

template <typename T, int N, int MODE, int PR = 0>
__global__ void __launch_bounds__(128, N > 36 ? 2 : (MODE == XY_PASS1_DENS ? 3 : 4)) k_xy(XYArgs a, cplx<T>* __restrict__ cbuf, const T* __restrict__ vloc,
                                               const cplx<T>* __restrict__ vpr, const cplx<T>* __restrict__ ur,
                                               cplx<T>* __restrict__ nprt, cplx<T>* __restrict__ grid_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NP = N + 1;
  constexpr int NN = N * N;
  const int iz = blockIdx.x, g = blockIdx.y;
  const int BO = a.bo;
  const SphereDev& s = a.s;
  cplx<T>* Cs = reinterpret_cast<cplx<T>*>(smem_raw);                 // [BO][cb_ncol]
  cplx<T>* Ys = Cs + BO * a.cb_ncol;                                    // [BO][nrow_max][NP]
  constexpr int S = 128 / N;                                           // line slots
  cplx<T>* Pl = Ys + BO * s.nrow_max * NP;                              // [N][N] v' (pass 2)
  cplx<T>* Pb = Pl + (MODE == XY_PASS2 ? NN : 0);                       // [S][N][N] density
  T* Pv = reinterpret_cast<T*>(Pb + (MODE == XY_PASS1_DENS ? S * NN : 0));  // [N][N] V (real)
  const long plane = (long)NN;
  const int ls = threadIdx.x / N, lj1 = threadIdx.x - ls * N;           // line slot, column

  if (MODE == XY_PASS1 || MODE == XY_PASS1_DENS) {
    for (int i = threadIdx.x; i < NN; i += blockDim.x) Pv[i] = vloc[iz * plane + i];
  } else if (MODE == XY_PASS2) {
    for (int i = threadIdx.x; i < NN; i += blockDim.x) Pl[i] = vpr[iz * plane + i];
  }
  if (MODE == XY_PASS1_DENS)
    for (int i = threadIdx.x; i < S * NN; i += blockDim.x) Pb[i] = czero<T>();

  const int o_begin = a.o_off + g * a.per_group;
  const int o_end = a.o_off + min(a.norb, g * a.per_group + a.per_group);
  // The next batch's column-buffer rows of this plane (cb_ncol is even: 16-byte multiples)
  // are prefetched into L2 while this batch is transformed; the density pass also prefetches
  // the current batch's orbital-grid planes before its row transforms, which then hide the
  // HBM latency.  (Prefetching the next batch's grid planes a whole batch ahead was
  // measured: their lines were evicted before use and re-read, +20 % DRAM.)
  auto prefetch_batch = [&](int obatch) {
    const int t = threadIdx.x;
    if (t < BO && obatch + t < o_end)
      prefetch_l2(cbuf + (long)(obatch + t) * N * a.cb_ncol + (long)iz * a.cb_ncol,
                  (unsigned)(a.cb_ncol * sizeof(cplx<T>)));
  };
  prefetch_batch(o_begin);
  for (int ob = o_begin; ob < o_end; ob += BO) {
    const int nb = min(BO, o_end - ob);
    __syncthreads();
    if (ob + BO < o_end) prefetch_batch(ob + BO);
    if (MODE == XY_PASS1_DENS && threadIdx.x < nb) {
      const int o = ob + threadIdx.x;
      if (a.f_pervec.div(o) == a.dens_vec)
        prefetch_l2(ur + (long)a.f_pervec.mod(o) * N * plane + iz * plane, (unsigned)(NN * sizeof(cplx<T>)));
    }
    if (MODE != XY_PASS2) {
      for (int i = threadIdx.x; i < nb * a.cb_ncol; i += blockDim.x) {
        const int b = a.f_ncol.div(i), c = i - b * a.cb_ncol;
        const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
        Cs[i] = (c < s.ncol[k]) ? cbuf[(long)o * N * a.cb_ncol + (long)iz * a.cb_ncol + c] : czero<T>();
      }
      __syncthreads();
      // inverse FFT along axis 1 of every sphere row (fixed m2)
      for (int i = threadIdx.x; i < nb * s.nrow_max; i += blockDim.x) {
        const int b = a.f_nrow.div(i), r = i - b * s.nrow_max;
        const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
        if (r >= s.nrow[k]) continue;
        const int4 rw = s.row[k * s.nrow_max + r];
        cplx<T> l[N];
        const cplx<T>* cs = Cs + b * a.cb_ncol + rw.y;
#pragma unroll
        for (int p = 0; p < N; ++p) {
          const int j = wrapn<N>(p - rw.z);
          l[p] = (j < rw.w && LL_INB(rw.y >= 0 && rw.y + j < a.cb_ncol)) ? cs[j] : czero<T>();
        }
        fft_line_in<T, N, +1, (MODE == XY_STORE ? 0 : PR)>(l);
        cplx<T>* ys = Ys + (b * s.nrow_max + r) * NP;
#pragma unroll
        for (int p = 0; p < N; ++p) ys[p] = l[p];
      }
      __syncthreads();
    }
    // axis 2: one line per (orbital, j1), element p of the line at grid point (j2 = p, j1)
#pragma unroll 1
    for (int b = ls; ls < S && b < nb; b += S) {
      const int j1 = lj1;
      const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
      const int nr = s.nrow[k];
      const int m2min = s.row[k * s.nrow_max].x;
      cplx<T> l[N];
      if (MODE == XY_PASS2) {
        const cplx<T>* u = ur + (long)a.f_pervec.mod(o) * N * plane + iz * plane + j1;
#pragma unroll
        for (int p = 0; p < N; ++p) l[p] = cmul(Pl[p * N + j1], u[p * N]);
      } else {
#pragma unroll
        for (int p = 0; p < N; ++p) {
          const int r = wrapn<N>(p - m2min);
          l[p] = (r < nr && LL_INB(r < s.nrow_max)) ? Ys[(b * s.nrow_max + r) * NP + j1] : czero<T>();
        }
        fft_line_in<T, N, +1, (MODE == XY_STORE ? 0 : PR)>(l);
        if (MODE == XY_STORE) {
          cplx<T>* dst = grid_out + (long)o * N * plane + iz * plane + j1;
#pragma unroll
          for (int p = 0; p < N; ++p) dst[p * N] = l[p];
          continue;
        }
        if (MODE == XY_PASS1_DENS && a.f_pervec.div(o) == a.dens_vec) {
          // conj(u) x of this line into this thread's own column of its slot
          const cplx<T>* u = ur + (long)a.f_pervec.mod(o) * N * plane + iz * plane + j1;
          cplx<T>* pb = Pb + ls * NN + j1;
#pragma unroll
          for (int p = 0; p < N; ++p) pb[p * N] = pb[p * N] + cjmul(u[p * N], l[p]);
        }
#pragma unroll
        for (int p = 0; p < N; ++p) l[p] = l[p] * Pv[p * N + j1];
      }
      fft_line<T, N, -1>(l);
#pragma unroll
      for (int p = 0; p < N; ++p) {
        const int r = wrapn<N>(p - m2min);
        if (line_kept<N, PR>(p) && r < nr && LL_INB(r < s.nrow_max)) Ys[(b * s.nrow_max + r) * NP + j1] = l[p];
      }
    }
    __syncthreads();
    if (MODE == XY_STORE) continue;
    // forward FFT along axis 1 of every row, keep the row's columns
    for (int i = threadIdx.x; i < nb * s.nrow_max; i += blockDim.x) {
      const int b = a.f_nrow.div(i), r = i - b * s.nrow_max;
      const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
      if (r >= s.nrow[k]) continue;
      const int4 rw = s.row[k * s.nrow_max + r];
      cplx<T> l[N];
      const cplx<T>* ys = Ys + (b * s.nrow_max + r) * NP;
#pragma unroll
      for (int p = 0; p < N; ++p) l[p] = ys[p];
      fft_line<T, N, -1>(l);
      cplx<T>* cs = Cs + b * a.cb_ncol + rw.y;
#pragma unroll
      for (int p = 0; p < N; ++p) {
        const int j = wrapn<N>(p - rw.z);
        if (line_kept<N, PR>(p) && j < rw.w && LL_INB(rw.y >= 0 && rw.y + j < a.cb_ncol)) cs[j] = l[p];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb * a.cb_ncol; i += blockDim.x) {
      const int b = a.f_ncol.div(i), c = i - b * a.cb_ncol;
      const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
      if (c >= s.ncol[k]) continue;
      cplx<T>* dst = cbuf + (long)o * N * a.cb_ncol + (long)iz * a.cb_ncol + c;
      *dst = (MODE == XY_PASS2) ? *dst + Cs[i] : Cs[i];
    }
  }
  if (MODE == XY_PASS1_DENS) {  // the slots summed in order
    __syncthreads();
    for (int i = threadIdx.x; i < NN; i += blockDim.x) {
      cplx<T> acc = Pb[i];
      for (int q = 1; q < S; ++q) acc = acc + Pb[q * NN + i];
      nprt[(long)g * N * plane + iz * plane + i] = acc;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Response potential of one density (Eqs. 12-13): n'(r) from the group partials, 3D FFT,
// Hartree 4 pi/|Q+G|^2, inverse FFT, plus f_xc(n0) n'.  Three launches over the grid.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_hxc_fwd(const cplx<T>* __restrict__ nprt, int ngroups, T scale,
                                                cplx<T>* __restrict__ nr, cplx<T>* __restrict__ ng) {
  __shared__ cplx<T> P[N][N + 1];
  const int iz = blockIdx.x;
  const long plane = (long)N * N;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    cplx<T> acc = czero<T>();
    for (int gi = 0; gi < ngroups; ++gi) acc = acc + nprt[(long)gi * N * plane + iz * plane + i];
    acc = acc * scale;
    nr[iz * plane + i] = acc;
    P[i / N][i % N] = acc;
  }
  __syncthreads();
  if (threadIdx.x < N) {  // axis 1, row j2
    const int j2 = threadIdx.x;
    cplx<T> l[N];
#pragma unroll
    for (int p = 0; p < N; ++p) l[p] = P[j2][p];
    fft_line<T, N, -1>(l);
#pragma unroll
    for (int p = 0; p < N; ++p) P[j2][p] = l[p];
  }
  __syncthreads();
  if (threadIdx.x < N) {  // axis 2, column m1
    const int m1 = threadIdx.x;
    cplx<T> l[N];
#pragma unroll
    for (int p = 0; p < N; ++p) l[p] = P[p][m1];
    fft_line<T, N, -1>(l);
#pragma unroll
    for (int p = 0; p < N; ++p) ng[iz * plane + p * N + m1] = l[p];
  }
}

// The response density averaged over the small group of Q (Sec. 2.6): out(r_j) = (1/nsym)
// sum_S scale n~(r_{M_S j}), n~ = the sum of the density groups (the order of k_hxc_fwd),
// M_S the integer matrices sym[S] on the grid indices (j1, j2, j3), mod N.  Grid layout
// [j3][j2][j1]; grid-stride loop over the N^3 points.
template <typename T>
__global__ void k_dens_sym(const cplx<T>* __restrict__ nprt, int ngroups, int n, T scale, int nsym,
                           const int* __restrict__ sym, cplx<T>* __restrict__ out) {
  const long n3 = (long)n * n * n;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n3; p += (long)gridDim.x * blockDim.x) {
    const int j1 = (int)(p % n), j2 = (int)((p / n) % n), j3 = (int)(p / ((long)n * n));
    cplx<T> acc = czero<T>();
    for (int s = 0; s < nsym; ++s) {
      const int* m = sym + 9 * s;
      const int i1 = (((m[0] * j1 + m[1] * j2 + m[2] * j3) % n) + n) % n;
      const int i2 = (((m[3] * j1 + m[4] * j2 + m[5] * j3) % n) + n) % n;
      const int i3 = (((m[6] * j1 + m[7] * j2 + m[8] * j3) % n) + n) % n;
      const long q = ((long)i3 * n + i2) * n + i1;
      cplx<T> v = czero<T>();
      for (int g = 0; g < ngroups; ++g) v = v + nprt[(long)g * n3 + q];
      acc = acc + v * scale;
    }
    out[p] = acc * (T(1) / (T)nsym);
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(64) k_hxc_z(cplx<T>* __restrict__ ng, const T* __restrict__ whart) {
  const int line = blockIdx.x * blockDim.x + threadIdx.x;   // (m2, m1)
  if (line >= N * N) return;
  const long plane = (long)N * N;
  cplx<T> l[N];
#pragma unroll
  for (int p = 0; p < N; ++p) l[p] = ng[p * plane + line];
  fft_line<T, N, -1>(l);
#pragma unroll
  for (int p = 0; p < N; ++p) l[p] = l[p] * whart[p * plane + line];
  fft_line<T, N, +1>(l);
#pragma unroll
  for (int p = 0; p < N; ++p) ng[p * plane + line] = l[p];
}

template <typename T, int N>
__global__ void __launch_bounds__(64) k_hxc_inv(const cplx<T>* __restrict__ ng, const cplx<T>* __restrict__ nr,
                                                const T* __restrict__ fxc, cplx<T>* __restrict__ vpr) {
  __shared__ cplx<T> P[N][N + 1];
  const int iz = blockIdx.x;
  const long plane = (long)N * N;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) P[i / N][i % N] = ng[iz * plane + i];
  __syncthreads();
  if (threadIdx.x < N) {  // axis 2 inverse, column m1
    const int m1 = threadIdx.x;
    cplx<T> l[N];
#pragma unroll
    for (int p = 0; p < N; ++p) l[p] = P[p][m1];
    fft_line<T, N, +1>(l);
#pragma unroll
    for (int p = 0; p < N; ++p) P[p][m1] = l[p];
  }
  __syncthreads();
  if (threadIdx.x < N) {  // axis 1 inverse, row j2
    const int j2 = threadIdx.x;
    cplx<T> l[N];
#pragma unroll
    for (int p = 0; p < N; ++p) l[p] = P[j2][p];
    fft_line<T, N, +1>(l);
    const long base = iz * plane + (long)j2 * N;
#pragma unroll
    for (int p = 0; p < N; ++p) vpr[base + p] = l[p] + nr[base + p] * fxc[base + p];
  }
}

// ---------------------------------------------------------------------------------------
// Reductions.  Every sum below runs in a fixed order (per-thread strided partial sums, lanes,
// then warps), so results are bitwise reproducible.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// All-pairs dots out[i*nj + j] = mult[i] * sum_g conj(A[i*lda + g]) B[j*ldb + g] over g < npw,
// eight pairs at a time: per-thread partial sums in T, warp sums in T, warps summed in
// double.  `red`: 16 doubles per warp.  Called by the whole block; ends synchronised.
template <typename T>
__device__ void block_dots(const cplx<T>* A, long lda, const cplx<T>* B, long ldb, int npw, int ni, int nj,
                           const double* mult, cplx<double>* out, double* red) {
  const int np = ni * nj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = 0; c0 < np; c0 += 8) {
    T acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = T(0);
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int pr = c0 + q;
        if (pr < np) {
          const int i = pr / nj, j = pr - i * nj;
          const cplx<T> t = cjmul(A[i * lda + g], B[j * ldb + g]);
          acc[2 * q] += t.x;
          acc[2 * q + 1] += t.y;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const T v = warp_sum_t(acc[q]);
      if (lane == 0) red[warp * 16 + q] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 8 && c0 + (int)threadIdx.x < np) {
      const int pr = c0 + threadIdx.x;
      double re = 0.0, im = 0.0;
      for (int w = 0; w < nw; ++w) {
        re += red[w * 16 + 2 * threadIdx.x];
        im += red[w * 16 + 2 * threadIdx.x + 1];
      }
      const double m = mult ? mult[pr / nj] : 1.0;
      out[pr] = mk(re * m, im * m);
    }
    __syncthreads();
  }
}

// The same for compile-time NI x NJ (the common small shapes) in one pass: every thread keeps
// all NI*NJ complex partial sums in registers.  `red`: 2*NI*NJ doubles per warp.
template <typename T, int NI, int NJ>
__device__ void block_dots_fixed(const cplx<T>* A, long lda, const cplx<T>* B, long ldb, int npw,
                                 const double* mult, cplx<double>* out, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T acc[NI][NJ][2];
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j][0] = acc[i][j][1] = T(0);
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    cplx<T> a[NI], b[NJ];
#pragma unroll
    for (int i = 0; i < NI; ++i) a[i] = A[i * lda + g];
#pragma unroll
    for (int j = 0; j < NJ; ++j) b[j] = B[j * ldb + g];
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        acc[i][j][0] += a[i].x * b[j].x + a[i].y * b[j].y;
        acc[i][j][1] += a[i].x * b[j].y - a[i].y * b[j].x;
      }
  }
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T v = warp_sum_t(acc[i][j][c]);
        if (lane == 0) red[warp * (2 * NI * NJ) + (i * NJ + j) * 2 + c] = (double)v;
      }
  __syncthreads();
  if (threadIdx.x < NI * NJ) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nw; ++w) {
      re += red[w * (2 * NI * NJ) + 2 * threadIdx.x];
      im += red[w * (2 * NI * NJ) + 2 * threadIdx.x + 1];
    }
    const double m = mult ? mult[threadIdx.x / NJ] : 1.0;
    out[threadIdx.x] = mk(re * m, im * m);
  }
  __syncthreads();
}

// Fixed-shape dots when (ni, nj) is one of the compiled shapes, else the chunked form.
// `red` must hold max(16, 2*ni*nj) doubles per warp.
template <typename T>
__device__ __forceinline__ void small_dots(const cplx<T>* A, long lda, const cplx<T>* B, long ldb, int npw, int ni,
                                           int nj, const double* mult, cplx<double>* out, double* red) {
  if (ni == 4 && nj == 4) block_dots_fixed<T, 4, 4>(A, lda, B, ldb, npw, mult, out, red);
  else if (ni == 8 && nj == 4) block_dots_fixed<T, 8, 4>(A, lda, B, ldb, npw, mult, out, red);
  else if (ni == 2 && nj == 4) block_dots_fixed<T, 2, 4>(A, lda, B, ldb, npw, mult, out, red);
  else if (ni == 1 && nj == 1) block_dots_fixed<T, 1, 1>(A, lda, B, ldb, npw, mult, out, red);
  else block_dots<T>(A, lda, B, ldb, npw, ni, nj, mult, out, red);
}

// The P_c dot block S = U^H x (nbnd x nv): the 4 x 4 shape in registers, others chunked.
// (A separate dispatcher from small_dots keeps the 8 x 4 KB shape's registers out of the
// kernels that only project.)
template <typename T>
__device__ __forceinline__ void proj_dots(const cplx<T>* A, long lda, const cplx<T>* B, long ldb, int npw, int ni,
                                          int nj, cplx<double>* out, double* red) {
  if (ni == 4 && nj == 4) block_dots_fixed<T, 4, 4>(A, lda, B, ldb, npw, nullptr, out, red);
  else block_dots<T>(A, lda, B, ldb, npw, ni, nj, nullptr, out, red);
}

// x[v][g] -= sum_w U[w][g] S[w][v] for nv orbitals x of one k against its nbnd occupied
// states U (S = U^H x, nbnd x nv).  The coefficients are rounded to T once: conversions from
// double run on the slow FP64 pipe.
template <typename T>
__device__ __forceinline__ void subtract_projection(cplx<T>* x, const cplx<T>* uk, const cplx<double>* S, int nbnd,
                                                    int nv, int npw_pad) {
  __shared__ cplx<T> St[32 * 32];
  for (int i = threadIdx.x; i < nbnd * nv; i += blockDim.x) St[i] = mk((T)S[i].x, (T)S[i].y);
  __syncthreads();
  for (int i = threadIdx.x; i < nv * npw_pad; i += blockDim.x) {
    const int v = i / npw_pad, gi = i - v * npw_pad;
    cplx<T> t = x[i];
    for (int w = 0; w < nbnd; ++w) t = t - cmul(uk[(long)w * npw_pad + gi], St[w * nv + v]);
    x[i] = t;
  }
  __syncthreads();
}

// Metals (Sec. 2.6; smeared occupations f).  With c_mv = max(1 - f_m/f_v, 0) the weight of the
// projector on empty states P_{c,v} for the states m of k+Q and band v of k, the library
// iterates on z = Q^-1 (sqrt(f_v) x), Q = P_{c,v}^{1/2} (weight sqrt(c_mv) on the states of
// k+Q kept, 1 off them): there the operator D + Q W Q is symmetric (W: the Hartree-XC response
// of the density of Q z with the weights sqrt(f_v) folded into u_k), so the recursions need no
// metric, and the components along the kept states are not scaled down by sqrt(c) (in FP32 a
// scaled-down component would carry rounding blown up by 1/sqrt(c) into the scalar products).
// The image Q z feeds the FFT pipeline; the per-k projections restore Q^-1.  With Delta_mv =
// eps_{m,k+Q} - eps_{vk}, four [nks][nbnd (m)][nbnd (v)] tables in double:
//   sp   = 1 - sqrt(c) (1 where c = 0)  coefficient of S = U^H t in the operator's projection
//   da   = [c > 0] (1 - c) Delta        coefficient of Z = U^H z there (D's component along m)
//   keep = [c == 0]                     the projection P'_v of the Lanczos vectors
//   qh   = [c > 0] (1 - sqrt(c))        the image: Q z = z - U (qh Z)
// All null: an insulator.
struct MetalDev {
  const double* sp;
  const double* da;
  const double* keep;
  const double* qh;
};

static __device__ __forceinline__ long metal_idx(int k, int m, int v, int nbnd) {
  return ((long)k * nbnd + m) * nbnd + v;
}

// The sum of one double per thread over the block, in a fixed order (threads' values by warp,
// then the warps in order); every thread gets it.  Ends synchronised.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double wsum[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
  __syncthreads();
  return t;
}

// x <- P_c x for every orbital of k (in place); with coef ([nks][nbnd][nbnd], m-major), the
// component along u_m of band v is removed with weight coef[k][m][v] instead of 1.  The bands
// of k are independent: grid (nks, nvec, nsplit) with nsplit dividing nbnd, each CTA taking
// nbnd/nsplit of them.  block 128.
template <typename T>
__global__ void __launch_bounds__(128) k_project(int nks, int nbnd, int npw_pad, const int* __restrict__ npw,
                                                 const cplx<T>* __restrict__ ukq, cplx<T>* __restrict__ x,
                                                 const double* __restrict__ coef) {
  __shared__ cplx<double> cf[32 * 32];
  __shared__ double red[4 * 16];
  const int k = blockIdx.x, vec = blockIdx.y;
  const int nv = nbnd / gridDim.z, v0 = blockIdx.z * nv;
  const long base = (((long)vec * nks + k) * nbnd + v0) * npw_pad;
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  block_dots<T>(uk, npw_pad, x + base, npw_pad, npw[k], nbnd, nv, nullptr, cf, red);
  if (coef) {
    for (int i = threadIdx.x; i < nbnd * nv; i += blockDim.x) {
      const int m = i / nv;
      const double c = coef[((long)k * nbnd + m) * nbnd + v0 + i - m * nv];
      cf[i] = mk(cf[i].x * c, cf[i].y * c);
    }
    __syncthreads();
  }
  subtract_projection<T>(x + base, uk, cf, nbnd, nv, npw_pad);
}

// A metal's image of a batch vector z for the FFT pipeline: img = Q z = z - U (qh Z) and
// zp = [c > 0] Z, Z = U^H z (double), per (vector, k).  grid (nks, nvec), block 128.
template <typename T>
__global__ void __launch_bounds__(128) k_metal_image(int nks, int nbnd, int npw_pad, const int* __restrict__ npw,
                                                     const cplx<T>* __restrict__ ukq, const cplx<T>* __restrict__ z,
                                                     cplx<T>* __restrict__ img, cplx<double>* __restrict__ zp,
                                                     MetalDev md) {
  __shared__ cplx<double> cf[32 * 32];
  __shared__ double red[4 * 16];
  const int k = blockIdx.x, vec = blockIdx.y;
  const long base = ((long)vec * nks + k) * nbnd * npw_pad;
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  block_dots<T>(uk, npw_pad, z + base, npw_pad, npw[k], nbnd, nbnd, nullptr, cf, red);
  for (int i = threadIdx.x; i < nbnd * nbnd; i += blockDim.x) {
    const long ci = (long)k * nbnd * nbnd + i;
    const cplx<double> v = cf[i];
    const double kept = md.keep[ci] == 0.0 ? 1.0 : 0.0, q = md.qh[ci];
    zp[(long)vec * nks * nbnd * nbnd + ci] = mk(v.x * kept, v.y * kept);
    cf[i] = mk(v.x * q, v.y * q);
  }
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) img[base + i] = z[base + i];
  __syncthreads();
  subtract_projection<T>(img + base, uk, cf, nbnd, nbnd, npw_pad);
}

// ---------------------------------------------------------------------------------------
// Device-side Lanczos bookkeeping.
struct Coef {
  double* beta;            // [cap]
  cplx<double>* gamma;     // [cap]
  cplx<double>* zpart;     // [cap][nks]  per-k partials of z_j
  int* err;                // [2] code, first failing step
};

__device__ __forceinline__ void flag_error(int* err, int code, int step) {
  if (atomicCAS(err, 0, code) == 0) err[1] = step;
}

// (1/n) sum_i p[i*stride + offset], i < n, by the whole block in a fixed order; every thread
// gets the result.
__device__ __forceinline__ double block_mean(const double* p, int n, int stride = 1, int offset = 0) {
  __shared__ double wsum[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[(long)i * stride + offset];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
  __syncthreads();
  return t / n;
}

// Pseudo-Hermitian step j (read from the device step counter, so that a captured step can be
// replayed) for one band group of one k-point (P_c, the norm and z act band by
// band, so groups of bpc bands are independent): beta_j from the ngrp partials per k of
// Re(r_j^H X_j) (every block re-reduces them in the same order), the group's z_j partial,
// r_{j+1} = P_c(X_j/beta_j - beta_j v_{j-1}) formed in shared memory and written to R (a
// metal: keep = MetalDev::keep, the projection P'_v), v_j = r_j/beta_j.  The sphere columns of r_{j+1} are then inverse-FFT'd along axis 3 by
// k_zinv.  grid (nks, ngrp), block 256.  smem: r [bpc][npw_pad], S [nbnd*bpc] (double
// complex), reduction scratch.
template <typename T>
__global__ void __launch_bounds__(256) k_ph_update(const int* __restrict__ jdev, SphereDev s, int nbnd, int bpc,
                                                   const double* __restrict__ part, cplx<T>* __restrict__ R,
                                                   const cplx<T>* __restrict__ X, cplx<T>* __restrict__ Vp,
                                                   const cplx<T>* __restrict__ y, const cplx<T>* __restrict__ ukq,
                                                   Coef co, double tol, const double* __restrict__ keep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = *jdev, r_upper = (j % 2 == 0) ? 1 : 0;   // step index from the device counter
  const int npw_pad = s.npw_pad, nks = s.nks;
  const int k = blockIdx.x, grp = blockIdx.y, ngrp = gridDim.y;
  cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<double>* cf = reinterpret_cast<cplx<double>*>(rs + bpc * npw_pad);
  double* red = reinterpret_cast<double*>(cf + nbnd * bpc);
  __shared__ double sbeta;
  const double b2 = block_mean(part, nks * ngrp) * ngrp;
  if (threadIdx.x == 0) {
    double b = 1.0;
    if (!(b2 > tol)) flag_error(co.err, b2 <= 0.0 ? DEV_NOTPD : DEV_BREAKDOWN, j);
    else b = sqrt(b2);
    sbeta = b;
    if (k == 0 && grp == 0) { co.beta[j - 1] = b; co.gamma[j - 1] = mk(b, 0.0); }
  }
  __syncthreads();
  const double b = sbeta;
  const long base = ((long)k * nbnd + grp * bpc) * npw_pad;
  const int np = s.npw[k];
  const long zi = (long)(j - 1) * nks * ngrp + (long)k * ngrp + grp;
  if (r_upper) {  // z_j partial = (y, r_j)/beta_j over the group's bands
    block_dots_fixed<T, 1, 1>(y + base, 0, R + base, 0, bpc * npw_pad, nullptr, cf, red);
    if (threadIdx.x == 0) co.zpart[zi] = mk(cf[0].x / b, cf[0].y / b);
  } else if (threadIdx.x == 0) {
    co.zpart[zi] = mk(0.0, 0.0);
  }
  const T ib = (T)(1.0 / b), bb = (T)b;
  for (int i = threadIdx.x; i < bpc * npw_pad; i += blockDim.x) {
    const cplx<T> r = R[base + i];
    rs[i] = X[base + i] * ib - Vp[base + i] * bb;
    Vp[base + i] = r * ib;
  }
  __syncthreads();
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  proj_dots<T>(uk, npw_pad, rs, npw_pad, np, nbnd, bpc, cf, red);
  if (keep) {  // a metal: only the states with c_mv = 0 are removed
    for (int i = threadIdx.x; i < nbnd * bpc; i += blockDim.x) {
      const int m = i / bpc;
      const double c = keep[metal_idx(k, m, grp * bpc + i - m * bpc, nbnd)];
      cf[i] = mk(cf[i].x * c, cf[i].y * c);
    }
    __syncthreads();
  }
  subtract_projection<T>(rs, uk, cf, nbnd, bpc, npw_pad);
  for (int i = threadIdx.x; i < bpc * npw_pad; i += blockDim.x) R[base + i] = rs[i];
}

// A metal's projection coefficients of the operator for one band group of k (kept out of line:
// the insulators' kernel keeps its registers): cf <- sp S - da Z (Z = U^H z of the input, from
// k_metal_image), so that the output's component along a kept u_m is sqrt(c) S + (1 - c)
// Delta Z; returns the term sum qh Re(conj(Z) <u_m|X>) that turns the partial Re(Q z, X) the
// kernel forms into Re(z, X) (to every thread).
static __device__ __noinline__ double metal_operator_coefs(const MetalDev md, int k, int v0, int nbnd, int bpc,
                                                    const cplx<double>* zp, cplx<double>* cf) {
  double corr = 0.0;
  for (int i = threadIdx.x; i < nbnd * bpc; i += blockDim.x) {
    const int m = i / bpc;
    const long ci = metal_idx(k, m, v0 + i - m * bpc, nbnd);
    const cplx<double> sv = cf[i], zv = zp[ci];
    const double p = md.sp[ci], d = md.da[ci];
    const cplx<double> c = mk(p * sv.x - d * zv.x, p * sv.y - d * zv.y);
    corr += md.qh[ci] * (zv.x * (sv.x - c.x) + zv.y * (sv.y - c.y));   // Re conj(Z) <u_m|X>
    cf[i] = c;
  }
  return block_sum(corr);
}

// Last stage of the operator fused with the per-k projections, for one group of bpc bands of
// one k-point (the kinetic, KB and P_c terms act band by band): forward FFT of the group's
// columns along axis 3 and gather of the sphere (1/N^3), + (1/2|k+Q+G|^2 - eps_vk) x, + KB
// sum_p beta_p D_p <beta_p|x>, then P_c, the output X and the group's partial Re(x^H X)
// (a metal: x is the image Q z, zp holds Z = U^H z per vector; the output is the operator
// on z through the MetalDev tables, and the partial Re(z^H X)).
// grid (nks, nvec, ngrp), block 256.  smem: x, t [bpc][npw_pad]; coefficients; scratch.
template <typename T, int N, int PR = 0>
__global__ void __launch_bounds__(256, 2) k_zfwd_proj(SphereDev s, int nbnd, int bpc, const cplx<T>* __restrict__ cbuf,
                                                   int cb_ncol, const cplx<T>* __restrict__ xin,
                                                   const T* __restrict__ kin, const double* __restrict__ eps,
                                                   const cplx<T>* __restrict__ ukq, const cplx<T>* __restrict__ bkq,
                                                   const double* __restrict__ dij, int nproj,
                                                   cplx<T>* __restrict__ xout, double* __restrict__ part,
                                                   MetalDev md, const cplx<double>* __restrict__ zp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int npw_pad = s.npw_pad, nks = s.nks;
  const int k = blockIdx.x, vec = blockIdx.y, grp = blockIdx.z, ngrp = gridDim.z;
  const int v0 = grp * bpc;
  cplx<T>* xs = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* ts = xs + bpc * npw_pad;
  cplx<double>* cf = reinterpret_cast<cplx<double>*>(ts + bpc * npw_pad);   // [max(nproj, nbnd) * bpc]
  double* red = reinterpret_cast<double*>(cf + (nproj > nbnd ? nproj : nbnd) * bpc);
  __shared__ T epsk[32];
  const long o0 = ((long)vec * nks + k) * nbnd + v0;      // first orbital of the group
  const long base = o0 * npw_pad;
  const int np = s.npw[k];
  const cplx<T>* bk = bkq + (long)k * nproj * npw_pad;
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  if (threadIdx.x < bpc) epsk[threadIdx.x] = (T)eps[k * nbnd + v0 + threadIdx.x];
  __syncthreads();
  for (int i = threadIdx.x; i < bpc * npw_pad; i += blockDim.x) {
    const int v = i / npw_pad, gi = i - v * npw_pad;
    const cplx<T> xv = xin[base + i];
    xs[i] = xv;
    ts[i] = xv * (kin[(long)k * npw_pad + gi] - epsk[v]);
  }
  __syncthreads();
  const int nc = s.ncol[k];
  const T scale = T(1) / T(N * N * N);
  for (int it = threadIdx.x; it < bpc * nc; it += blockDim.x) {
    const int v = it / nc, c = it - v * nc;
    const int4 cl = s.col[k * s.ncol_max + c];
    if (!LL_INB(c < cb_ncol)) continue;
    const cplx<T>* src = cbuf + (o0 + v) * (long)N * cb_ncol + c;
    cplx<T> a[N];
#pragma unroll
    for (int p = 0; p < N; ++p) a[p] = src[(long)p * cb_ncol];
    fft_line<T, N, -1>(a);
    const int st = s.colstart[k * s.ncol_max + c];
    cplx<T>* dst = ts + v * npw_pad + st;
#pragma unroll
    for (int p = 0; p < N; ++p) {
      const int i = wrapn<N>(p - cl.z);
      if (line_kept<N, PR>(p) && i < cl.w && LL_INB(st >= 0 && st + i < npw_pad)) dst[i] = dst[i] + a[p] * scale;
    }
  }
  __syncthreads();
  if (nproj > 0) {
    small_dots<T>(bk, npw_pad, xs, npw_pad, np, nproj, bpc, dij, cf, red);   // D_p <beta_p|x_v>
    cplx<T>* ct = reinterpret_cast<cplx<T>*>(red);    // the coefficients in T (red is free now)
    for (int i = threadIdx.x; i < nproj * bpc; i += blockDim.x) ct[i] = mk((T)cf[i].x, (T)cf[i].y);
    __syncthreads();
    for (int i = threadIdx.x; i < bpc * npw_pad; i += blockDim.x) {
      const int v = i / npw_pad, gi = i - v * npw_pad;
      cplx<T> acc = ts[i];
      for (int p = 0; p < nproj; ++p) acc = acc + cmul(bk[(long)p * npw_pad + gi], ct[p * bpc + v]);
      ts[i] = acc;
    }
    __syncthreads();
  }
  small_dots<T>(uk, npw_pad, ts, npw_pad, np, nbnd, bpc, nullptr, cf, red);
  const double corr =
      md.sp ? metal_operator_coefs(md, k, v0, nbnd, bpc, zp + (long)vec * nks * nbnd * nbnd, cf) : 0.0;
  subtract_projection<T>(ts, uk, cf, nbnd, bpc, npw_pad);
  for (int i = threadIdx.x; i < bpc * npw_pad; i += blockDim.x) xout[base + i] = ts[i];
  small_dots<T>(xs, 0, ts, 0, bpc * npw_pad, 1, 1, nullptr, cf, red);
  if (threadIdx.x == 0) part[((long)vec * nks + k) * ngrp + grp] = cf[0].x + corr;
}

// Non-Hermitian step j after the two operator applications XV = L v_j, XW = L^dag w_j, for
// one group of bpc bands of one k-point: v_hat = P_c(XV - gamma_j v_{j-1}), w_hat =
// P_c(XW - conj(beta_j) w_{j-1}) (stored in XV, XW), the group's partials of s = (w_hat,
// v_hat) and of z_j = (y, v_j) (a metal: keep = MetalDev::keep, the projection P'_v).
// grid (nks, ngrp), block 128.
template <typename T>
__global__ void __launch_bounds__(128) k_nh_update(int j, int upper, int nks, int nbnd, int bpc, int npw_pad,
                                                   const int* __restrict__ npw, cplx<T>* __restrict__ XV,
                                                   cplx<T>* __restrict__ XW, const cplx<T>* __restrict__ Vp,
                                                   const cplx<T>* __restrict__ Wp, const cplx<T>* __restrict__ Vc,
                                                   const cplx<T>* __restrict__ y, const cplx<T>* __restrict__ ukq,
                                                   Coef co, cplx<double>* __restrict__ spart,
                                                   const double* __restrict__ keep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* vs = reinterpret_cast<cplx<T>*>(smem_raw);          // [bpc][npw_pad]
  cplx<T>* ws = vs + bpc * npw_pad;
  cplx<double>* cf = reinterpret_cast<cplx<double>*>(ws + bpc * npw_pad);   // [nbnd * bpc]
  double* red = reinterpret_cast<double*>(cf + nbnd * bpc);
  const int k = blockIdx.x, grp = blockIdx.y, ngrp = gridDim.y;
  const long base = ((long)k * nbnd + grp * bpc) * npw_pad;
  const long zi = (long)(j - 1) * nks * ngrp + (long)k * ngrp + grp;
  const int np = npw[k];
  const double bj = co.beta[j - 1];
  const cplx<double> gj = co.gamma[j - 1];
  const cplx<T> g = mk((T)gj.x, (T)gj.y), bc = mk((T)bj, (T)0);
  if (upper) {  // z_j partial = (y, v_j) over the group's bands
    block_dots<T>(y + base, 0, Vc + base, 0, bpc * npw_pad, 1, 1, nullptr, cf, red);
    if (threadIdx.x == 0) co.zpart[zi] = cf[0];
  } else if (threadIdx.x == 0) {
    co.zpart[zi] = mk(0.0, 0.0);
  }
  for (int i = threadIdx.x; i < bpc * npw_pad; i += blockDim.x) {
    vs[i] = XV[base + i] - cmul(g, Vp[base + i]);
    ws[i] = XW[base + i] - cmul(bc, Wp[base + i]);
  }
  __syncthreads();
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  for (int h = 0; h < 2; ++h) {
    cplx<T>* xs = h ? ws : vs;
    block_dots<T>(uk, npw_pad, xs, npw_pad, np, nbnd, bpc, nullptr, cf, red);
    if (keep) {  // a metal: P'_v, only the states with c_mv = 0 removed
      for (int i = threadIdx.x; i < nbnd * bpc; i += blockDim.x) {
        const int m = i / bpc;
        const double c = keep[metal_idx(k, m, grp * bpc + i - m * bpc, nbnd)];
        cf[i] = mk(cf[i].x * c, cf[i].y * c);
      }
      __syncthreads();
    }
    subtract_projection<T>(xs, uk, cf, nbnd, bpc, npw_pad);
  }
  for (int i = threadIdx.x; i < bpc * npw_pad; i += blockDim.x) {
    XV[base + i] = vs[i];
    XW[base + i] = ws[i];
  }
  block_dots<T>(ws, 0, vs, 0, bpc * npw_pad, 1, 1, nullptr, cf, red);
  if (threadIdx.x == 0) spart[(long)k * ngrp + grp] = cf[0];
}

// Non-Hermitian normalisation at the end of step j: beta_{j+1} = sqrt|s|, gamma_{j+1} =
// s/beta_{j+1}; v_{j-1} <- v_j, v_j <- v_hat/beta; w_{j-1} <- w_j, w_j <- w_hat/conj(gamma).
template <typename T>
__global__ void __launch_bounds__(128) k_nh_normalize(int j, int nks, int nbnd, int npw_pad, int nchunk,
                                                      const cplx<double>* __restrict__ spart,
                                                      const cplx<T>* __restrict__ XV, const cplx<T>* __restrict__ XW,
                                                      cplx<T>* __restrict__ Vc, cplx<T>* __restrict__ Vp,
                                                      cplx<T>* __restrict__ Wc, cplx<T>* __restrict__ Wp, Coef co,
                                                      double tol) {
  __shared__ cplx<double> sc[2];
  const int k = blockIdx.x;
  // spart: nks nchunk partials (one per k, or per (k, chunk) on the split path)
  const double sr = block_mean(reinterpret_cast<const double*>(spart), nks * nchunk, 2, 0) * nchunk;
  const double si = block_mean(reinterpret_cast<const double*>(spart), nks * nchunk, 2, 1) * nchunk;
  if (threadIdx.x == 0) {
    const double a = sqrt(sr * sr + si * si);
    double b = sqrt(a);
    cplx<double> gm = mk(sr / b, si / b);
    if (!(a > tol)) { flag_error(co.err, DEV_BREAKDOWN, j + 1); b = 1.0; gm = mk(1.0, 0.0); }
    sc[0] = mk(b, 0.0);
    sc[1] = gm;
    if (k == 0) { co.beta[j] = b; co.gamma[j] = gm; }
  }
  __syncthreads();
  const double b = sc[0].x;
  const cplx<double> gm = sc[1];
  // 1/conj(gamma) = gamma/|gamma|^2
  const double gg = gm.x * gm.x + gm.y * gm.y;
  const cplx<T> igc = mk((T)(gm.x / gg), (T)(gm.y / gg));
  const T ib = (T)(1.0 / b);
  const long base = (long)k * nbnd * npw_pad;
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    Vp[base + i] = Vc[base + i];
    Vc[base + i] = XV[base + i] * ib;
    Wp[base + i] = Wc[base + i];
    Wc[base + i] = cmul(XW[base + i], igc);
  }
}

// z_j = (1/nks) sum_k zpart[j][k] for j in [j0, j1)
// Device step counter of the pseudo-Hermitian recursion: set before a run of steps, advanced
// at the end of every step (one thread).
static __global__ void k_step_set(int* jdev, int j) { *jdev = j; }
static __global__ void k_step_next(int* jdev) { *jdev += 1; }

// (nzp partials per step: one per k, or one per (k, chunk) on the split path)
static __global__ void k_reduce_z(const cplx<double>* __restrict__ zpart, int nzp, int nks, int j0, int j1,
                                  cplx<double>* __restrict__ z) {
  const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= j1) return;
  double zr = 0, zi = 0;
  for (int k = 0; k < nzp; ++k) { zr += zpart[(long)j * nzp + k].x; zi += zpart[(long)j * nzp + k].y; }
  z[j] = mk(zr / nks, zi / nks);
}

// ---------------------------------------------------------------------------------------
// Set-up kernels.
// For each Miller of sphere(k+Q): its index in sphere(k) (both lexicographic), or -1.
static __global__ void k_intersection_map(int nks, const int* __restrict__ off_k, const int* __restrict__ npw_k,
                                   const int* __restrict__ mil_k, const int* __restrict__ off_q,
                                   const int* __restrict__ npw_q, const int* __restrict__ mil_q, int npw_pad,
                                   int* __restrict__ map) {
  const int k = blockIdx.x;
  const int* mk_ = mil_k + 3L * off_k[k];
  const int n = npw_k[k];
  for (int i = threadIdx.x; i < npw_pad; i += blockDim.x) {
    int res = -1;
    if (i < npw_q[k]) {
      const int* q = mil_q + 3L * (off_q[k] + i);
      int lo = 0, hi = n - 1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int* m = mk_ + 3 * mid;
        int c = (m[0] != q[0]) ? (m[0] < q[0] ? -1 : 1)
              : (m[1] != q[1]) ? (m[1] < q[1] ? -1 : 1)
              : (m[2] != q[2]) ? (m[2] < q[2] ? -1 : 1) : 0;
        if (c == 0) { res = mid; break; }
        if (c < 0) lo = mid + 1; else hi = mid - 1;
      }
    }
    map[(long)k * npw_pad + i] = res;
  }
}

// y_{vk}(G) = u_{vk}(G) where G is also in sphere(k), else 0 (projection follows).
// grid (nks, nbnd), block 128.
template <typename T>
__global__ void k_gather_y(int nks, int nbnd, int npw_pad_q, int npw_pad_k, const int* __restrict__ map,
                           const cplx<T>* __restrict__ uk, cplx<T>* __restrict__ y) {
  const int k = blockIdx.x, v = blockIdx.y;
  for (int g = threadIdx.x; g < npw_pad_q; g += blockDim.x) {
    const int m = map[(long)k * npw_pad_q + g];
    y[((long)k * nbnd + v) * npw_pad_q + g] =
        (m >= 0 && LL_INB(m < npw_pad_k)) ? uk[((long)k * nbnd + v) * npw_pad_k + m] : czero<T>();
  }
}

// ALDA kernel f_xc = d v_xc/dn of Slater exchange + Perdew-Zunger 1981 correlation, in
// double, from the ground-state density; 0 where n <= 1e-10.
__device__ __forceinline__ double pz81_fxc(double n) {
  if (!(n > 1e-10)) return 0.0;
  const double pi = 3.14159265358979323846;
  const double rs = cbrt(3.0 / (4.0 * pi * n));
  const double cx = 0.75 * cbrt(3.0 / pi);
  const double fx = -4.0 / 9.0 * cx * pow(n, -2.0 / 3.0);
  double d1, d2;
  if (rs >= 1.0) {
    const double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
    const double s = sqrt(rs);
    const double den = 1.0 + b1 * s + b2 * rs;
    const double dden = b1 / (2.0 * s) + b2;
    const double d2den = -b1 / (4.0 * s * s * s);
    d1 = -g * dden / (den * den);
    d2 = -g * (d2den * den - 2.0 * dden * dden) / (den * den * den);
  } else {
    const double A = 0.0311, C = 0.0020, D = -0.0116;
    d1 = A / rs + C * (log(rs) + 1.0) + D;
    d2 = -A / (rs * rs) + C / rs;
  }
  const double dvc = 2.0 / 3.0 * d1 - rs / 3.0 * d2;
  return fx + dvc * (-rs / (3.0 * n));
}

// ---- set-up from device-resident inputs (ll_system_desc.where = LL_WHERE_DEVICE) --------

// The smallest index of a NaN or infinity among n values into *first, which the caller sets
// to all ones beforehand (left so when every value is finite).
static __global__ void k_first_nonfinite(const double* __restrict__ p, long n, unsigned long long* first) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (!isfinite(p[i])) atomicMin(first, (unsigned long long)i);
}

// Packed complex rows [k][row][npw[k]] (k blocks at nrow * off[k]) -> padded [k][row][npw_pad]
// in T, zero on the padding, each row times rscale[k][row] when given.  grid (nks, nrow),
// block 256.
template <typename T>
__global__ void k_pad_rows(const double* __restrict__ src, const int* __restrict__ off, const int* __restrict__ npw,
                           int nrow, int npw_pad, const double* __restrict__ rscale, cplx<T>* __restrict__ dst) {
  const int k = blockIdx.x, r = blockIdx.y, n = npw[k];
  const double* s = src + 2 * ((long)nrow * off[k] + (long)r * n);
  // u_k only: sqrt of the k-point weight times sqrt of the band's occupation (a metal)
  const double f = rscale ? rscale[(long)k * nrow + r] : 1.0;
  cplx<T>* d = dst + ((long)k * nrow + r) * npw_pad;
  for (int g = threadIdx.x; g < npw_pad; g += blockDim.x)
    d[g] = g < n ? mk((T)(f * s[2 * g]), (T)(f * s[2 * g + 1])) : czero<T>();
}

// Grids [j1][j2][j3] -> [j3][j2][j1]: V in T, the density in double.
template <typename T>
__global__ void k_grids_in(int n, const double* __restrict__ vloc, const double* __restrict__ rho, T* __restrict__ vl,
                           double* __restrict__ rh) {
  const long n3 = (long)n * n * n;
  for (long dst = (long)blockIdx.x * blockDim.x + threadIdx.x; dst < n3; dst += (long)gridDim.x * blockDim.x) {
    const long j1 = dst % n, j2 = (dst / n) % n, j3 = dst / ((long)n * n);
    const long src = (j1 * n + j2) * n + j3;
    vl[dst] = (T)vloc[src];
    rh[dst] = rho[src];
  }
}

template <typename T>
__global__ void k_fxc(long n3, const double* __restrict__ rho, T* __restrict__ fxc, int on) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n3; i += (long)gridDim.x * blockDim.x)
    fxc[i] = on ? (T)pz81_fxc(rho[i]) : T(0);
}

template <typename T>
__global__ void k_scale(long n, const cplx<T>* __restrict__ a, double s, cplx<T>* __restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = a[i] * (T)s;
}

// part[k] = Re sum conj(a) b over the k block (for norms).
template <typename T>
__global__ void __launch_bounds__(128) k_dot_re(int nks, int nbnd, int npw_pad, const cplx<T>* __restrict__ a,
                                                const cplx<T>* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[4];
  const int k = blockIdx.x;
  const long base = (long)k * nbnd * npw_pad;
  double acc = 0;
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    const cplx<T> t = cjmul(a[base + i], b[base + i]);
    acc += (double)t.x;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[k] = s;
  }
}

// ---------------------------------------------------------------------------------------
// Spectrum (Eqs. 32-33, 5): per frequency, with A = (w + i eta) I - T, chi_LL = z^T A^-1 e_1
// = u_1 where A^T u = z, eliminated from the bottom row up (the continued fraction):
//   d_M = w, r_M = z_M;  d_j = w - beta_{j+1} gamma_{j+1} / d_{j+1},
//   r_j = z_j + beta_{j+1} r_{j+1} / d_{j+1};  u_1 = r_1 / d_1.
// chi = pref b_1 u_1, eps^-1 = 1 + v_Q chi, eps = 1/eps^-1.  One thread per frequency.
__device__ __forceinline__ cplx<double> cdiv(cplx<double> a, cplx<double> b) {
  const double d = b.x * b.x + b.y * b.y;
  return mk((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Continuation of the coefficients past the m computed ones (Sec. 2.5, Sec. 3.3): for an
// index i >= m, beta_i = b[i % 2] and gamma_i = g[i % 2] ('constant': b[0] = b[1]); z_i = 0.
struct ExtrapTail {
  double b[2];
  cplx<double> g[2];
};

// The tail constants: means over the positions max(1, m/2)..m-1, both parities together
// (kind 1, constant) or each parity apart (kind 2, bi-constant), fixed summation order.
// One block of 256 threads.
static __global__ void __launch_bounds__(256) k_extrap_tail(int m, int kind, const double* __restrict__ beta,
                                                            const cplx<double>* __restrict__ gamma,
                                                            ExtrapTail* __restrict__ tail) {
  __shared__ double red[8][6];
  const int h = m / 2 > 1 ? m / 2 : 1;
  double s[6] = {0, 0, 0, 0, 0, 0};   // per parity: beta, Re gamma, Im gamma
  for (int i = h + threadIdx.x; i < m; i += blockDim.x) {
    const int p = (kind == 2) ? (i & 1) : 0;
    s[3 * p] += beta[i];
    s[3 * p + 1] += gamma[i].x;
    s[3 * p + 2] += gamma[i].y;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const double v = warp_sum(s[c]);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int c = 0; c < 6; ++c) t[c] += red[w][c];
    int n[2] = {0, 0};
    for (int i = h; i < m; ++i) ++n[(kind == 2) ? (i & 1) : 0];
    for (int p = 0; p < 2; ++p) {
      const int q = (kind == 2) ? p : 0;
      const double c = n[q] > 0 ? 1.0 / n[q] : 0.0;
      tail->b[p] = t[3 * q] * c;
      tail->g[p] = mk(t[3 * q + 1] * c, t[3 * q + 2] * c);
    }
  }
}

// m_total > m continues the chain with `tail` (T grows to m_total x m_total; z stays m long).
static __global__ void k_spectrum(int m, int m_total, const ExtrapTail* __restrict__ tail,
                                  const double* __restrict__ beta, const cplx<double>* __restrict__ gamma,
                                  const cplx<double>* __restrict__ z, int nw, const double* __restrict__ w_ha,
                                  double eta, double pref, double vq, cplx<double>* __restrict__ chi,
                                  cplx<double>* __restrict__ epsi, cplx<double>* __restrict__ eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  if (m_total < m || !tail) m_total = m;
  const cplx<double> w = mk(w_ha[i], eta);
  cplx<double> d = w, r = (m_total > m) ? mk(0.0, 0.0) : z[m - 1];
  for (int j = m_total - 2; j >= 0; --j) {
    const int c = j + 1;
    const double b = c < m ? beta[c] : tail->b[c & 1];
    const cplx<double> g = c < m ? gamma[c] : tail->g[c & 1];
    const cplx<double> q = cdiv(cmul(mk(b, 0.0), g), d);
    const cplx<double> rr = cdiv(mk(b * r.x, b * r.y), d);
    d = w - q;
    r = (j < m ? z[j] : mk(0.0, 0.0)) + rr;
  }
  const cplx<double> u1 = cdiv(r, d);
  const cplx<double> c = u1 * (pref * beta[0]);
  chi[i] = c;
  const cplx<double> ei = mk(1.0 + vq * c.x, vq * c.y);
  epsi[i] = ei;
  eps[i] = cdiv(mk(1.0, 0.0), ei);
}

}  // namespace ll
