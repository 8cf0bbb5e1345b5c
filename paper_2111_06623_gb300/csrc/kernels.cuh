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
  const int4* col;      // [nks][ncol_max]  (m1, m2, m3 of the first point, point count)
  const int* colstart;  // [nks][ncol_max]  first point of the column in the sphere order
  const int4* row;      // [nks][nrow_max]  (m1, first column, m2 of the first column, columns)
};

__device__ __forceinline__ int wrap(int m, int n) { int r = m % n; return r < 0 ? r + n : r; }

template <typename T>
__device__ __forceinline__ cplx<T> ldc(const cplx<T>* p) { return *p; }

// ---------------------------------------------------------------------------------------
// Sphere -> columns: scatter each column's points and inverse-FFT along axis 3.
// grid (nks, nvec), block 128; item = (v, column).
template <typename T, int N>
__global__ void __launch_bounds__(128) k_zinv(SphereDev s, const cplx<T>* __restrict__ x, int nbnd,
                                              cplx<T>* __restrict__ cbuf, int cb_ncol) {
  const int k = blockIdx.x, vec = blockIdx.y;
  const int nc = s.ncol[k];
  for (int it = threadIdx.x; it < nbnd * nc; it += blockDim.x) {
    const int v = it / nc, c = it - v * nc;
    const long o = ((long)vec * s.nks + k) * nbnd + v;
    const int4 cl = s.col[k * s.ncol_max + c];
    const int st = s.colstart[k * s.ncol_max + c];
    const cplx<T>* src = x + o * s.npw_pad + st;
    cplx<T> a[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
      const int i = wrap(p - cl.z, N);
      a[p] = (i < cl.w) ? src[i] : czero<T>();
    }
    fft_line<T, N, +1>(a);
    cplx<T>* dst = cbuf + o * (long)N * cb_ncol + c;
#pragma unroll
    for (int p = 0; p < N; ++p) dst[(long)p * cb_ncol] = a[p];
  }
}

// Columns -> sphere: forward FFT along axis 3, gather the column's points, scale 1/N^3.
template <typename T, int N>
__global__ void __launch_bounds__(128) k_zfwd(SphereDev s, const cplx<T>* __restrict__ cbuf, int cb_ncol,
                                              int nbnd, cplx<T>* __restrict__ out) {
  const int k = blockIdx.x, vec = blockIdx.y;
  const int nc = s.ncol[k];
  const T scale = T(1) / T(N * N * N);
  for (int it = threadIdx.x; it < nbnd * nc; it += blockDim.x) {
    const int v = it / nc, c = it - v * nc;
    const long o = ((long)vec * s.nks + k) * nbnd + v;
    const int4 cl = s.col[k * s.ncol_max + c];
    const int st = s.colstart[k * s.ncol_max + c];
    const cplx<T>* src = cbuf + o * (long)N * cb_ncol + c;
    cplx<T> a[N];
#pragma unroll
    for (int p = 0; p < N; ++p) a[p] = src[(long)p * cb_ncol];
    fft_line<T, N, -1>(a);
    cplx<T>* dst = out + o * s.npw_pad + st;
#pragma unroll
    for (int p = 0; p < N; ++p) {
      const int i = wrap(p - cl.z, N);
      if (i < cl.w) dst[i] = a[p] * scale;
    }
  }
  // zero the padding of every orbital of this k
  const int np = s.npw[k];
  for (int it = threadIdx.x; it < nbnd * (s.npw_pad - np); it += blockDim.x) {
    const int v = it / (s.npw_pad - np), i = np + it % (s.npw_pad - np);
    out[(((long)vec * s.nks + k) * nbnd + v) * s.npw_pad + i] = czero<T>();
  }
}

// ---------------------------------------------------------------------------------------
// Per-plane pass of one operator application.  grid (N planes, groups), block 128.
// For every orbital of the group (BO at a time): inverse 2D FFT of the plane's columns,
// t(r) = V(r) x(r), optional response-density accumulation conj(u(r)) x(r), forward 2D FFT
// back to the columns (in place).  mode 0: pass 1 (V x, density if dens_vec matches);
// mode 1: pass 2 (t(r) = v'(r) u(r) from the orbital grid, added into the columns);
// mode 2: inverse only, store x(r) into `grid_out` (orbital grids at set-up).
struct XYArgs {
  SphereDev s;
  int nbnd, norb;              // orbitals handled by this launch
  int cb_ncol;
  int per_group;               // orbitals per group
  int o_off;                   // first orbital of this launch (orbital o = o_off + local index)
  int dens_vec;                // vector whose orbitals feed the density (-1: none)
  int mode;
};

template <typename T, int N, int BO>
__global__ void __launch_bounds__(128) k_xy(XYArgs a, cplx<T>* __restrict__ cbuf, const T* __restrict__ vloc,
                                            const cplx<T>* __restrict__ vpr, const cplx<T>* __restrict__ ur,
                                            cplx<T>* __restrict__ nprt, cplx<T>* __restrict__ grid_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int iz = blockIdx.x, g = blockIdx.y;
  const SphereDev& s = a.s;
  constexpr int NP = N + 1;
  cplx<T>* Cs = reinterpret_cast<cplx<T>*>(smem_raw);                 // [BO][cb_ncol]
  cplx<T>* Ys = Cs + BO * a.cb_ncol;                                    // [BO][nrow_max][NP]
  cplx<T>* Ds = Ys + BO * s.nrow_max * NP;                              // [BO][N][NP] (density)
  cplx<T>* Pl = Ds + ((a.mode == 0 && a.dens_vec >= 0) ? BO * N * NP : 0);  // plane [N][NP]
  const bool want_dens = (a.mode == 0 && a.dens_vec >= 0);
  const long plane = (long)N * N;

  // the plane of V (mode 0) or v' (mode 1)
  if (a.mode == 0) {
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) Pl[(i / N) * NP + i % N] = mk(vloc[iz * plane + i], T(0));
  } else if (a.mode == 1) {
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) Pl[(i / N) * NP + i % N] = vpr[iz * plane + i];
  }
  if (want_dens)
    for (int i = threadIdx.x; i < BO * N * NP; i += blockDim.x) Ds[i] = czero<T>();

  const int o_begin = a.o_off + g * a.per_group;
  const int o_end = a.o_off + min(a.norb, g * a.per_group + a.per_group);
  for (int ob = o_begin; ob < o_end; ob += BO) {
    const int nb = min(BO, o_end - ob);
    __syncthreads();
    // load the plane's column values of each orbital
    if (a.mode != 1) {
      for (int i = threadIdx.x; i < nb * a.cb_ncol; i += blockDim.x) {
        const int b = i / a.cb_ncol, c = i - b * a.cb_ncol;
        const int o = ob + b, k = (o / a.nbnd) % s.nks;
        Cs[i] = (c < s.ncol[k]) ? cbuf[(long)o * N * a.cb_ncol + (long)iz * a.cb_ncol + c] : czero<T>();
      }
      __syncthreads();
      // inverse FFT along axis 2 of every sphere row (fixed m1)
      for (int i = threadIdx.x; i < nb * s.nrow_max; i += blockDim.x) {
        const int b = i / s.nrow_max, r = i - b * s.nrow_max;
        const int o = ob + b, k = (o / a.nbnd) % s.nks;
        if (r >= s.nrow[k]) continue;
        const int4 rw = s.row[k * s.nrow_max + r];
        cplx<T> l[N];
        const cplx<T>* cs = Cs + b * a.cb_ncol + rw.y;
#pragma unroll
        for (int p = 0; p < N; ++p) {
          const int j = wrap(p - rw.z, N);
          l[p] = (j < rw.w) ? cs[j] : czero<T>();
        }
        fft_line<T, N, +1>(l);
        cplx<T>* ys = Ys + (b * s.nrow_max + r) * NP;
#pragma unroll
        for (int p = 0; p < N; ++p) ys[p] = l[p];
      }
      __syncthreads();
    }
    // axis 1: one line per (orbital, j2)
    for (int i = threadIdx.x; i < nb * N; i += blockDim.x) {
      const int b = i / N, j2 = i - b * N;
      const int o = ob + b, k = (o / a.nbnd) % s.nks;
      const int nr = s.nrow[k];
      const int m1min = s.row[k * s.nrow_max].x;
      const int ko = o % (s.nks * a.nbnd);   // orbital index within its vector
      cplx<T> l[N];
      if (a.mode == 1) {
        const cplx<T>* u = ur + (long)ko * N * plane + iz * plane + (long)j2 * N;
#pragma unroll
        for (int p = 0; p < N; ++p) l[p] = cmul(Pl[j2 * NP + p], u[p]);
      } else {
#pragma unroll
        for (int p = 0; p < N; ++p) {
          const int r = wrap(p - m1min, N);
          l[p] = (r < nr) ? Ys[(b * s.nrow_max + r) * NP + j2] : czero<T>();
        }
        fft_line<T, N, +1>(l);
        if (a.mode == 2) {
          cplx<T>* dst = grid_out + (long)o * N * plane + iz * plane + (long)j2 * N;
#pragma unroll
          for (int p = 0; p < N; ++p) dst[p] = l[p];
          continue;
        }
        if (want_dens && o / (s.nks * a.nbnd) == a.dens_vec) {
          const cplx<T>* u = ur + (long)ko * N * plane + iz * plane + (long)j2 * N;
          cplx<T>* d = Ds + (b * N + j2) * NP;
#pragma unroll
          for (int p = 0; p < N; ++p) d[p] = d[p] + cjmul(u[p], l[p]);
        }
#pragma unroll
        for (int p = 0; p < N; ++p) l[p] = l[p] * Pl[j2 * NP + p].x;
      }
      fft_line<T, N, -1>(l);
#pragma unroll
      for (int p = 0; p < N; ++p) {
        const int r = wrap(p - m1min, N);
        if (r < nr) Ys[(b * s.nrow_max + r) * NP + j2] = l[p];
      }
    }
    __syncthreads();
    if (a.mode == 2) continue;
    // forward FFT along axis 2 of every row, keep the row's columns
    for (int i = threadIdx.x; i < nb * s.nrow_max; i += blockDim.x) {
      const int b = i / s.nrow_max, r = i - b * s.nrow_max;
      const int o = ob + b, k = (o / a.nbnd) % s.nks;
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
        const int j = wrap(p - rw.z, N);
        if (j < rw.w) cs[j] = l[p];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb * a.cb_ncol; i += blockDim.x) {
      const int b = i / a.cb_ncol, c = i - b * a.cb_ncol;
      const int o = ob + b, k = (o / a.nbnd) % s.nks;
      if (c >= s.ncol[k]) continue;
      cplx<T>* dst = cbuf + (long)o * N * a.cb_ncol + (long)iz * a.cb_ncol + c;
      *dst = (a.mode == 1) ? *dst + Cs[i] : Cs[i];
    }
  }
  if (want_dens) {
    __syncthreads();
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
      const int j2 = i / N, j1 = i - j2 * N;
      cplx<T> acc = czero<T>();
      for (int b = 0; b < BO; ++b) acc = acc + Ds[(b * N + j2) * NP + j1];
      nprt[(long)g * N * plane + iz * plane + i] = acc;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Response potential of one density (Eqs. 12-13): n'(r) from the group partials, 3D FFT,
// Hartree 4 pi/|Q+G|^2, inverse FFT, plus f_xc(n0) n'.  Three launches over the grid.
template <typename T, int N>
__global__ void __launch_bounds__(64) k_hxc_fwd(const cplx<T>* __restrict__ nprt, int ngroups, T scale,
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
// Block reductions in double (fixed order: lanes, then warps) -> deterministic.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Dots conj(A_i) . B_j over npw for a list of (i, j) pairs, one warp per pair.  Results
// (times `mult[i]` when given) into out[pair] as complex double.
template <typename T>
__device__ void pair_dots(const cplx<T>* A, int lda, const cplx<T>* B, int ldb, int npw, int ni, int nj,
                          const double* mult, cplx<double>* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int pr = warp; pr < ni * nj; pr += nw) {
    const int i = pr / nj, j = pr - i * nj;
    const cplx<T>* a = A + (long)i * lda;
    const cplx<T>* b = B + (long)j * ldb;
    T re = 0, im = 0;
    for (int g = lane; g < npw; g += 32) {
      const cplx<T> t = cjmul(a[g], b[g]);
      re += t.x;
      im += t.y;
    }
    double dr = warp_sum((double)re), di = warp_sum((double)im);
    if (lane == 0) {
      const double m = mult ? mult[i] : 1.0;
      out[pr] = mk(dr * m, di * m);
    }
  }
}

// The rest of the operator per k-point: kinetic and -eps, KB projectors, P_c, and the
// partial Re(x^H X) of the pseudo-Hermitian norm.  grid (nks, nvec), block 128.
// smem: xs, ts [nbnd][npw_pad], coefficient scratch.
template <typename T>
__global__ void __launch_bounds__(128) k_proj(int nks, int nbnd, int npw_pad, const int* __restrict__ npw,
                                              const cplx<T>* __restrict__ xin, const cplx<T>* __restrict__ tin,
                                              const T* __restrict__ kin, const double* __restrict__ eps,
                                              const cplx<T>* __restrict__ ukq, const cplx<T>* __restrict__ bkq,
                                              const double* __restrict__ dij, int nproj, cplx<T>* __restrict__ xout,
                                              double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = blockIdx.x, vec = blockIdx.y;
  const int np = npw[k];
  cplx<T>* xs = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* ts = xs + nbnd * npw_pad;
  cplx<double>* cf = reinterpret_cast<cplx<double>*>(ts + nbnd * npw_pad);   // [max(nproj,nbnd) * nbnd]
  __shared__ double red[4];
  const long base = ((long)vec * nks + k) * nbnd * npw_pad;
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    const int v = i / npw_pad, gi = i - v * npw_pad;
    const cplx<T> xv = xin[base + i];
    xs[i] = xv;
    const T d = kin[(long)k * npw_pad + gi] - (T)eps[k * nbnd + v];
    ts[i] = tin[base + i] + xv * d;
  }
  __syncthreads();
  if (nproj > 0) {
    const cplx<T>* bk = bkq + (long)k * nproj * npw_pad;
    pair_dots<T>(bk, npw_pad, xs, npw_pad, np, nproj, nbnd, dij, cf);   // D_p <beta_p|x_v>
    __syncthreads();
    for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
      const int v = i / npw_pad, gi = i - v * npw_pad;
      cplx<T> acc = ts[i];
      for (int p = 0; p < nproj; ++p) {
        const cplx<double> c = cf[p * nbnd + v];
        acc = acc + cmul(bk[(long)p * npw_pad + gi], mk((T)c.x, (T)c.y));
      }
      ts[i] = acc;
    }
    __syncthreads();
  }
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  pair_dots<T>(uk, npw_pad, ts, npw_pad, np, nbnd, nbnd, nullptr, cf);       // S = U^H t
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    const int v = i / npw_pad, gi = i - v * npw_pad;
    cplx<T> t = ts[i];
    for (int w = 0; w < nbnd; ++w) {
      const cplx<double> c = cf[w * nbnd + v];
      t = t - cmul(uk[(long)w * npw_pad + gi], mk((T)c.x, (T)c.y));
    }
    xout[base + i] = t;
    const cplx<T> xv = xs[i];
    acc += (double)(xv.x * t.x + xv.y * t.y);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[vec * nks + k] = s;
  }
}

// x <- P_c x for every orbital of k (in place).  grid (nks, nvec), block 128.
template <typename T>
__global__ void __launch_bounds__(128) k_project(int nks, int nbnd, int npw_pad, const int* __restrict__ npw,
                                                 const cplx<T>* __restrict__ ukq, cplx<T>* __restrict__ x) {
  __shared__ cplx<double> cf[32 * 32];
  const int k = blockIdx.x, vec = blockIdx.y;
  const long base = ((long)vec * nks + k) * nbnd * npw_pad;
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  pair_dots<T>(uk, npw_pad, x + base, npw_pad, npw[k], nbnd, nbnd, nullptr, cf);
  __syncthreads();
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    const int v = i / npw_pad, gi = i - v * npw_pad;
    cplx<T> t = x[base + i];
    for (int w = 0; w < nbnd; ++w) {
      const cplx<double> c = cf[w * nbnd + v];
      t = t - cmul(uk[(long)w * npw_pad + gi], mk((T)c.x, (T)c.y));
    }
    x[base + i] = t;
  }
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

// Sum of per-k partials in a fixed order, times 1/nks.
__device__ __forceinline__ double sum_parts(const double* p, int nks) {
  double s = 0.0;
  for (int i = 0; i < nks; ++i) s += p[i];
  return s / nks;
}

// Pseudo-Hermitian step j (1-based) before the operator: beta_j from the partials of
// Re(r_j^H X_j); v_j = r_j/beta_j; z_j partial; r_{j+1} = P_c(X_j/beta_j - beta_j v_{j-1}).
// grid nks, block 128.
template <typename T>
__global__ void __launch_bounds__(128) k_update_ph(int j, int r_upper, int nks, int nbnd, int npw_pad,
                                                   const int* __restrict__ npw, const double* __restrict__ part,
                                                   cplx<T>* __restrict__ R, const cplx<T>* __restrict__ X,
                                                   cplx<T>* __restrict__ Vp, const cplx<T>* __restrict__ y,
                                                   const cplx<T>* __restrict__ ukq, Coef co, double tol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);          // [nbnd][npw_pad]
  cplx<double>* cf = reinterpret_cast<cplx<double>*>(rs + nbnd * npw_pad);   // [nbnd*nbnd + 1]
  __shared__ double sbeta;
  const int k = blockIdx.x;
  if (threadIdx.x == 0) {
    const double b2 = sum_parts(part, nks);
    double b = 0.0;
    if (!(b2 > tol)) {
      flag_error(co.err, b2 <= 0.0 ? DEV_NOTPD : DEV_BREAKDOWN, j);
      b = 1.0;
    } else {
      b = sqrt(b2);
    }
    sbeta = b;
    if (k == 0) { co.beta[j - 1] = b; co.gamma[j - 1] = mk(b, 0.0); }
  }
  __syncthreads();
  const double b = sbeta;
  const long base = (long)k * nbnd * npw_pad;
  const int np = npw[k];
  // z_j partial: (y, r_j) / beta_j when r_j is upper
  if (r_upper) {
    // one warp per band, then the bands summed in order
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int v = warp; v < nbnd; v += nw) {
      T re = 0, im = 0;
      for (int g = lane; g < np; g += 32) {
        const cplx<T> t = cjmul(y[base + (long)v * npw_pad + g], R[base + (long)v * npw_pad + g]);
        re += t.x; im += t.y;
      }
      const double dr = warp_sum((double)re), di = warp_sum((double)im);
      if (lane == 0) cf[v] = mk(dr, di);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double zr = 0, zi = 0;
      for (int v = 0; v < nbnd; ++v) { zr += cf[v].x; zi += cf[v].y; }
      co.zpart[(long)(j - 1) * nks + k] = mk(zr / b, zi / b);
    }
    __syncthreads();
  } else if (threadIdx.x == 0) {
    co.zpart[(long)(j - 1) * nks + k] = mk(0.0, 0.0);
  }
  const T ib = (T)(1.0 / b), bb = (T)b;
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    const cplx<T> r = R[base + i];
    const cplx<T> xv = X[base + i];
    const cplx<T> vp = Vp[base + i];
    rs[i] = xv * ib - vp * bb;
    Vp[base + i] = r * ib;
  }
  __syncthreads();
  const cplx<T>* uk = ukq + base;
  pair_dots<T>(uk, npw_pad, rs, npw_pad, np, nbnd, nbnd, nullptr, cf);
  __syncthreads();
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    const int v = i / npw_pad, gi = i - v * npw_pad;
    cplx<T> t = rs[i];
    for (int w = 0; w < nbnd; ++w) {
      const cplx<double> c = cf[w * nbnd + v];
      t = t - cmul(uk[(long)w * npw_pad + gi], mk((T)c.x, (T)c.y));
    }
    R[base + i] = t;
  }
}

// Non-Hermitian step j after the two operator applications XV = L v_j, XW = L^dag w_j:
// v_hat = P_c(XV - gamma_j v_{j-1}), w_hat = P_c(XW - conj(beta_j) w_{j-1}) (stored in
// XV, XW), per-k partials of s = (w_hat, v_hat) and of z_j = (y, v_j).  grid nks.
template <typename T>
__global__ void __launch_bounds__(128) k_nh_update(int j, int upper, int nks, int nbnd, int npw_pad,
                                                   const int* __restrict__ npw, cplx<T>* __restrict__ XV,
                                                   cplx<T>* __restrict__ XW, const cplx<T>* __restrict__ Vp,
                                                   const cplx<T>* __restrict__ Wp, const cplx<T>* __restrict__ Vc,
                                                   const cplx<T>* __restrict__ y, const cplx<T>* __restrict__ ukq,
                                                   Coef co, cplx<double>* __restrict__ spart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* vs = reinterpret_cast<cplx<T>*>(smem_raw);          // [nbnd][npw_pad]
  cplx<T>* ws = vs + nbnd * npw_pad;
  cplx<double>* cf = reinterpret_cast<cplx<double>*>(ws + nbnd * npw_pad);   // [2 * nbnd * nbnd]
  __shared__ double red[2][4];
  const int k = blockIdx.x;
  const long base = (long)k * nbnd * npw_pad;
  const int np = npw[k];
  const double bj = co.beta[j - 1];
  const cplx<double> gj = co.gamma[j - 1];
  const cplx<T> g = mk((T)gj.x, (T)gj.y), bc = mk((T)bj, (T)0);
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    vs[i] = XV[base + i] - cmul(g, Vp[base + i]);
    ws[i] = XW[base + i] - cmul(bc, Wp[base + i]);
  }
  __syncthreads();
  const cplx<T>* uk = ukq + base;
  pair_dots<T>(uk, npw_pad, vs, npw_pad, np, nbnd, nbnd, nullptr, cf);
  pair_dots<T>(uk, npw_pad, ws, npw_pad, np, nbnd, nbnd, nullptr, cf + nbnd * nbnd);
  __syncthreads();
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < nbnd * npw_pad; i += blockDim.x) {
    const int v = i / npw_pad, gi = i - v * npw_pad;
    cplx<T> a = vs[i], b2 = ws[i];
    for (int w = 0; w < nbnd; ++w) {
      const cplx<double> c = cf[w * nbnd + v], d = cf[nbnd * nbnd + w * nbnd + v];
      const cplx<T> u = uk[(long)w * npw_pad + gi];
      a = a - cmul(u, mk((T)c.x, (T)c.y));
      b2 = b2 - cmul(u, mk((T)d.x, (T)d.y));
    }
    XV[base + i] = a;
    XW[base + i] = b2;
    const cplx<T> t = cjmul(b2, a);
    sr += (double)t.x;
    si += (double)t.y;
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sr; red[1][threadIdx.x >> 5] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b3 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b3 += red[1][w]; }
    spart[k] = mk(a, b3);
  }
  // z_j = (y, v_j) when v_j is upper
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (upper) {
    for (int v = warp; v < nbnd; v += nw) {
      T re = 0, im = 0;
      for (int gg = lane; gg < np; gg += 32) {
        const cplx<T> t = cjmul(y[base + (long)v * npw_pad + gg], Vc[base + (long)v * npw_pad + gg]);
        re += t.x; im += t.y;
      }
      const double dr = warp_sum((double)re), di = warp_sum((double)im);
      if (lane == 0) cf[v] = mk(dr, di);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double zr = 0, zi = 0;
    if (upper) for (int v = 0; v < nbnd; ++v) { zr += cf[v].x; zi += cf[v].y; }
    co.zpart[(long)(j - 1) * nks + k] = mk(zr, zi);
  }
}

// Non-Hermitian normalisation at the end of step j: beta_{j+1} = sqrt|s|, gamma_{j+1} =
// s/beta_{j+1}; v_{j-1} <- v_j, v_j <- v_hat/beta; w_{j-1} <- w_j, w_j <- w_hat/conj(gamma).
template <typename T>
__global__ void __launch_bounds__(128) k_nh_normalize(int j, int nks, int nbnd, int npw_pad,
                                                      const cplx<double>* __restrict__ spart,
                                                      const cplx<T>* __restrict__ XV, const cplx<T>* __restrict__ XW,
                                                      cplx<T>* __restrict__ Vc, cplx<T>* __restrict__ Vp,
                                                      cplx<T>* __restrict__ Wc, cplx<T>* __restrict__ Wp, Coef co,
                                                      double tol) {
  __shared__ cplx<double> sc[2];
  const int k = blockIdx.x;
  if (threadIdx.x == 0) {
    double sr = 0, si = 0;
    for (int i = 0; i < nks; ++i) { sr += spart[i].x; si += spart[i].y; }
    sr /= nks;
    si /= nks;
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

// z_j = (1/nks) sum_k zpart[j][k] for j in [j0, j1).
static __global__ void k_reduce_z(const cplx<double>* __restrict__ zpart, int nks, int j0, int j1,
                           cplx<double>* __restrict__ z) {
  const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= j1) return;
  double zr = 0, zi = 0;
  for (int k = 0; k < nks; ++k) { zr += zpart[(long)j * nks + k].x; zi += zpart[(long)j * nks + k].y; }
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
template <typename T>
__global__ void k_gather_y(int nks, int nbnd, int npw_pad_q, int npw_pad_k, const int* __restrict__ map,
                           const cplx<T>* __restrict__ uk, cplx<T>* __restrict__ y) {
  const int k = blockIdx.x;
  for (int i = threadIdx.x; i < nbnd * npw_pad_q; i += blockDim.x) {
    const int v = i / npw_pad_q, g = i - v * npw_pad_q;
    const int m = map[(long)k * npw_pad_q + g];
    y[((long)k * nbnd + v) * npw_pad_q + g] =
        (m >= 0) ? uk[((long)k * nbnd + v) * npw_pad_k + m] : czero<T>();
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

static __global__ void k_spectrum(int m, const double* __restrict__ beta, const cplx<double>* __restrict__ gamma,
                           const cplx<double>* __restrict__ z, int nw, const double* __restrict__ w_ha, double eta,
                           double pref, double vq, cplx<double>* __restrict__ chi, cplx<double>* __restrict__ epsi,
                           cplx<double>* __restrict__ eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const cplx<double> w = mk(w_ha[i], eta);
  cplx<double> d = w, r = z[m - 1];
  for (int j = m - 2; j >= 0; --j) {
    const cplx<double> bg = cmul(mk(beta[j + 1], 0.0), gamma[j + 1]);
    const cplx<double> q = cdiv(bg, d);
    const cplx<double> rr = cdiv(mk(beta[j + 1] * r.x, beta[j + 1] * r.y), d);
    d = w - q;
    r = z[j] + rr;
  }
  const cplx<double> u1 = cdiv(r, d);
  const cplx<double> c = u1 * (pref * beta[0]);
  chi[i] = c;
  const cplx<double> ei = mk(1.0 + vq * c.x, vq * c.y);
  epsi[i] = ei;
  eps[i] = cdiv(mk(1.0, 0.0), ei);
}

}  // namespace ll
