// The per-plane pass of k_xy (kernels.cuh) with every line transform split over a lane pair
// (fft_pair_dit / fft_pair_dif, fft.cuh): each lane holds half a line, so the pass needs about
// half the registers per thread and fits twice the warps per SM.  Same modes, same shared-
// memory layout, same results up to rounding order; blocks of 4N threads (two slots of N
// lane pairs for the axis-2 lines), even N only.
//
// Layouts per pair (h = lane & 1, H = N/2):
//   rows inverse   in: m1 = 2m + h (gathered from the columns)  out: j1 = H h + m
//   lines inverse  in: m2 = 2m + h (gathered from the rows)     out: j2 = H h + m
//   real space     V, v', u, the density at (j2 = H h + m, j1)
//   lines forward  in: j2 = H h + m                             out: m2 = 2m + h -> rows
//   rows forward   in: j1 = H h + m                             out: m1 = 2m + h -> columns
#pragma once
#include "kernels.cuh"

namespace ll {

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(4 * N, (sizeof(T) == 4 ? (N > 36 ? 3 : 4) : 2)) k_xyp(XYArgs a, cplx<T>* __restrict__ cbuf,
                                                                const T* __restrict__ vloc,
                                                                const cplx<T>* __restrict__ vpr,
                                                                const cplx<T>* __restrict__ ur,
                                                                cplx<T>* __restrict__ nprt,
                                                                cplx<T>* __restrict__ grid_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int H = N / 2;
  constexpr int NP = N + 1;
  constexpr int NN = N * N;
  constexpr int S = 2;                                                  // line slots
  const int iz = blockIdx.x, g = blockIdx.y;
  const int BO = a.bo;
  const SphereDev& s = a.s;
  cplx<T>* Cs = reinterpret_cast<cplx<T>*>(smem_raw);                 // [BO][cb_ncol]
  cplx<T>* Ys = Cs + BO * a.cb_ncol;                                    // [BO][nrow_max][NP]
  cplx<T>* Pl = Ys + BO * s.nrow_max * NP;                              // [N][N] v' (pass 2)
  cplx<T>* Pb = Pl + (MODE == XY_PASS2 ? NN : 0);                       // [S][N][N] density
  T* Pv = reinterpret_cast<T*>(Pb + (MODE == XY_PASS1_DENS ? S * NN : 0));  // [N][N] V (real)
  const long plane = (long)NN;
  const int lane = threadIdx.x & 31, h = threadIdx.x & 1, pr = threadIdx.x >> 1;
  const unsigned pmask = 3u << (lane & 30);                             // this lane pair
  const int ls = pr / N, lj1 = pr - ls * N;                             // line slot, column

  if (MODE == XY_PASS1 || MODE == XY_PASS1_DENS) {
    for (int i = threadIdx.x; i < NN; i += blockDim.x) Pv[i] = vloc[iz * plane + i];
  } else if (MODE == XY_PASS2) {
    for (int i = threadIdx.x; i < NN; i += blockDim.x) Pl[i] = vpr[iz * plane + i];
  }
  if (MODE == XY_PASS1_DENS)
    for (int i = threadIdx.x; i < S * NN; i += blockDim.x) Pb[i] = czero<T>();

  const int o_begin = a.o_off + g * a.per_group;
  const int o_end = a.o_off + min(a.norb, g * a.per_group + a.per_group);
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
      // inverse FFT along axis 1 of every sphere row, one lane pair per row
      for (int i = pr; i < nb * s.nrow_max; i += blockDim.x / 2) {
        const int b = a.f_nrow.div(i), r = i - b * s.nrow_max;
        const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
        if (r >= s.nrow[k]) continue;                 // both lanes of the pair alike
        const int4 rw = s.row[k * s.nrow_max + r];
        cplx<T> l[H];
        const cplx<T>* cs = Cs + b * a.cb_ncol + rw.y;
#pragma unroll
        for (int m = 0; m < H; ++m) {
          const int j = wrapn<N>(2 * m + h - rw.z);
          l[m] = (j < rw.w && LL_INB(rw.y >= 0 && rw.y + j < a.cb_ncol)) ? cs[j] : czero<T>();
        }
        fft_pair_dit<T, H, +1>(l, h, pmask);
        cplx<T>* ys = Ys + (b * s.nrow_max + r) * NP + H * h;
#pragma unroll
        for (int m = 0; m < H; ++m) ys[m] = l[m];
      }
      __syncthreads();
    }
    // axis 2: one lane pair per (orbital, j1); lane h holds j2 = H h + m after the inverse
#pragma unroll 1
    for (int b = ls; ls < S && b < nb; b += S) {
      const int j1 = lj1;
      const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
      const int nr = s.nrow[k];
      const int m2min = s.row[k * s.nrow_max].x;
      cplx<T> l[H];
      if (MODE == XY_PASS2) {
        const cplx<T>* u = ur + (long)a.f_pervec.mod(o) * N * plane + iz * plane + j1;
#pragma unroll
        for (int m = 0; m < H; ++m) {
          const int j2 = H * h + m;
          l[m] = cmul(Pl[j2 * N + j1], u[j2 * N]);
        }
      } else {
#pragma unroll
        for (int m = 0; m < H; ++m) {
          const int r = wrapn<N>(2 * m + h - m2min);
          l[m] = (r < nr && LL_INB(r < s.nrow_max)) ? Ys[(b * s.nrow_max + r) * NP + j1] : czero<T>();
        }
        fft_pair_dit<T, H, +1>(l, h, pmask);
        if (MODE == XY_STORE) {
          cplx<T>* dst = grid_out + (long)o * N * plane + iz * plane + j1;
#pragma unroll
          for (int m = 0; m < H; ++m) dst[(H * h + m) * N] = l[m];
          continue;
        }
        if (MODE == XY_PASS1_DENS && a.f_pervec.div(o) == a.dens_vec) {
          const cplx<T>* u = ur + (long)a.f_pervec.mod(o) * N * plane + iz * plane + j1;
          cplx<T>* pb = Pb + ls * NN + j1;
#pragma unroll
          for (int m = 0; m < H; ++m) {
            const int j2 = H * h + m;
            pb[j2 * N] = pb[j2 * N] + cjmul(u[j2 * N], l[m]);
          }
        }
#pragma unroll
        for (int m = 0; m < H; ++m) l[m] = l[m] * Pv[(H * h + m) * N + j1];
      }
      fft_pair_dif<T, H, -1>(l, h, pmask);
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int r = wrapn<N>(2 * m + h - m2min);
        if (r < nr && LL_INB(r < s.nrow_max)) Ys[(b * s.nrow_max + r) * NP + j1] = l[m];
      }
    }
    __syncthreads();
    if (MODE == XY_STORE) continue;
    // forward FFT along axis 1 of every row, keep the row's columns
    for (int i = pr; i < nb * s.nrow_max; i += blockDim.x / 2) {
      const int b = a.f_nrow.div(i), r = i - b * s.nrow_max;
      const int o = ob + b, k = a.f_nks.mod(a.f_nbnd.div(o));
      if (r >= s.nrow[k]) continue;
      const int4 rw = s.row[k * s.nrow_max + r];
      cplx<T> l[H];
      const cplx<T>* ys = Ys + (b * s.nrow_max + r) * NP + H * h;
#pragma unroll
      for (int m = 0; m < H; ++m) l[m] = ys[m];
      fft_pair_dif<T, H, -1>(l, h, pmask);
      cplx<T>* cs = Cs + b * a.cb_ncol + rw.y;
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int j = wrapn<N>(2 * m + h - rw.z);
        if (j < rw.w && LL_INB(rw.y >= 0 && rw.y + j < a.cb_ncol)) cs[j] = l[m];
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

}  // namespace ll
