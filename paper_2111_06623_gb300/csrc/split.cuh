// Per-k work of the pseudo-Hermitian step split over several CTAs per k-point (sm_103a).
//
// The fused per-k kernels (k_ph_update, k_zfwd_proj) hold a whole k block of two vectors,
// 2 nbnd npw complex values, in one CTA's shared memory.  Systems whose k blocks do not fit
// (the eight-atom cell: 16 bands x 1632 plane waves, 420 KB in FP32) take this path: every
// k block is cut into chunks of kChunk plane waves (for the projections) or of kLines column
// lines (for the axis-3 transforms), one CTA each, and the small dot blocks of P_c and of
// the KB projectors are formed as per-chunk partial sums that the next kernel reduces over
// the chunks in a fixed order (deterministic, no atomics).
//
// One pseudo-Hermitian step here: k_sp_start (beta_j, z_j partial, r_{j+1} before P_c,
// partial U^H r) -> k_sp_coef, k_sp_apply (P_c) -> k_zinv (axis-3 inverse FFT over several
// CTAs per k) -> planes and response
// potential as in the fused path -> k_sp_zfwd (axis-3 forward FFT, gather, kinetic - eps)
// -> k_sp_dots (partial B^H x, U^H t) -> k_sp_coef (coefficients) -> k_sp_apply (KB, P_c,
// output, norm partial).
#pragma once
#include "kernels.cuh"

namespace ll {

constexpr int kChunk = 512;    // plane waves per projection chunk
constexpr int kLines = 256;    // column lines per axis-3 CTA
constexpr int kTile = 32;      // plane waves per shared-memory tile of the dot blocks
constexpr int kTileP = kTile + 1;  // padded row of a tile (conflict-free column reads)
constexpr int kMaxPairs = 2048;  // ni * nj of one dot block (nproj <= 64, nbnd <= 32)

// sum_i p[i], i < n, by the whole block in a fixed order; every thread gets the result.
__device__ __forceinline__ double block_sum(const double* p, int n) {
  __shared__ double wsum[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
  __syncthreads();
  return t;
}

// out[i*nj + j] = sum_{g0 <= g < g1} conj(A[i*lda + g]) B[j*ldb + g] for all ni x nj pairs.
// Each thread owns up to kMaxPairs/blockDim pairs; the plane waves stream through shared
// memory in tiles of kTile, each tile summed in T and added to a double accumulator.
// `tile`: (ni + nj) * kTileP complex T of shared memory.  Called by the whole block.
template <typename T>
__device__ void chunk_dots(const cplx<T>* A, long lda, const cplx<T>* B, long ldb, int g0, int g1, int ni, int nj,
                           cplx<T>* tile, cplx<double>* out) {
  constexpr int PPT = kMaxPairs / 256;
  const int np = ni * nj;
  double ar[PPT], ai[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) ar[q] = ai[q] = 0.0;
  cplx<T>* At = tile;
  cplx<T>* Bt = tile + ni * kTileP;
  for (int t0 = g0; t0 < g1; t0 += kTile) {
    const int nt = min(kTile, g1 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < (ni + nj) * kTile; e += blockDim.x) {
      const int row = e / kTile, g = e - row * kTile;
      cplx<T> v = czero<T>();
      if (g < nt) v = row < ni ? A[(long)row * lda + t0 + g] : B[(long)(row - ni) * ldb + t0 + g];
      tile[row * kTileP + g] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int pr = threadIdx.x + q * blockDim.x;
      if (pr < np) {
        const int i = pr / nj, j = pr - i * nj;
        T sr = T(0), si = T(0);
        for (int g = 0; g < kTile; ++g) {
          const cplx<T> a = At[i * kTileP + g], b = Bt[j * kTileP + g];
          sr += a.x * b.x + a.y * b.y;
          si += a.x * b.y - a.y * b.x;
        }
        ar[q] += (double)sr;
        ai[q] += (double)si;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int pr = threadIdx.x + q * blockDim.x;
    if (pr < np) out[pr] = mk(ar[q], ai[q]);
  }
  __syncthreads();
}

// Step j, first part: beta_j = sqrt((1/nks) sum of the norm partials), the z_j partial of
// the chunk, r_{j+1} = X_j/beta_j - beta_j v_{j-1} into R, v_j = r_j/beta_j into Vp, and the
// chunk's partial U^H r_{j+1}.  grid (nks, nchunk), block 256.
template <typename T>
__global__ void __launch_bounds__(256) k_sp_start(const int* __restrict__ jdev, int nks, int nbnd, int npw_pad,
                                                  const int* __restrict__ npw, int nchunk,
                                                  const double* __restrict__ part, cplx<T>* __restrict__ R,
                                                  const cplx<T>* __restrict__ X, cplx<T>* __restrict__ Vp,
                                                  const cplx<T>* __restrict__ y, const cplx<T>* __restrict__ ukq,
                                                  Coef co, double tol, cplx<double>* __restrict__ spart,
                                                  int dots) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = *jdev, r_upper = (j % 2 == 0) ? 1 : 0;   // step index from the device counter
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw);
  __shared__ double sbeta;
  __shared__ double zred[2][8];
  const int k = blockIdx.x, c = blockIdx.y;
  const int g0 = c * kChunk, g1 = min(npw_pad, g0 + kChunk);
  const double b2 = block_sum(part, nks * nchunk) / nks;
  if (threadIdx.x == 0) {
    double b = 1.0;
    if (!(b2 > tol)) flag_error(co.err, b2 <= 0.0 ? DEV_NOTPD : DEV_BREAKDOWN, j);
    else b = sqrt(b2);
    sbeta = b;
    if (k == 0 && c == 0) { co.beta[j - 1] = b; co.gamma[j - 1] = mk(b, 0.0); }
  }
  __syncthreads();
  const double b = sbeta;
  const long base = (long)k * nbnd * npw_pad;
  const int zi = (j - 1) * nks * nchunk + k * nchunk + c;
  if (r_upper) {  // z_j partial = (y, r_j)/beta_j over the chunk
    double zr = 0.0, zim = 0.0;
    for (int e = threadIdx.x; e < nbnd * (g1 - g0); e += blockDim.x) {
      const int v = e / (g1 - g0), g = g0 + e - v * (g1 - g0);
      const cplx<T> a = y[base + (long)v * npw_pad + g], r = R[base + (long)v * npw_pad + g];
      zr += (double)(a.x * r.x + a.y * r.y);
      zim += (double)(a.x * r.y - a.y * r.x);
    }
    zr = warp_sum(zr);
    zim = warp_sum(zim);
    if ((threadIdx.x & 31) == 0) { zred[0][threadIdx.x >> 5] = zr; zred[1][threadIdx.x >> 5] = zim; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += zred[0][w]; si += zred[1][w]; }
      co.zpart[zi] = mk(sr / b, si / b);
    }
  } else if (threadIdx.x == 0) {
    co.zpart[zi] = mk(0.0, 0.0);
  }
  __syncthreads();
  const T ib = (T)(1.0 / b), bb = (T)b;
  for (int e = threadIdx.x; e < nbnd * (g1 - g0); e += blockDim.x) {
    const int v = e / (g1 - g0), g = g0 + e - v * (g1 - g0);
    const long i = base + (long)v * npw_pad + g;
    const cplx<T> r = R[i];
    R[i] = X[i] * ib - Vp[i] * bb;
    Vp[i] = r * ib;
  }
  if (!dots) return;   // the partial U^H r_{j+1} comes from the tensor-core kernel
  __syncthreads();
  chunk_dots<T>(ukq + base, npw_pad, R + base, npw_pad, g0, max(g0, min(g1, npw[k])), nbnd, nbnd, tile,
                spart + ((long)k * nchunk + c) * nbnd * nbnd);
}

// Operator, last stage, first part: forward FFT of the columns along axis 3, gather of the
// sphere (1/N^3) plus (1/2|k+Q+G|^2 - eps_vk) x into t = out.  grid (nks, nvec, lines).
template <typename T, int N>
__global__ void __launch_bounds__(kLines) k_sp_zfwd(SphereDev s, int nbnd, const cplx<T>* __restrict__ cbuf,
                                                    int cb_ncol, const cplx<T>* __restrict__ xin,
                                                    const T* __restrict__ kin, const double* __restrict__ eps,
                                                    cplx<T>* __restrict__ xout) {
  const int k = blockIdx.x, vec = blockIdx.y, nks = s.nks, npw_pad = s.npw_pad;
  const int nc = s.ncol[k];
  const int it = blockIdx.z * kLines + threadIdx.x;
  if (it >= nbnd * nc) return;
  const int v = it / nc, c = it - v * nc;
  const long o = ((long)vec * nks + k) * nbnd + v;
  const int4 cl = s.col[k * s.ncol_max + c];
  if (!LL_INB(c < cb_ncol)) return;
  const cplx<T>* src = cbuf + o * (long)N * cb_ncol + c;
  cplx<T> a[N];
#pragma unroll
  for (int p = 0; p < N; ++p) a[p] = src[(long)p * cb_ncol];
  fft_line<T, N, -1>(a);
  const T scale = T(1) / T(N * N * N);
  const T ev = (T)eps[k * nbnd + v];
  const int st = s.colstart[k * s.ncol_max + c];
  const cplx<T>* x = xin + o * npw_pad + st;
  const T* kn = kin + (long)k * npw_pad + st;
  cplx<T>* t = xout + o * npw_pad + st;
#pragma unroll
  for (int p = 0; p < N; ++p) {
    const int i = wrapn<N>(p - cl.z);
    if (i < cl.w && LL_INB(st >= 0 && st + i < npw_pad)) t[i] = x[i] * (kn[i] - ev) + a[p] * scale;
  }
}

// Partial dot blocks of one chunk: C = B^H x (nproj x nbnd, when nproj > 0) and
// S1 = U^H t (nbnd x nbnd).  grid (nks, nvec, nchunk), block 256.
template <typename T>
__global__ void __launch_bounds__(256) k_sp_dots(int nks, int nbnd, int npw_pad, const int* __restrict__ npw,
                                                 int nchunk, int nproj,
                                                 const cplx<T>* __restrict__ xin, const cplx<T>* __restrict__ t,
                                                 const cplx<T>* __restrict__ ukq, const cplx<T>* __restrict__ bkq,
                                                 cplx<double>* __restrict__ cpart, cplx<double>* __restrict__ spart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw);
  const int k = blockIdx.x, vec = blockIdx.y, c = blockIdx.z;
  const int g0 = c * kChunk, g1 = max(g0, min(npw[k], g0 + kChunk));   // sphere points only
  const long kv = (long)vec * nks + k;
  const long base = kv * nbnd * npw_pad;
  if (nproj > 0)
    chunk_dots<T>(bkq + (long)k * nproj * npw_pad, npw_pad, xin + base, npw_pad, g0, g1, nproj, nbnd, tile,
                  cpart + (kv * nchunk + c) * nproj * nbnd);
  chunk_dots<T>(ukq + (long)k * nbnd * npw_pad, npw_pad, t + base, npw_pad, g0, g1, nbnd, nbnd, tile,
                spart + (kv * nchunk + c) * nbnd * nbnd);
}

// Operator, last stage: the coefficients of one (vector, k), reduced over the chunks in a fixed
// order: c = D o (B^H x) (nproj x nbnd) and S = U^H t + (U^H B) c (nbnd x nbnd), rounded to T
// into coef[kv] = [c | S].  ub: U^H B per k, [nbnd][nproj] (double).  A metal (MetalDev,
// kernels.cuh) turns S into the coefficients of its projections: kind 1 (the operator) sp S - da
// Z with Z = zp[kv] from the image, and mcorr[kv] = sum qh Re(conj(Z) (S - C)), the term that
// makes the norm partial of the image Re(z, X); kind 2 (the update) keep S; kind 3 (the image
// Q z, S = U^H z) qh S, with zp[kv] = S on the kept states.  kind 0: S itself.
// grid nks * nvec, block 256.
template <typename T>
__global__ void __launch_bounds__(256) k_sp_coef(int nks, int nbnd, int nchunk, int nproj,
                                                 const double* __restrict__ dij, const cplx<double>* __restrict__ ub,
                                                 const cplx<double>* __restrict__ cpart,
                                                 const cplx<double>* __restrict__ spart, cplx<T>* __restrict__ coef,
                                                 int kind = 0, MetalDev md = MetalDev{nullptr, nullptr, nullptr, nullptr},
                                                 cplx<double>* __restrict__ zp = nullptr,
                                                 double* __restrict__ mcorr = nullptr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<double>* cd = reinterpret_cast<cplx<double>*>(smem_raw);   // [nproj * nbnd]
  const long kv = blockIdx.x;
  const int k = (int)(kv % nks);
  cplx<T>* out = coef + kv * (long)(nproj + nbnd) * nbnd;
  for (int p = threadIdx.x; p < nproj * nbnd; p += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int cc = 0; cc < nchunk; ++cc) {
      re += cpart[(kv * nchunk + cc) * nproj * nbnd + p].x;
      im += cpart[(kv * nchunk + cc) * nproj * nbnd + p].y;
    }
    const double m = dij[p / nbnd];
    cd[p] = mk(re * m, im * m);
    out[p] = mk((T)(re * m), (T)(im * m));
  }
  __syncthreads();
  double corr = 0.0;
  for (int p = threadIdx.x; p < nbnd * nbnd; p += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int cc = 0; cc < nchunk; ++cc) {
      re += spart[(kv * nchunk + cc) * nbnd * nbnd + p].x;
      im += spart[(kv * nchunk + cc) * nbnd * nbnd + p].y;
    }
    const int w = p / nbnd, v = p - w * nbnd;
    for (int q = 0; q < nproj; ++q) {
      const cplx<double> a = ub[((long)k * nbnd + w) * nproj + q], d = cd[q * nbnd + v];
      re += a.x * d.x - a.y * d.y;
      im += a.x * d.y + a.y * d.x;
    }
    if (kind == 1) {
      const long mi = ((long)k * nbnd + w) * nbnd + v;
      const cplx<double> z = zp[kv * nbnd * nbnd + p];
      const double cr = md.sp[mi] * re - md.da[mi] * z.x, ci = md.sp[mi] * im - md.da[mi] * z.y;
      corr += md.qh[mi] * (z.x * (re - cr) + z.y * (im - ci));
      re = cr;
      im = ci;
    } else if (kind == 2) {
      const double kp = md.keep[((long)k * nbnd + w) * nbnd + v];
      re *= kp;
      im *= kp;
    } else if (kind == 3) {
      const long mi = ((long)k * nbnd + w) * nbnd + v;
      const double kept = md.keep[mi] == 0.0 ? 1.0 : 0.0, q = md.qh[mi];
      zp[kv * nbnd * nbnd + p] = mk(re * kept, im * kept);
      re *= q;
      im *= q;
    }
    out[nproj * nbnd + p] = mk((T)re, (T)im);
  }
  if (kind == 1) {
    corr = block_sum(corr);
    if (threadIdx.x == 0) mcorr[kv] = corr;
  }
}

// A metal's term of the norm partial (k_sp_coef, kind 1) added to the first chunk's partial of
// each (vector, k).  grid 1, block 256.
static __global__ void k_sp_addcorr(int nkv, int nchunk, const double* __restrict__ mcorr, double* __restrict__ part) {
  for (int kv = threadIdx.x; kv < nkv; kv += blockDim.x) part[(long)kv * nchunk] += mcorr[kv];
}

// Operator, last stage, applied: t <- t + B c - U S (= P_c (t + B c)) on one chunk of plane
// waves of one (vector, k), zero on the padding, and the chunk's partial Re(x^H t).  The chunk
// is walked in sub-tiles of kSub plane waves: the sub-tile's projector and occupied-state
// values (nproj + nbnd rows) are staged in shared memory once and serve every band, so each
// is read from L2 once per chunk instead of once per band.  Thread t takes plane wave
// t % kSub of the sub-tile and bands t / kSub, t / kSub + 256 / kSub, ...
// grid (nks, nvec, nchunk), block 256; dynamic smem (nproj + nbnd) (kSub + nbnd) complex T.
constexpr int kSub = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_sp_apply(int nks, int nbnd, int npw_pad, const int* __restrict__ npw,
                                                  int nchunk, int nproj, const cplx<T>* __restrict__ xin,
                                                  cplx<T>* __restrict__ t, const cplx<T>* __restrict__ ukq,
                                                  const cplx<T>* __restrict__ bkq, const cplx<T>* __restrict__ coef,
                                                  double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int VS = 256 / kSub;                                   // band strides per sub-tile
  cplx<T>* Ct = reinterpret_cast<cplx<T>*>(smem_raw);             // [nproj][nbnd] then [nbnd][nbnd]
  cplx<T>* Bt = Ct + (nproj + nbnd) * nbnd;                        // [nproj][kSub] then [nbnd][kSub]
  __shared__ double wred[8];
  const int k = blockIdx.x, vec = blockIdx.y, c = blockIdx.z;
  const long kv = (long)vec * nks + k;
  const int np = npw[k];
  const int g0 = c * kChunk, g1 = min(npw_pad, g0 + kChunk);
  const int nrow = nproj + nbnd;
  const cplx<T>* cf = coef + kv * (long)nrow * nbnd;
  for (int i = threadIdx.x; i < nrow * nbnd; i += blockDim.x) Ct[i] = cf[i];
  const long base = kv * nbnd * npw_pad;
  const cplx<T>* uk = ukq + (long)k * nbnd * npw_pad;
  const cplx<T>* bk = bkq + (long)k * nproj * npw_pad;
  const int gl = threadIdx.x % kSub, vb = threadIdx.x / kSub;
  double nr = 0.0;
  for (int s0 = g0; s0 < g1; s0 += kSub) {
    __syncthreads();
    for (int e = threadIdx.x; e < nrow * kSub; e += blockDim.x) {
      const int row = e / kSub, g = s0 + e - row * kSub;
      cplx<T> v = czero<T>();
      if (g < g1) v = row < nproj ? bk[(long)row * npw_pad + g] : uk[(long)(row - nproj) * npw_pad + g];
      Bt[e] = v;
    }
    __syncthreads();
    const int g = s0 + gl;
    if (g < g1) {
      for (int v = vb; v < nbnd; v += VS) {
        const long i = base + (long)v * npw_pad + g;
        cplx<T> acc = czero<T>();
        if (g < np) {
          acc = t[i];
          for (int q = 0; q < nproj; ++q) acc = acc + cmul(Bt[q * kSub + gl], Ct[q * nbnd + v]);
          for (int w = 0; w < nbnd; ++w) acc = acc - cmul(Bt[(nproj + w) * kSub + gl], Ct[(nproj + w) * nbnd + v]);
          if (part) {
            const cplx<T> x = xin[i];
            nr += (double)(x.x * acc.x + x.y * acc.y);
          }
        }
        t[i] = acc;
      }
    }
  }
  if (!part) return;   // the projection of the update step: no norm
  nr = warp_sum(nr);
  if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = nr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += wred[w];
    part[kv * nchunk + c] = sum;
  }
}

// Set-up: partial U^H B per (k, chunk).  grid (nks, nchunk), block 256.
template <typename T>
__global__ void __launch_bounds__(256) k_sp_ub(int nbnd, int npw_pad, const int* __restrict__ npw, int nchunk,
                                               int nproj, const cplx<T>* __restrict__ ukq,
                                               const cplx<T>* __restrict__ bkq, cplx<double>* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw);
  const int k = blockIdx.x, c = blockIdx.y;
  const int g0 = c * kChunk, g1 = max(g0, min(npw[k], g0 + kChunk));
  chunk_dots<T>(ukq + (long)k * nbnd * npw_pad, npw_pad, bkq + (long)k * nproj * npw_pad, npw_pad, g0, g1, nbnd,
                nproj, tile, part + ((long)k * nchunk + c) * nbnd * nproj);
}

// Set-up: U^H B per k from the chunk partials (double).  grid nks, block 256.
static __global__ void k_sp_reduce(int nchunk, int np, const cplx<double>* __restrict__ part,
                                   cplx<double>* __restrict__ out) {
  const int k = blockIdx.x;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      re += part[((long)k * nchunk + c) * np + p].x;
      im += part[((long)k * nchunk + c) * np + p].y;
    }
    out[(long)k * np + p] = mk(re, im);
  }
}

// Non-Hermitian step j on the split path, first part (the fused k_nh_update cut in two):
// z_j partial = (y, v_j) over the chunk, v_hat = XV - gamma_j v_{j-1} and w_hat = XW -
// beta_j w_{j-1} in place, and the chunk's partials of U^H v_hat, U^H w_hat.
// grid (nks, nchunk), block 256; dynamic smem 2 nbnd kTileP complex T.
template <typename T>
__global__ void __launch_bounds__(256) k_sp_nh_start(int j, int upper, int nks, int nbnd, int npw_pad,
                                                     const int* __restrict__ npw, int nchunk, cplx<T>* __restrict__ XV,
                                                     cplx<T>* __restrict__ XW, const cplx<T>* __restrict__ Vp,
                                                     const cplx<T>* __restrict__ Wp, const cplx<T>* __restrict__ Vc,
                                                     const cplx<T>* __restrict__ y, const cplx<T>* __restrict__ ukq,
                                                     Coef co, cplx<double>* __restrict__ spart2, int dots) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw);
  __shared__ double zred[2][8];
  const int k = blockIdx.x, c = blockIdx.y;
  const int g0 = c * kChunk, g1 = min(npw_pad, g0 + kChunk), n = g1 - g0;
  const long base = (long)k * nbnd * npw_pad;
  const int zi = (j - 1) * nks * nchunk + k * nchunk + c;
  if (upper) {  // z_j partial = (y, v_j) over the chunk
    double zr = 0.0, zim = 0.0;
    for (int e = threadIdx.x; e < nbnd * n; e += blockDim.x) {
      const int v = e / n;
      const long i = base + (long)v * npw_pad + g0 + e - v * n;
      const cplx<T> a = y[i], r = Vc[i];
      zr += (double)(a.x * r.x + a.y * r.y);
      zim += (double)(a.x * r.y - a.y * r.x);
    }
    zr = warp_sum(zr);
    zim = warp_sum(zim);
    if ((threadIdx.x & 31) == 0) { zred[0][threadIdx.x >> 5] = zr; zred[1][threadIdx.x >> 5] = zim; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += zred[0][w]; si += zred[1][w]; }
      co.zpart[zi] = mk(sr, si);
    }
  } else if (threadIdx.x == 0) {
    co.zpart[zi] = mk(0.0, 0.0);
  }
  const double bj = co.beta[j - 1];
  const cplx<double> gj = co.gamma[j - 1];
  const cplx<T> g = mk((T)gj.x, (T)gj.y), bc = mk((T)bj, (T)0);
  for (int e = threadIdx.x; e < nbnd * n; e += blockDim.x) {
    const int v = e / n;
    const long i = base + (long)v * npw_pad + g0 + e - v * n;
    XV[i] = XV[i] - cmul(g, Vp[i]);
    XW[i] = XW[i] - cmul(bc, Wp[i]);
  }
  if (!dots) return;   // the partials U^H v_hat, U^H w_hat come from the tensor-core kernel
  __syncthreads();
  const int ge = max(g0, min(g1, npw[k]));
  cplx<double>* out = spart2 + ((long)k * nchunk + c) * 2 * nbnd * nbnd;
  chunk_dots<T>(ukq + base, npw_pad, XV + base, npw_pad, g0, ge, nbnd, nbnd, tile, out);
  chunk_dots<T>(ukq + base, npw_pad, XW + base, npw_pad, g0, ge, nbnd, nbnd, tile, out + nbnd * nbnd);
}

// Second part: P_c on v_hat and w_hat with the coefficients reduced over the chunks (fixed
// order), and the chunk's partial s = (w_hat, v_hat).  grid (nks, nchunk), block 256.
template <typename T>
__global__ void __launch_bounds__(256) k_sp_nh_proj(int nks, int nbnd, int npw_pad, const int* __restrict__ npw,
                                                    int nchunk, cplx<T>* __restrict__ XV, cplx<T>* __restrict__ XW,
                                                    const cplx<T>* __restrict__ ukq,
                                                    const cplx<double>* __restrict__ spart2,
                                                    cplx<double>* __restrict__ spart,
                                                    const double* __restrict__ keep = nullptr) {
  __shared__ cplx<T> Sv[32 * 32], Sw[32 * 32];
  __shared__ double sred[2][8];
  const int k = blockIdx.x, c = blockIdx.y;
  const int nn = nbnd * nbnd;
  for (int p = threadIdx.x; p < nn; p += blockDim.x) {
    double vr = 0.0, vi = 0.0, wr = 0.0, wi = 0.0;
    for (int cc = 0; cc < nchunk; ++cc) {
      const cplx<double>* q = spart2 + ((long)k * nchunk + cc) * 2 * nn;
      vr += q[p].x; vi += q[p].y;
      wr += q[nn + p].x; wi += q[nn + p].y;
    }
    const double kp = keep ? keep[(long)k * nn + p] : 1.0;   // a metal: P'_v
    Sv[p] = mk((T)(vr * kp), (T)(vi * kp));
    Sw[p] = mk((T)(wr * kp), (T)(wi * kp));
  }
  __syncthreads();
  const int g0 = c * kChunk, g1 = min(npw_pad, g0 + kChunk), n = g1 - g0;
  const int np = npw[k];
  const long base = (long)k * nbnd * npw_pad;
  const cplx<T>* uk = ukq + base;
  double sr = 0.0, si = 0.0;
  for (int e = threadIdx.x; e < nbnd * n; e += blockDim.x) {
    const int v = e / n, g = g0 + e - v * n;
    const long i = base + (long)v * npw_pad + g;
    cplx<T> a = XV[i], b = XW[i];
    for (int w = 0; w < nbnd; ++w) {
      const cplx<T> u = uk[(long)w * npw_pad + g];
      a = a - cmul(u, Sv[w * nbnd + v]);
      b = b - cmul(u, Sw[w * nbnd + v]);
    }
    XV[i] = a;
    XW[i] = b;
    if (g < np) {
      sr += (double)(b.x * a.x + b.y * a.y);
      si += (double)(b.x * a.y - b.y * a.x);
    }
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  if ((threadIdx.x & 31) == 0) { sred[0][threadIdx.x >> 5] = sr; sred[1][threadIdx.x >> 5] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sred[0][w]; b += sred[1][w]; }
    spart[(long)k * nchunk + c] = mk(a, b);
  }
}

}  // namespace ll
