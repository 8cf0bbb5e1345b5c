// The projections of the split per-k path on the tensor cores (FP32 path, sm_103a).
//
// The dot blocks of P_c (Eq. 16) and of the Kleinman-Bylander projectors, S = U^H t and
// C = B^H x over the plane waves of one chunk, are one real matrix product per CTA:
//
//   D = A Bop^T,  A and Bop rows = complex rows viewed as interleaved real vectors of length
//   2 npw (K), so that for complex rows a, b
//     a . b          = sum_g (a_r b_r + a_i b_i)  = Re(conj(a) b)
//     a . swap(b)    = sum_g (a_r b_i - a_i b_r)  = Im(conj(a) b),   swap(b) = (b_i, -b_r)
//
// Every FP32 value is split into three BF16 parts (hi + mid + lo, tc.cuh) and the six
// products hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid are accumulated in FP32 in tensor
// memory: FP32 accuracy (the dropped products are below 2^-24 of the terms).
//
// Row assignment (M = 128 rows of A, N = nb rows of Bop, nb a multiple of 32):
//   TC_OP  (operator output):  A = [B (nproj) | t | swap(t)],  Bop = [x | swap(x) | U]
//          C[p][v] = (D[p][v], D[p][nbnd+v]),  S[w][v] = (D[nproj+v][2nbnd+w], D[nproj+nbnd+v][2nbnd+w])
//   TC_U   (update, P_c):      A = [r | swap(r)],               Bop = [U]
//          S[w][v] = (D[v][w], D[nbnd+v][w])
//   TC_U2  (non-Hermitian):    A = [v | swap(v) | w | swap(w)], Bop = [U]
// The chunk partials (cplx<double>, the layout of the CUDA-core chunk_dots) are reduced over
// the chunks in a fixed order by k_sp_coef / k_sp_nh_proj, as before.
//
// Pipeline: the FP32 rows stream into a ring of kTcRaw stages of kTcPw plane waves in shared
// memory (cp.async, two stages ahead), so that HBM stays busy while a stage is split into the
// BF16 tiles; one elected thread issues the MMAs and commits them to an mbarrier that the CTA
// waits on (bounded) before it overwrites the tiles.
#pragma once
#include "split.cuh"
#include "tc.cuh"

namespace ll {

constexpr int kTcKs = 2;              // K steps (16 real values = 8 plane waves) per stage
constexpr int kTcPw = 8 * kTcKs;      // plane waves per stage
constexpr int kTcF4 = kTcPw / 2;      // 16-byte pieces (two complex values) per row and stage
constexpr int kTcMaxRows = 192;       // source rows of one CTA at most
constexpr int kTcMaxF4 = (kTcMaxRows * kTcF4 + 255) / 256;   // pieces per thread and stage
constexpr int kTcThreads = 256;
constexpr int kTcATile = 128 * 32;    // bytes of one K step of A (128 rows)
constexpr int kTcRaw = 3;             // FP32 stages in flight (cp.async ring)
constexpr int kTcRawRow = kTcPw * 8 + 16;   // bytes of one source row of a raw stage (padded)

enum TcMode { TC_OP = 0, TC_U = 1, TC_U2 = 2 };

struct TcDotsArgs {
  int nks, nbnd, npw_pad, nchunk, nproj, nb;
  const int* npw;
  const float4* x;      // operator input (TC_OP)
  const float4* t;      // operator output (TC_OP), r (TC_U), v_hat (TC_U2)
  const float4* t2;     // w_hat (TC_U2)
  const float4* ukq;
  const float4* bkq;
  cplx<double>* cpart;
  cplx<double>* spart;
  int* err;
  const int* jdev;
};

template <int MODE>
__host__ __device__ __forceinline__ int tc_nsrc(int nbnd, int nproj) {
  return MODE == TC_OP ? nproj + 3 * nbnd : (MODE == TC_U ? 2 * nbnd : 3 * nbnd);
}

// Shared memory of k_tc_dots: the FP32 ring (kTcRaw stages of the CTA's source rows, rows
// padded to kTcRawRow bytes) and three BF16 levels of kTcKs K steps of [A tile | Bop tile].
__host__ __device__ inline size_t tc_dots_raw_bytes(int nsrc) {
  return (size_t)kTcRaw * ((nsrc + 7) / 8 * 8) * kTcRawRow;
}
__host__ __device__ inline size_t tc_dots_smem(int nb, int nsrc) {
  return tc_dots_raw_bytes(nsrc) + (size_t)3 * kTcKs * (kTcATile + 32 * nb);
}

// Source row s of the CTA's unique rows: its global row (in 16-byte units of npw_pad/2) and
// where it goes: A row (or -1), A row of its swap (or -1), Bop row, Bop row of its swap.
template <int MODE>
__device__ __forceinline__ const float4* tc_src(const TcDotsArgs& a, int k, long kv, int s, int& da, int& das,
                                                int& db, int& dbs) {
  const int nb = a.nbnd, np = a.nproj;
  const long h = a.npw_pad / 2;
  da = das = db = dbs = -1;
  if (MODE == TC_OP) {
    if (s < np) { da = s; return a.bkq + ((long)k * np + s) * h; }
    s -= np;
    if (s < nb) { da = np + s; das = np + nb + s; return a.t + (kv * nb + s) * h; }
    s -= nb;
    if (s < nb) { db = s; dbs = nb + s; return a.x + (kv * nb + s) * h; }
    s -= nb;
    db = 2 * nb + s;
    return a.ukq + ((long)k * nb + s) * h;
  } else if (MODE == TC_U) {
    if (s < nb) { da = s; das = nb + s; return a.t + ((long)k * nb + s) * h; }
    s -= nb;
    db = s;
    return a.ukq + ((long)k * nb + s) * h;
  } else {
    if (s < nb) { da = s; das = nb + s; return a.t + ((long)k * nb + s) * h; }
    s -= nb;
    if (s < nb) { da = 2 * nb + s; das = 3 * nb + s; return a.t2 + ((long)k * nb + s) * h; }
    s -= nb;
    db = s;
    return a.ukq + ((long)k * nb + s) * h;
  }
}

// 16-byte global -> shared copy; bytes < 16 copies that many and zero-fills the rest.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint2 pack_bf16x4(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c, __nv_bfloat16 d) {
  uint2 r;
  r.x = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
  r.y = (uint32_t)__bfloat16_as_ushort(c) | ((uint32_t)__bfloat16_as_ushort(d) << 16);
  return r;
}

// Split four FP32 values into the three BF16 levels, packed four to eight bytes.
__device__ __forceinline__ void split4(float4 v, uint2& hi, uint2& mid, uint2& lo) {
  __nv_bfloat16 h[4], m[4], l[4];
  bf16_split3(v.x, h[0], m[0], l[0]);
  bf16_split3(v.y, h[1], m[1], l[1]);
  bf16_split3(v.z, h[2], m[2], l[2]);
  bf16_split3(v.w, h[3], m[3], l[3]);
  hi = pack_bf16x4(h[0], h[1], h[2], h[3]);
  mid = pack_bf16x4(m[0], m[1], m[2], m[3]);
  lo = pack_bf16x4(l[0], l[1], l[2], l[3]);
}

// Piece i of this thread in a stage: source row and 16-byte piece f of the row.  A warp's 32
// pieces are 8 consecutive rows x 4 pieces of one K step, so that its BF16 stores (8 bytes
// at row r, K offset 4 f') fill all 32 banks twice over, and its ring reads (rows 144 bytes
// apart) are conflict-free by quarter warp.
__device__ __forceinline__ void tc_piece(int e, int& row, int& f) {
  const int q = e >> 5, lane = e & 31;
  row = (q / kTcKs) * 8 + (lane & 7);
  f = (q % kTcKs) * 4 + (lane >> 3);
}

// grid (nks, nvec, nchunk) for TC_OP, (nks, 1, nchunk) otherwise; block kTcThreads; dynamic
// shared memory tc_dots_smem(nb, nsrc).
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 2) k_tc_dots(TcDotsArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = blockIdx.x, vec = blockIdx.y, c = blockIdx.z;
  const long kv = (long)vec * a.nks + k;
  const int nb = a.nb;
  const uint32_t ncols = nb <= 128 ? 128u : 256u;
  const int nsrc = tc_nsrc<MODE>(a.nbnd, a.nproj);
  const int nsrc8 = (nsrc + 7) / 8 * 8;
  const int npiece = nsrc8 * kTcF4;
  const size_t raw_slot = (size_t)nsrc8 * kTcRawRow;
  unsigned char* raw = tsm;
  unsigned char* tile = tsm + kTcRaw * raw_slot;
  const size_t step_bytes = (size_t)kTcATile + 32 * nb;
  const size_t lev_bytes = kTcKs * step_bytes;
  const int g0 = c * kChunk;
  const int g1 = max(g0, min(a.npw[k], g0 + kChunk));
  const int nstage = max(1, (g1 - g0 + kTcPw - 1) / kTcPw);

  if (warp == 0) tc_alloc(&tslot, ncols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tslot;
  const uint32_t idesc = tc_idesc_bf16(128, nb);

  // the FP32 pieces of stage st into ring slot st % kTcRaw (zero beyond the chunk's sphere)
  auto issue = [&](int st) {
    const int gs = g0 + st * kTcPw;
    unsigned char* slot = raw + (size_t)(st % kTcRaw) * raw_slot;
#pragma unroll
    for (int i = 0; i < kTcMaxF4; ++i) {
      const int e = tid + i * kTcThreads;
      if (e < npiece) {
        int row, f;
        tc_piece(e, row, f);
        if (row < nsrc) {
          const int g = gs + 2 * f;
          int da, das, db, dbs;
          const float4* src = tc_src<MODE>(a, k, kv, row, da, das, db, dbs);
          const int bytes = g < g1 ? (g + 1 < g1 ? 16 : 8) : 0;
          cp_async16(slot + row * kTcRawRow + f * 16, src + (bytes ? (g >> 1) : 0), bytes);
        }
      }
    }
  };
  // ring slot st % kTcRaw -> the three BF16 levels of A and Bop (and the swapped copies)
  auto convert = [&](int st) {
    const unsigned char* slot = raw + (size_t)(st % kTcRaw) * raw_slot;
#pragma unroll
    for (int i = 0; i < kTcMaxF4; ++i) {
      const int e = tid + i * kTcThreads;
      if (e < npiece) {
        int row, f;
        tc_piece(e, row, f);
        if (row < nsrc) {
          int da, das, db, dbs;
          tc_src<MODE>(a, k, kv, row, da, das, db, dbs);
          const int ks = f >> 2, kin = (f & 3) * 4;
          const float4 v = *reinterpret_cast<const float4*>(slot + row * kTcRawRow + f * 16);
          uint2 h, m, l;
          split4(v, h, m, l);
          unsigned char* base = tile + ks * step_bytes;
          if (da >= 0) {
            const uint32_t o = tc_off(da, kin);
            *reinterpret_cast<uint2*>(base + o) = h;
            *reinterpret_cast<uint2*>(base + lev_bytes + o) = m;
            *reinterpret_cast<uint2*>(base + 2 * lev_bytes + o) = l;
          }
          if (db >= 0) {
            const uint32_t o = kTcATile + tc_off(db, kin);
            *reinterpret_cast<uint2*>(base + o) = h;
            *reinterpret_cast<uint2*>(base + lev_bytes + o) = m;
            *reinterpret_cast<uint2*>(base + 2 * lev_bytes + o) = l;
          }
          if (das >= 0 || dbs >= 0) {   // swap: (im, -re) per complex value
            split4(make_float4(v.y, -v.x, v.w, -v.z), h, m, l);
            const uint32_t o = das >= 0 ? tc_off(das, kin) : kTcATile + tc_off(dbs, kin);
            *reinterpret_cast<uint2*>(base + o) = h;
            *reinterpret_cast<uint2*>(base + lev_bytes + o) = m;
            *reinterpret_cast<uint2*>(base + 2 * lev_bytes + o) = l;
          }
        }
      }
    }
  };

  bool ok = true;
  uint32_t phase = 0;
  issue(0);
  cp_async_commit();
  if (nstage > 1) issue(1);
  cp_async_commit();
  for (int st = 0; st < nstage; ++st) {
    if (st + 2 < nstage) issue(st + 2);
    cp_async_commit();
    cp_async_wait<2>();            // this thread's pieces of stage st have landed
    if (st > 0) {                  // the tensor core has finished reading the BF16 tiles
      if (!mbar_wait(&bar, phase)) ok = false;
      phase ^= 1;
      tc_fence_after();
    }
    convert(st);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t s0 = smem_u32(tile);
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
      for (int ks = 0; ks < kTcKs; ++ks)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint32_t sa = s0 + (uint32_t)(pa[p] * lev_bytes + ks * step_bytes);
          const uint32_t sb = s0 + (uint32_t)(pb[p] * lev_bytes + ks * step_bytes + kTcATile);
          tc_mma(taddr, tc_desc(sa), tc_desc(sb), idesc, (st > 0 || ks > 0 || p > 0) ? 1 : 0);
        }
      tc_commit(&bar);
    }
  }
  cp_async_wait<0>();
  if (!mbar_wait(&bar, phase)) ok = false;
  tc_fence_after();
  if (!ok && lane == 0) flag_error(a.err, DEV_TIMEOUT, a.jdev ? *a.jdev : 0);

  // epilogue: warp w reads lanes 32 (w % 4).. and the column half w / 4
  const int row = (warp & 3) * 32 + lane;
  const int half = nb / 2, cbeg = (warp >> 2) * half;
  const int nbd = a.nbnd, np = a.nproj, nn = nbd * nbd;
  double* cp = MODE == TC_OP ? reinterpret_cast<double*>(a.cpart + (kv * a.nchunk + c) * np * nbd) : nullptr;
  double* sp = reinterpret_cast<double*>(
      a.spart + (MODE == TC_OP ? (kv * a.nchunk + c) * nn
                               : ((long)k * a.nchunk + c) * (MODE == TC_U2 ? 2 * nn : nn)));
  for (int c0 = cbeg; c0 < cbeg + half; c0 += 16) {
    float d[16];
    tc_ld16(taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, d);
    if (!ok) continue;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int col = c0 + i;
      const double val = (double)d[i];
      if (MODE == TC_OP) {
        if (row < np) {
          if (col < nbd) cp[2 * (row * nbd + col)] = val;
          else if (col < 2 * nbd) cp[2 * (row * nbd + col - nbd) + 1] = val;
        } else if (row < np + 2 * nbd && col >= 2 * nbd && col < 3 * nbd) {
          const int r = row - np, v = r % nbd, w = col - 2 * nbd;
          sp[2 * (w * nbd + v) + (r >= nbd ? 1 : 0)] = val;
        }
      } else if (col < nbd) {
        const int blk = MODE == TC_U2 ? row / (2 * nbd) : 0;
        const int r = row - blk * 2 * nbd;
        if (row < (MODE == TC_U2 ? 4 : 2) * nbd) sp[2 * (blk * nn + col * nbd + r % nbd) + (r >= nbd ? 1 : 0)] = val;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(taddr, ncols);
}

}  // namespace ll

namespace ll {

// The projections applied, t <- t + B c - U S (= P_c (t + B c)), on the tensor cores:
//
//   D[g][n] = sum_k' A[g][k'] Bop[n][k'],  one tile of 128 plane waves g (M = 128),
//   A[g][2q + p]  = part p (re, im) of W_q(g),  W = [B (nproj rows) | U (nbnd rows)]
//   Bop[2v][2q] = Re c'_qv, Bop[2v][2q+1] = -Im c'_qv, Bop[2v+1][2q] = Im c'_qv,
//   Bop[2v+1][2q+1] = Re c'_qv,   c' = [c | -S] (the reduced coefficients of k_sp_coef)
//
// so that D[g][2v] + i D[g][2v+1] = sum_q W_q(g) c'_qv.  Same three-way BF16 split and six
// products as k_tc_dots.  The coefficient operand stays in shared memory for the CTA's
// whole chunk; the rows of W stream through in stages of kTaKs K steps (8 q each).  The
// epilogue adds D to t (zero on the sphere's padding) and forms the chunk's partial
// Re(x^H t) when a norm is wanted.
constexpr int kTaKs = 2;         // K steps per stage: 2 x 8 rows q of W
constexpr int kTaRows = 8 * kTaKs;
constexpr int kTaRing = 5;       // FP32 stages of W in flight (cp.async ring)
constexpr int kTaRawRow = 128 * 8 + 64;   // bytes of one W row of a raw stage (padded)
constexpr int kTaBands = 16;     // bands per epilogue group (a multiple of 8)

struct TcApplyArgs {
  int nks, nbnd, npw_pad, nchunk, nproj, nb, nks_k;  // nb = N (2 nbnd padded to 32); nks_k = K steps of K'
  const int* npw;
  const float2* x;       // operator input (norm partial), or null
  float2* t;             // vector updated in place
  const float2* ukq;
  const float2* bkq;
  const float2* coef;    // [kv][nproj + nbnd][nbnd]
  double* part;          // norm partial per (kv, chunk), or null
  int* err;
  const int* jdev;
};

__host__ __device__ inline size_t tc_apply_smem(int nb, int nks_k) {
  return (size_t)3 * nks_k * 32 * nb + (size_t)3 * kTaKs * kTcATile + (size_t)kTaRing * kTaRows * kTaRawRow;
}

// grid (nks, nvec, nchunk), block kTcThreads, dynamic shared memory tc_apply_smem(nb, nks_k).
// The rows of W of stage (tile, st) stream into a ring of FP32 stages (cp.async, kTaRing - 1
// stages ahead, across tiles), are split into the BF16 A tile and multiplied.
static __global__ void __launch_bounds__(kTcThreads, 1) k_tc_apply(TcApplyArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ double wred[kTcThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = blockIdx.x, vec = blockIdx.y, c = blockIdx.z;
  const long kv = (long)vec * a.nks + k;
  const int nb = a.nb, nbnd = a.nbnd, np = a.nproj, nq = np + nbnd, nks_k = a.nks_k;
  const long pad = a.npw_pad;
  const int npw = a.npw[k];
  const int g0 = c * kChunk, g1 = min(a.npw_pad, g0 + kChunk);
  const size_t bop_lev = (size_t)nks_k * 32 * nb;           // one level of the coefficient operand
  unsigned char* bop = tsm;
  unsigned char* ast = tsm + 3 * bop_lev;                    // A stage: [level][kTaKs][128 rows x 32 B]
  const size_t ast_lev = (size_t)kTaKs * kTcATile;
  unsigned char* ring = ast + 3 * ast_lev;                   // [kTaRing][kTaRows][kTaRawRow]
  const int nstage = (nq + kTaRows - 1) / kTaRows;          // stages per tile
  const int ntile = (g1 - g0 + 127) / 128;
  const int nseq = ntile * nstage;                           // (tile, stage) in order

  if (warp == 0) tc_alloc(&tslot, 128);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the coefficient operand, all three levels, zero outside the 2 nbnd x 2 nq block
  {
    const float2* cf = a.coef + kv * (long)nq * nbnd;
    for (int e = tid; e < nb * nks_k * 16; e += kTcThreads) {
      const int n = e / (nks_k * 16), kk = e - n * (nks_k * 16);
      const int q = kk >> 1, v = n >> 1;
      float val = 0.f;
      if (n < 2 * nbnd && q < nq) {
        float2 cc = cf[q * nbnd + v];
        if (q >= np) cc = make_float2(-cc.x, -cc.y);
        val = (n & 1) ? ((kk & 1) ? cc.x : cc.y) : ((kk & 1) ? -cc.y : cc.x);
      }
      __nv_bfloat16 h, m, l;
      bf16_split3(val, h, m, l);
      const uint32_t o = (uint32_t)((kk >> 4) * 32 * nb) + tc_off(n, kk & 15);
      *reinterpret_cast<__nv_bfloat16*>(bop + o) = h;
      *reinterpret_cast<__nv_bfloat16*>(bop + bop_lev + o) = m;
      *reinterpret_cast<__nv_bfloat16*>(bop + 2 * bop_lev + o) = l;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tslot;
  const uint32_t idesc = tc_idesc_bf16(128, nb);

  // copy mapping: 16-byte pieces (two plane waves of one row q), consecutive threads along g
  auto issue = [&](int sq) {
    if (sq >= nseq) return;
    const int gt = g0 + (sq / nstage) * 128, st = sq % nstage;
    unsigned char* slot = ring + (size_t)(sq % kTaRing) * kTaRows * kTaRawRow;
#pragma unroll
    for (int i = 0; i < kTaRows * 64 / kTcThreads; ++i) {
      const int e = tid + i * kTcThreads;
      const int ql = e >> 6, gp = e & 63;
      const int q = st * kTaRows + ql, g = gt + 2 * gp;
      const int bytes = (q < nq && g < npw) ? (g + 1 < npw ? 16 : 8) : 0;
      const float2* src = a.ukq;    // any valid address when nothing is copied
      if (bytes) src = (q < np ? a.bkq + ((long)k * np + q) * pad : a.ukq + ((long)k * nbnd + (q - np)) * pad) + g;
      cp_async16(slot + ql * kTaRawRow + gp * 16, src, bytes);
    }
  };
  // convert mapping: lane = (g % 8, q % 4), conflict-free 4-byte BF16 stores
  auto convert = [&](int sq) {
    const unsigned char* slot = ring + (size_t)(sq % kTaRing) * kTaRows * kTaRawRow;
#pragma unroll
    for (int i = 0; i < kTaRows * 128 / kTcThreads; ++i) {
      const int e = tid + i * kTcThreads;
      const int item = e >> 5, ln = e & 31;
      const int gl = (item & 15) * 8 + (ln & 7);         // plane wave in the tile
      const int ql = (item >> 4) * 4 + (ln >> 3);         // row q in the stage
      const float2 v = *reinterpret_cast<const float2*>(slot + ql * kTaRawRow + gl * 8);
      __nv_bfloat16 hr, mr, lr, hi, mi, li;
      bf16_split3(v.x, hr, mr, lr);
      bf16_split3(v.y, hi, mi, li);
      const int kk = 2 * ql;
      const uint32_t o = (uint32_t)((kk >> 4) * kTcATile) + tc_off(gl, kk & 15);
      *reinterpret_cast<uint32_t*>(ast + o) = (uint32_t)__bfloat16_as_ushort(hr) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
      *reinterpret_cast<uint32_t*>(ast + ast_lev + o) =
          (uint32_t)__bfloat16_as_ushort(mr) | ((uint32_t)__bfloat16_as_ushort(mi) << 16);
      *reinterpret_cast<uint32_t*>(ast + 2 * ast_lev + o) =
          (uint32_t)__bfloat16_as_ushort(lr) | ((uint32_t)__bfloat16_as_ushort(li) << 16);
    }
  };

  bool ok = true;
  uint32_t phase = 0;
  bool pending = false;          // MMAs committed and not yet waited for
  double nr = 0.0;
  const int row = (warp & 3) * 32 + lane;
  const int half = nb / 2, cbeg = (warp >> 2) * half;
  for (int i = 0; i < kTaRing - 1; ++i) {
    issue(i);
    cp_async_commit();
  }
  for (int sq = 0; sq < nseq; ++sq) {
    const int tile = sq / nstage, st = sq % nstage;
    issue(sq + kTaRing - 1);
    cp_async_commit();
    cp_async_wait<kTaRing - 1>();       // this thread's pieces of stage sq have landed
    if (pending) {                      // the tensor core has finished with the A tile
      if (!mbar_wait(&bar, phase)) ok = false;
      phase ^= 1;
      pending = false;
      tc_fence_after();
    }
    __syncthreads();                    // every thread's pieces of stage sq are in the ring
    convert(sq);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa0 = smem_u32(ast), sb0 = smem_u32(bop);
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
      for (int ks = 0; ks < kTaKs; ++ks) {
        const int kg = st * kTaKs + ks;   // K step of K'
        if (kg >= nks_k) break;
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint32_t sa = sa0 + (uint32_t)(pa[p] * ast_lev + ks * kTcATile);
          const uint32_t sb = sb0 + (uint32_t)(pb[p] * bop_lev + (size_t)kg * 32 * nb);
          tc_mma(taddr, tc_desc(sa), tc_desc(sb), idesc, (st > 0 || ks > 0 || p > 0) ? 1 : 0);
        }
      }
      tc_commit(&bar);
    }
    pending = true;
    if (st + 1 < nstage) continue;
    // epilogue: thread = plane wave gt + row, the bands of its column half, in groups of
    // kTaBands.  The group's t and x values are loaded before the wait for the tile's last
    // MMAs (the first group) or before its tensor-memory loads, so that their latency overlaps.
    const int gt = g0 + tile * 128;
    const int g = gt + row;
    const bool live = g < npw;
    for (int vb = 0; vb < half / 2; vb += kTaBands) {
      const int v0 = (cbeg >> 1) + vb;
      float2 tv[kTaBands], xv[kTaBands];
#pragma unroll
      for (int j = 0; j < kTaBands; ++j) {
        tv[j] = xv[j] = make_float2(0.f, 0.f);
        const int v = v0 + j;
        if (live && vb + j < half / 2 && v < nbnd) {
          const long idx = (kv * nbnd + v) * pad + g;
          tv[j] = a.t[idx];
          if (a.x) xv[j] = a.x[idx];
        }
      }
      if (vb == 0) {   // the tile's accumulator is complete once its last MMAs are
        if (!mbar_wait(&bar, phase)) ok = false;
        phase ^= 1;
        pending = false;
        tc_fence_after();
      }
#pragma unroll
      for (int h = 0; h < kTaBands / 8; ++h) {
        const int c0 = cbeg + 2 * vb + 16 * h;
        if (c0 >= cbeg + half) break;
        float d[16];
        tc_ld16(taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, d);
        if (!ok || g >= g1) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int j = 8 * h + i, v = v0 + j;
          if (v >= nbnd) continue;
          float2 r = make_float2(0.f, 0.f);
          if (live) {
            r = make_float2(tv[j].x + d[2 * i], tv[j].y + d[2 * i + 1]);
            nr += (double)(xv[j].x * r.x + xv[j].y * r.y);
          }
          a.t[(kv * nbnd + v) * pad + g] = r;
        }
      }
    }
    tc_fence_before();
    __syncthreads();   // every thread has read the accumulator before the next tile's MMAs
    tc_fence_after();
  }
  cp_async_wait<0>();
  if (!ok && lane == 0) flag_error(a.err, DEV_TIMEOUT, a.jdev ? *a.jdev : 0);
  if (a.part) {
    nr = warp_sum(nr);
    if (lane == 0) wred[warp] = nr;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < kTcThreads / 32; ++w) s += wred[w];
      a.part[kv * a.nchunk + c] = s;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(taddr, 128);
}

}  // namespace ll
