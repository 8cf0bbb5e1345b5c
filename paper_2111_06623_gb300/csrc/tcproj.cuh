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
// Pipeline: the FP32 rows of the next stage of kTcPw plane waves are loaded into registers
// while the tensor core works on the current stage; one elected thread issues the MMAs and
// commits them to an mbarrier that the CTA waits on (bounded) before it overwrites the stage.
#pragma once
#include "split.cuh"
#include "tc.cuh"

namespace ll {

constexpr int kTcKs = 4;              // K steps (16 real values = 8 plane waves) per stage
constexpr int kTcPw = 8 * kTcKs;      // plane waves per stage
constexpr int kTcF4 = kTcPw / 2;      // float4 (two complex values) per row and stage
constexpr int kTcMaxF4 = 12;          // float4 per thread and stage (at most 192 source rows)
constexpr int kTcThreads = 256;
constexpr int kTcATile = 128 * 32;    // bytes of one K step of A (128 rows)

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

// Shared memory of k_tc_dots: three BF16 levels of kTcKs K steps of [A tile | Bop tile].
__host__ __device__ constexpr size_t tc_dots_smem(int nb) {
  return (size_t)3 * kTcKs * (kTcATile + 32 * nb);
}

// Source row s of the CTA's unique rows: its global row (in float4 units of npw_pad/2) and
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

template <int MODE>
__host__ __device__ __forceinline__ int tc_nsrc(int nbnd, int nproj) {
  return MODE == TC_OP ? nproj + 3 * nbnd : (MODE == TC_U ? 2 * nbnd : 3 * nbnd);
}

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

// grid (nks, nvec, nchunk) for TC_OP, (nks, 1, nchunk) otherwise; block kTcThreads; dynamic
// shared memory tc_dots_smem(nb).
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
  const size_t step_bytes = (size_t)kTcATile + 32 * nb;
  const size_t lev_bytes = kTcKs * step_bytes;
  const int g0 = c * kChunk;
  const int g1 = max(g0, min(a.npw[k], g0 + kChunk));
  const int nstage = max(1, (g1 - g0 + kTcPw - 1) / kTcPw);
  const int nsrc = tc_nsrc<MODE>(a.nbnd, a.nproj);
  const int nel = nsrc * kTcF4;

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

  float4 reg[kTcMaxF4];
  auto load = [&](int st) {
    const int gs = g0 + st * kTcPw;
#pragma unroll
    for (int i = 0; i < kTcMaxF4; ++i) {
      const int e = tid + i * kTcThreads;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < nel) {
        const int s = e / kTcF4, f = e - s * kTcF4;
        const int g = gs + 2 * f;
        if (g < g1) {
          int da, das, db, dbs;
          const float4* src = tc_src<MODE>(a, k, kv, s, da, das, db, dbs);
          v = src[g >> 1];
          if (g + 1 >= g1) v.z = v.w = 0.f;
        }
      }
      reg[i] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int i = 0; i < kTcMaxF4; ++i) {
      const int e = tid + i * kTcThreads;
      if (e < nel) {
        const int s = e / kTcF4, f = e - s * kTcF4;
        int da, das, db, dbs;
        tc_src<MODE>(a, k, kv, s, da, das, db, dbs);
        const int ks = f >> 2, kin = (f & 3) * 4;
        const float4 v = reg[i];
        const float4 w = make_float4(v.y, -v.x, v.w, -v.z);   // swap: (im, -re) per complex value
        uint2 h, m, l, hs, ms, ls;
        split4(v, h, m, l);
        if (das >= 0 || dbs >= 0) split4(w, hs, ms, ls);
        unsigned char* base = tsm + ks * step_bytes;
        if (da >= 0) {
          const uint32_t o = tc_off(da, kin);
          *reinterpret_cast<uint2*>(base + o) = h;
          *reinterpret_cast<uint2*>(base + lev_bytes + o) = m;
          *reinterpret_cast<uint2*>(base + 2 * lev_bytes + o) = l;
        }
        if (das >= 0) {
          const uint32_t o = tc_off(das, kin);
          *reinterpret_cast<uint2*>(base + o) = hs;
          *reinterpret_cast<uint2*>(base + lev_bytes + o) = ms;
          *reinterpret_cast<uint2*>(base + 2 * lev_bytes + o) = ls;
        }
        if (db >= 0) {
          const uint32_t o = kTcATile + tc_off(db, kin);
          *reinterpret_cast<uint2*>(base + o) = h;
          *reinterpret_cast<uint2*>(base + lev_bytes + o) = m;
          *reinterpret_cast<uint2*>(base + 2 * lev_bytes + o) = l;
        }
        if (dbs >= 0) {
          const uint32_t o = kTcATile + tc_off(dbs, kin);
          *reinterpret_cast<uint2*>(base + o) = hs;
          *reinterpret_cast<uint2*>(base + lev_bytes + o) = ms;
          *reinterpret_cast<uint2*>(base + 2 * lev_bytes + o) = ls;
        }
      }
    }
  };

  bool ok = true;
  uint32_t phase = 0;
  load(0);
  for (int st = 0; st < nstage; ++st) {
    if (st > 0) {   // the tensor core has finished reading the previous stage
      if (!mbar_wait(&bar, phase)) ok = false;
      phase ^= 1;
      tc_fence_after();
    }
    store();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t s0 = smem_u32(tsm);
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
    if (st + 1 < nstage) load(st + 1);
  }
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
constexpr int kTaPer = kTaRows * 128 / kTcThreads;   // complex values per thread and stage

struct TcApplyArgs {
  int nks, nbnd, npw_pad, nchunk, nproj, nb, nks_k;  // nb = N (2 nbnd padded to 16); nks_k = K steps of K'
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

__host__ __device__ constexpr size_t tc_apply_smem(int nb, int nks_k) {
  return (size_t)3 * nks_k * 32 * nb + (size_t)3 * kTaKs * kTcATile;
}

// grid (nks, nvec, nchunk), block kTcThreads, dynamic shared memory tc_apply_smem(nb, nks_k).
static __global__ void __launch_bounds__(kTcThreads, 2) k_tc_apply(TcApplyArgs a) {
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
  const int nstage = (nq + kTaRows - 1) / kTaRows;

  float2 reg[kTaPer];
  auto load = [&](int gt, int st) {
#pragma unroll
    for (int i = 0; i < kTaPer; ++i) {
      const int e = tid + i * kTcThreads;
      const int ql = e >> 7, gl = e & 127;
      const int q = st * kTaRows + ql, g = gt + gl;
      float2 v = make_float2(0.f, 0.f);
      if (q < nq && g < npw)
        v = q < np ? a.bkq[((long)k * np + q) * pad + g] : a.ukq[((long)k * nbnd + q - np) * pad + g];
      reg[i] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int i = 0; i < kTaPer; ++i) {
      const int e = tid + i * kTcThreads;
      const int ql = e >> 7, gl = e & 127;
      const int kk = 2 * ql;                              // K' index within the stage
      __nv_bfloat16 hr, mr, lr, hi, mi, li;
      bf16_split3(reg[i].x, hr, mr, lr);
      bf16_split3(reg[i].y, hi, mi, li);
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
  for (int gt = g0; gt < g1; gt += 128) {
    load(gt, 0);
    for (int st = 0; st < nstage; ++st) {
      if (pending) {
        if (!mbar_wait(&bar, phase)) ok = false;
        phase ^= 1;
        pending = false;
        tc_fence_after();
      }
      store();
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
      if (st + 1 < nstage) load(gt, st + 1);
    }
    if (!mbar_wait(&bar, phase)) ok = false;
    phase ^= 1;
    pending = false;
    tc_fence_after();
    // epilogue: thread = plane wave gt + row, bands of its column half
    const int g = gt + row;
    for (int c0 = cbeg; c0 < cbeg + half; c0 += 16) {
      float d[16];
      tc_ld16(taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, d);
      if (!ok || g >= g1) continue;
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const int v = (c0 + i) >> 1;
        if (v >= nbnd) continue;
        const long idx = (kv * nbnd + v) * pad + g;
        float2 tv = make_float2(0.f, 0.f);
        if (g < npw) {
          tv = a.t[idx];
          tv.x += d[i];
          tv.y += d[i + 1];
          if (a.x) {
            const float2 xv = a.x[idx];
            nr += (double)(xv.x * tv.x + xv.y * tv.y);
          }
        }
        a.t[idx] = tv;
      }
    }
    tc_fence_before();
    __syncthreads();   // every thread has read the accumulator before the next tile's MMAs
  }
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
