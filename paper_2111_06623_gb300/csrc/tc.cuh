// Fifth-generation tensor-core primitives (tcgen05, sm_103a) as inline PTX: tensor-memory
// allocation, BF16 MMAs with FP32 accumulation in tensor memory, completion through an
// mbarrier, and tensor-memory loads.  Operands are staged in shared memory by the calling
// kernel in the canonical K-major layout without swizzle:
//
//   core matrix = 8 rows x 16 bytes (8 BF16 values of K), 128 contiguous bytes, row r at
//   byte 16 r; one MMA step covers K = 16, i.e. two core matrices along K.  A tile of R rows
//   (R a multiple of 8) and one K step is stored as [R/8][2][8][8] BF16: the 8-row groups
//   kTcSbo = 256 bytes apart (stride dimension), the two K halves kTcLbo = 128 bytes apart
//   (leading dimension); 32 R bytes per tile.
//
// The accumulator of an M = 128 MMA (cta_group::1) is row i in tensor-memory lane i, column
// j in column j (FP32).  Warp w of the CTA reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
//
// Every wait here is bounded: a wait that runs out records an error in the caller's status
// word and returns, so that no kernel can spin forever.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace ll {

constexpr uint32_t kTcLbo = 128;   // bytes between the two K halves of a core-matrix pair
constexpr uint32_t kTcSbo = 256;   // bytes between 8-row groups

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) (k < 16) inside one K-step tile of the layout above.
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
  return (uint32_t)((row >> 3) * kTcSbo + (k >> 3) * kTcLbo + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading and stride byte offsets (all in
// 16-byte units), descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((kTcLbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kTcSbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 accumulator, both K-major,
// N (multiple of 16, <= 256) and M (128).
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Tensor-memory allocation by one whole warp: ncols (a power of two >= 32) columns; the
// address is written to *slot (shared memory).
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Generic-proxy shared-memory writes made visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (+)= A B^T for one K step, issued by a single thread.
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// Arrive once on the mbarrier when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false when the bounded wait ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < (1L << 24); ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// 32 lanes x 16 consecutive FP32 columns: thread t of the warp gets row (lane base + t).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// FP32 -> three BF16 parts, a = hi + mid + lo up to 2^-24 |a| (each part the round-to-nearest
// BF16 of what the previous parts leave).
__device__ __forceinline__ void bf16_split3(float a, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(mid);
  lo = __float2bfloat16_rn(r2);
}

}  // namespace ll
