// Fifth-generation tensor-core MMA (tcgen05) with the accumulator in tensor
// memory, inline PTX for sm_103a: allocation of tensor-memory columns,
// shared-memory matrix descriptors, the instruction descriptor of a dense
// BF16 x BF16 -> FP32 product, issue, commit to an mbarrier and the load of
// the accumulator back to registers.
#pragma once

#include <cstdint>

#include "tma.cuh"

namespace hhg {

// Tensor-memory columns for the CTA (one whole warp executes it); the base
// address (lane 0, first column) is written to *slot in shared memory.
// ncols: a power of two, 32..512.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// one whole warp, the one that allocated
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Orders tensor-core operations around a CTA barrier: "before" ahead of the
// barrier in the thread that issued or read, "after" behind it in the
// thread that issues or reads next.
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory descriptor of a K-major operand without swizzling: the
// operand is made of 8-row x 16-byte core matrices (8 rows of 8 BF16, each
// core matrix 128 contiguous bytes); lbo = byte distance between core
// matrices adjacent in K, sbo = between core matrices adjacent in M (or N).
// Address, lbo and sbo are multiples of 16 bytes below 256 KB.
__device__ __forceinline__ uint64_t smem_desc_kmajor(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = (uint64_t)((smem_u32(p) & 0x3FFFFu) >> 4);
  return a | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46);   // descriptor version 1; base offset 0, layout 0 = no swizzle
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// no negation or sparsity; M x N product shape.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                       // D format FP32
         | (1u << 7)                     // A format BF16
         | (1u << 10)                    // B format BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// D[tmem] (+)= A * B, issued by one thread; accumulate = false overwrites D.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}

// The mbarrier receives one arrival when every earlier tcgen05.mma of this
// thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of the tensor-memory lane of this thread: warp
// w of a warpgroup reads lanes 32 (w % 4) .. + 31 (taddr = lane << 16 | column).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace hhg
