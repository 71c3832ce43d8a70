// fv_umma.cuh -- the fifth-generation tensor core instructions (tcgen05) used
// by the learned correction's convolutions, as inline PTX:
//   - shared-memory matrix descriptors for the no-swizzle K-major layout,
//   - the instruction descriptor of kind::f16 (BF16 x BF16 -> FP32),
//   - TMEM allocation, the MMA, its commit to an mbarrier, a bounded wait,
//     and the TMEM -> register load of the accumulator.
//
// No-swizzle K-major layout: a "core matrix" is 8 rows x 16 bytes (8 BF16
// along K), its rows 16 bytes apart.  The descriptor gives the start of the
// first core matrix, the byte step between core matrices adjacent along K
// (leading byte offset) and between groups of 8 rows along M or N (stride
// byte offset).  One MMA of K = 16 reads two core matrices along K.
#pragma once

#include <cstdint>

namespace umma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (no swizzle): start address, K step and
// M/N step in bytes (all multiples of 16); bit 46 is the descriptor version
// of this architecture.
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t kstep, uint32_t mnstep) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((kstep >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((mnstep >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Allocates `ncols` TMEM columns (a power of two >= 32) for the CTA; one
// whole warp calls it and the address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(slot)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// D (TMEM) = A * B (+ D if accumulate), issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The mbarrier completes its phase when every MMA this thread issued before
// has finished.
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
}

// Waits for phase `parity` of the mbarrier, at most `limit` polls; returns
// whether it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity));
  }
  return done != 0;
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;");
}
// Orders this thread's shared-memory stores before later tensor-core reads.
__device__ __forceinline__ void fence_smem_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (the warp reads its
// 32 lanes; the address carries the warp's first lane in bits 16..31).
__device__ __forceinline__ void ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace umma
