// tcgen05 (5th-generation tensor core) helpers shared by the kernels that
// contract on the tensor cores: TF32 conversion, shared-memory matrix and
// instruction descriptors for the K-major no-swizzle core-matrix layout, the
// MMA issue and commit, the thread-sync fences, and tensor-memory allocation.
//
// Core-matrix layout (no swizzle, K-major): an operand tile of R rows x BK
// 32-bit elements is stored as 8-row x 16-byte core matrices; element (r, k)
// sits at (r / 8) * SBO + (k / 4) * LBO + (r % 8) * 16 + (k % 4) * 4 bytes,
// with LBO the distance between core matrices along K and SBO between groups
// of 8 rows.
#pragma once

#include "common.cuh"

namespace lpk {

__device__ __forceinline__ uint32_t tc_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// shared-memory matrix descriptor: K-major, no swizzle, byte offsets lbo / sbo
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // fixed descriptor version of tcgen05
  // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
  return d;
}

// instruction descriptor: kind::tf32, FP32 accumulator, K-major A and B, M x N
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int m, int n) {
  return (1u << 4)      // D format F32
         | (2u << 7)    // A format TF32
         | (2u << 10)   // B format TF32
         | (0u << 15)   // A K-major
         | (0u << 16)   // B K-major
         | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on `bar` once every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit_to(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// warp-wide: allocate `ncols` (power of two >= 32) tensor-memory columns, the
// base address written to *slot (shared memory); then give up the permit so
// that other CTAs on the SM may allocate
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// 8 consecutive 32-bit columns of this warp's 32 TMEM lanes (lane = thread)
__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace lpk
