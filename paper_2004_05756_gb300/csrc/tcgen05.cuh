// 5th-generation tensor-core (tcgen05) helpers shared by the kernels that issue MMAs from
// shared memory into tensor memory (TMEM): the FP32 projection contraction and the reduced
// assembly of many candidate designs.
#pragma once
#include <stdint.h>

namespace topo {

// Shared-memory matrix descriptor: K-major operand in 8-row x 128-B atoms with the 128-byte
// swizzle; start address >> 4 (bits 0-13), leading offset unused for this layout, stride
// between 8-row atoms 1024 B (bits 32-45), descriptor version 1 (bits 46-47), swizzle mode 2
// (bits 61-63). The tile base must be 1024-byte aligned, so the base offset is 0. Advancing
// the start address by 32 B (descriptor + 2) steps K by 32 B inside the swizzle atom.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// Byte offset of the 16-byte chunk `chunk` (0..7) of row `row` in a K-major tile of 128-byte
// rows with the 128-byte swizzle (chunk index XOR row mod 8 inside each 8-row, 1024-byte atom):
// the layout a TMA load with CU_TENSOR_MAP_SWIZZLE_128B writes and smem_desc_sw128 reads.
__device__ __forceinline__ uint32_t sw128_offset(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Arrive once on the mbarrier when every tcgen05 operation this thread issued before has
// completed (their shared-memory reads and TMEM writes included).
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ...).
__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace topo
