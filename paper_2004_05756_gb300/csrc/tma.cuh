// Tensor-memory-accelerator (TMA) copies and mbarrier waits shared by the kernels that stage
// operands with cp.async.bulk.tensor: the tcgen05 projection contraction and the TMA-staged
// 2D block apply. Every wait is bounded: on expiry the context status becomes
// TOPO_ERR_TIMEOUT and the caller unwinds.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace topo {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

struct Ctl {
  volatile int* abort;  // shared: set by the first wait that expires
  int* status;          // global context status word
  long long limit;      // cycles per wait
};

// Teardown waits (copies and MMAs already in flight) get a fixed generous bound, independent
// of the caller's wait limit: a CTA must not leave while its copies can still land.
constexpr long long kTeardownCycles = 4000000000LL;

// Wait for the phase of `bar` with the given parity to complete. Gives up (false) when another
// wait of the CTA already expired (honour_abort) or after ctl.limit cycles, recording the
// timeout.
__device__ inline bool wait_bar(uint32_t bar, uint32_t parity, const Ctl& ctl, bool honour_abort) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (honour_abort && *ctl.abort) return false;
    if (clock64() - t0 > ctl.limit) {
      *ctl.abort = 1;
      atomicCAS(ctl.status, 0, (int)TOPO_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// One 2D tiled box load into shared memory, completing `bytes` on the mbarrier `bar`.
// The innermost coordinate x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Host: encode a 2D tensor map over an FP32 column-major rows x cols block with leading
// dimension ld (elements; ld * 4 must be a multiple of 16, A 16-byte aligned) and box
// box_x x box_y; elements outside the block read as zero. swizzle128 selects the 128-byte
// swizzle, otherwise the box lands unswizzled, x fastest. False when the driver entry point
// is missing or the encoder rejects the arguments.
bool encode_map_f32_2d(CUtensorMap* m, const float* A, long long ld, long long rows, long long cols, unsigned box_x,
                       unsigned box_y, bool swizzle128);

}  // namespace topo
