// Bulk-copy (TMA, cp.async.bulk) and mbarrier helpers shared by the pipelined radix passes
// (k_onesweep_pipe.cu, k_radix_chunk.cu).  Every wait is bounded (kSpinLimit polls).
#pragma once

#include "common.cuh"

namespace reindex {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint32_t round16(uint32_t x) { return (x + 15u) & ~15u; }

// Bounded wait for a buffer's bulk copy.  On timeout the error is recorded and the wait is
// repeated once (bounded) so that the copy has landed before the CTA moves on or exits.
__device__ __forceinline__ void wait_tile(uint64_t* bar, uint32_t parity, Control* c) {
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
      if (mbar_try_wait(bar, parity)) return;
    record_error(c, kErrTimeout);
  }
}

}  // namespace reindex
