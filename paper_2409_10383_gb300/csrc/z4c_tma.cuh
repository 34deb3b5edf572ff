// Bulk asynchronous copies global -> shared through the Tensor Memory
// Accelerator (cp.async.bulk, completion counted on an mbarrier), and the
// mbarrier operations around them.  Inline PTX for sm_90 and later
// (sm_103a here).  A CTA that is not launched as a cluster is its own
// cluster of one, so the shared::cluster forms address the CTA's own
// shared memory.
//
// Every wait is bounded: mbar_wait gives up after a fixed number of
// try_wait rounds and returns false, so a copy that never lands turns into
// an error status instead of a hung kernel.
#pragma once

#include <cstdint>

namespace z4c {

#ifndef Z4C_TMA_PROVIDED

// The CTA's dynamic shared memory (size given at launch).
__device__ __forceinline__ unsigned char *dyn_smem() {
  extern __shared__ __align__(128) unsigned char z4c_dyn_smem[];
  return z4c_dyn_smem;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Initialise an mbarrier expecting `count` arrivals per phase.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make initialised mbarriers visible to the async proxy (before first use).
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of transactions for this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// global memory into shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Wait until the phase with the given parity of `bar` has completed.
// Returns false if it has not after `rounds` try_wait attempts (each of
// which may suspend the thread for a hardware-chosen time).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t rounds = 1u << 22) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t r = 0; r < rounds; ++r) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

#endif  // Z4C_TMA_PROVIDED

}  // namespace z4c
