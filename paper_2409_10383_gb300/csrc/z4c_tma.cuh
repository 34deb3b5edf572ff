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

// Ask the TMA unit to bring `bytes` (a multiple of 16) from a 16-byte
// aligned global address into L2 ahead of use.  No completion to wait for,
// no registers held: the loads that follow simply find the lines in L2.
__device__ __forceinline__ void l2_prefetch(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// L2 prefetch of storage rows [r0, r1) of storage plane `plane` of array f
// (S elements per array) of a block whose field 0 starts at base + boff:
// one bulk request for the whole run of rows, ghosts along x included.
// Skipped past the last storage plane (e2) or where the run is not 16-byte
// aligned (block offset, row length or array size not a multiple of 16
// bytes).
template <class T>
__device__ __forceinline__ void prefetch_rows(const T *base, int f, int32_t S, int plane, int r0, int r1, int e0,
                                              int e1, int e2, int64_t boff) {
  constexpr int A = 16 / sizeof(T);
  if (plane >= e2 || r1 <= r0 || (boff % A) != 0 || (e0 % A) != 0 || (S % A) != 0) return;
  r0 = r0 < 0 ? 0 : r0;
  r1 = r1 > e1 ? e1 : r1;
  const int64_t first = boff + (int64_t)f * S + ((int64_t)plane * e1 + r0) * e0;
  l2_prefetch(base + first, (uint32_t)((r1 - r0) * e0 * (int)sizeof(T)));
}

// How many interior planes ahead of its own tile the FP32 stencil kernels
// prefetch: the split RHS kernels (shadow fields and stored derivatives)
// and the y/z pre-pass (shadow fields).  Tiles run plane after plane, so
// plane k + 4 (the stencil's reach) is first touched in HBM by the tiles at
// plane k; the bulk request brings its rows whole instead of line by line
// as the stencil loads reach them.
constexpr int PF_RHS = 4, PF_PRE = 4;

}  // namespace z4c
