// FP32-RHS fused interior kernel with shared-memory staging (schedule 3).
#include <type_traits>

#include "z4c_staged.cuh"

namespace z4c {
cudaError_t launch_staged_f32(int order, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (order != 6) return cudaErrorInvalidValue;
  constexpr size_t smem = StageGeom<6>::SMEM;
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(staged_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  staged_kernel<6><<<ntiles, dim3(TX, TY), smem, st>>>(a, tiles);
  return cudaGetLastError();
}

// Failure-detection probe: the staged kernel's bounded wait, made to run
// out.  One thread announces 16 bytes on an mbarrier and no copy is ever
// issued, so the phase cannot complete; after `rounds` try_wait attempts
// mbar_wait gives up and the kernel reports it the way staged_kernel does
// (status word |= 1) and returns.  No asynchronous copy is in flight when
// the CTA exits.
__global__ void wait_probe_kernel(int32_t *status, uint32_t rounds) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  mbar_arrive_expect_tx(&bar, 16);
  if (!mbar_wait(&bar, 0, rounds)) atomicOr(status, 1);
}

cudaError_t launch_wait_probe(int32_t *status, int rounds, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(status, (uint32_t)rounds);
  return cudaGetLastError();
}
}  // namespace z4c
