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
}  // namespace z4c
