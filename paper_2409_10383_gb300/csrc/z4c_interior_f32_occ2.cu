// FP32-RHS fused interior kernel (pre-pass schedule) compiled for at least
// 2 resident CTAs per SM (fewer registers per thread, more warps to hide
// load latency); picked by the autotuner.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
cudaError_t launch_fused_pre_f32_occ2(int order, const StageArgs &a, const Tile *tiles, int ntiles,
                                       cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (order == 2) return launch_fused_f32_order2(2, a, tiles, ntiles, true, st);
  dim3 block(TX, TY);
  if (order == 4)
    interior_pre_kernel<4, true, 2><<<ntiles, block, 0, st>>>(a, tiles);
  else
    interior_pre_kernel<6, true, 2><<<ntiles, block, 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace z4c
