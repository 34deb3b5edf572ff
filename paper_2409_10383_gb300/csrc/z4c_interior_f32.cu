// FP32-RHS instantiations of the fused interior stage kernel: stencils and
// RHS algebra in FP32 from the FP32 shadow; 1/chi, RK update and constraint
// enforcement in FP64.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
template <bool F32>
cudaError_t launch_interior(int order, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  dim3 block(TX, TY);
  if (order == 4)
    interior_kernel<4, F32><<<ntiles, block, 0, st>>>(a, tiles);
  else
    interior_kernel<6, F32><<<ntiles, block, 0, st>>>(a, tiles);
  return cudaGetLastError();
}

cudaError_t launch_interior_f32(int order, const StageArgs &a, const Tile *tiles, int ntiles,
                                cudaStream_t st) {
  return launch_interior<true>(order, a, tiles, ntiles, st);
}
}  // namespace z4c
