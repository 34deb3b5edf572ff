// FP32-RHS instantiations of the fused interior stage kernel: stencils and
// RHS algebra in FP32 from the FP32 shadow; 1/chi, RK update and constraint
// enforcement in FP64.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
cudaError_t launch_interior_f32(int order, const StageArgs &a, const Tile *tiles, int ntiles,
                                cudaStream_t st) {
  return launch_interior<true>(order, a, tiles, ntiles, st);
}
}  // namespace z4c
