// FP64 instantiations of the fused interior stage kernel.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
cudaError_t launch_interior_f64(int order, const StageArgs &a, const Tile *tiles, int ntiles,
                                cudaStream_t st) {
  return launch_interior<false>(order, a, tiles, ntiles, st);
}
}  // namespace z4c
