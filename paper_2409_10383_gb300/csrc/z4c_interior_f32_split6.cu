// FP32-RHS split schedule (4), order 6: RHS kernels storing k, specialised
// for the cubic storage extents of common block sizes (n + 8 for n = 16, 24,
// 48, 64, 96), plus the runtime-stride kernel for any other shape.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
namespace {
template <int EXT>
cudaError_t go6(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  interior_pre_kernel<6, true, 4, true, EXT><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_split_rhs6(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  switch (ext) {
    case 24: return go6<24>(a, tiles, ntiles, st);
    case 32: return go6<32>(a, tiles, ntiles, st);
    case 56: return go6<56>(a, tiles, ntiles, st);
    case 72: return go6<72>(a, tiles, ntiles, st);
    case 104: return go6<104>(a, tiles, ntiles, st);
    default: return go6<0>(a, tiles, ntiles, st);
  }
}
}  // namespace z4c
