// FP64 fused interior kernel (pre-pass schedule), order 4, specialised for
// the cubic storage extents of common block sizes (30, 38, 54, 70, 102), plus the
// runtime-stride kernel for any other shape.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
namespace {
template <int EXT>
cudaError_t go(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  interior_pre_kernel<4, false, 1, false, EXT><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_fused_pre_f64_ext4(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (ext) {
    case 30: return go<30>(a, tiles, ntiles, st);
    case 38: return go<38>(a, tiles, ntiles, st);
    case 54: return go<54>(a, tiles, ntiles, st);
    case 70: return go<70>(a, tiles, ntiles, st);
    case 102: return go<102>(a, tiles, ntiles, st);
    default: return go<0>(a, tiles, ntiles, st);
  }
}
}  // namespace z4c
