// FP64 fused interior kernel (pre-pass schedule), order 6, specialised for
// the cubic storage extents of common block sizes (24, 32, 56, 72, 104), plus the
// runtime-stride kernel for any other shape.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
namespace {
template <int EXT>
cudaError_t go(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  interior_pre_kernel<6, false, 1, false, EXT><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_fused_pre_f64_ext6(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (ext) {
    case 24: return go<24>(a, tiles, ntiles, st);
    case 32: return go<32>(a, tiles, ntiles, st);
    case 56: return go<56>(a, tiles, ntiles, st);
    case 72: return go<72>(a, tiles, ntiles, st);
    case 104: return go<104>(a, tiles, ntiles, st);
    default: return go<0>(a, tiles, ntiles, st);
  }
}
}  // namespace z4c
