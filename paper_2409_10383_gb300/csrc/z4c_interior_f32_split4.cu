// FP32-RHS split schedule (4), order 4: RHS kernels storing k, specialised
// for the cubic storage extents of common block sizes (n + 6 for n = 24, 48,
// 64, 96), plus the runtime-stride kernel for any other shape; and the
// dispatch over the three orders.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
namespace {
template <int EXT>
cudaError_t go4(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  interior_pre_kernel<4, true, 4, true, EXT><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_split_rhs6(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);

bool split_ext_built(int order, int ext) {
  if (order == 2) return split_ext_built2(ext);
  if (order == 6) return ext == 24 || ext == 32 || ext == 56 || ext == 72 || ext == 104;
  return ext == 30 || ext == 54 || ext == 70 || ext == 102;
}

cudaError_t launch_split_rhs_f32(int order, int ext, const StageArgs &a, const Tile *tiles, int ntiles,
                                 cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (!split_ext_built(order, ext)) ext = 0;
  if (order == 6) return launch_split_rhs6(ext, a, tiles, ntiles, st);
  if (order == 2) return launch_split_rhs2(ext, a, tiles, ntiles, st);
  switch (ext) {
    case 30: return go4<30>(a, tiles, ntiles, st);
    case 54: return go4<54>(a, tiles, ntiles, st);
    case 70: return go4<70>(a, tiles, ntiles, st);
    case 102: return go4<102>(a, tiles, ntiles, st);
    default: return go4<0>(a, tiles, ntiles, st);
  }
}
}  // namespace z4c
