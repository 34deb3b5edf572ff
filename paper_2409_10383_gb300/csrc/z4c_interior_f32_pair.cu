// FP32-RHS split schedules 5 and 6 on wide tiles (32 x 4 or 64 x 2 cells,
// a warp along one row) for order 6 (4 ghosts) and n = 32, 64, 96, 128
// cells per axis: the RHS kernel with one cell per thread (schedule 5) or
// two cells per thread on packed f32x2 arithmetic (interior_pair_kernel,
// schedule 6).
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
namespace {
template <int ORD, int EXT>
cudaError_t go(int shape, bool pair, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (pair && shape == 1)
    interior_pair_kernel<ORD, EXT, 1><<<ntiles, dim3(TX, TY / 2), 0, st>>>(a, tiles);
  else if (pair && shape == 2)
    interior_pair_kernel<ORD, EXT, 2><<<ntiles, dim3(2 * TX, TY / 4), 0, st>>>(a, tiles);
  else if (shape == 1)
    interior_pre_kernel<ORD, true, 4, true, EXT, 1><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  else if (shape == 2)
    interior_pre_kernel<ORD, true, 4, true, EXT, 2><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}
}  // namespace

bool wide_ext_built(int order, int ext) {
  if (order == 6) return ext == 40 || ext == 72 || ext == 104 || ext == 136;
  return false;
}

cudaError_t launch_wide_rhs_f32(int order, int ext, int shape, bool pair, const StageArgs &a, const Tile *tiles,
                                int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (order == 6) {
    switch (ext) {
      case 40: return go<6, 40>(shape, pair, a, tiles, ntiles, st);
      case 72: return go<6, 72>(shape, pair, a, tiles, ntiles, st);
      case 104: return go<6, 104>(shape, pair, a, tiles, ntiles, st);
      case 136: return go<6, 136>(shape, pair, a, tiles, ntiles, st);
    }
  }
  return cudaErrorInvalidValue;
}
}  // namespace z4c
