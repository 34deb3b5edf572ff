// FP32-RHS interior kernels for 2nd-order differencing with 2 ghosts: the
// y/z pre-pass, the fused kernel (schedule 1; schedule 2 at occupancy 1, 2
// and 4) and the split schedule's RHS kernel (4), the last specialised for
// the cubic storage extents n + 4 of common block sizes (16, 48, 64, 96).
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
namespace {
template <int EXT>
cudaError_t go(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  interior_pre_kernel<2, true, 4, true, EXT><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_prepass_f32_order2(const StageArgs &a, const Tile *wtiles, int nwtiles, cudaStream_t st) {
  if (nwtiles <= 0) return cudaSuccess;
  dydz_kernel<2, true><<<nwtiles, dim3(TX, TY), 0, st>>>(a, wtiles);
  return cudaGetLastError();
}

cudaError_t launch_fused_f32_order2(int occ, const StageArgs &a, const Tile *tiles, int ntiles, bool pre,
                                    cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const dim3 block(TX, TY);
  if (!pre)
    interior_kernel<2, true><<<ntiles, block, 0, st>>>(a, tiles);
  else if (occ == 4)
    interior_pre_kernel<2, true, 4><<<ntiles, block, 0, st>>>(a, tiles);
  else if (occ == 2)
    interior_pre_kernel<2, true, 2><<<ntiles, block, 0, st>>>(a, tiles);
  else
    interior_pre_kernel<2, true, 1><<<ntiles, block, 0, st>>>(a, tiles);
  return cudaGetLastError();
}

bool split_ext_built2(int ext) { return ext == 20 || ext == 52 || ext == 68 || ext == 100; }

cudaError_t launch_split_rhs2(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (ext) {
    case 20: return go<20>(a, tiles, ntiles, st);
    case 52: return go<52>(a, tiles, ntiles, st);
    case 68: return go<68>(a, tiles, ntiles, st);
    case 100: return go<100>(a, tiles, ntiles, st);
    default: return go<0>(a, tiles, ntiles, st);
  }
}
}  // namespace z4c
