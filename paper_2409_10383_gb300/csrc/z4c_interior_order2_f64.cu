// FP64 interior kernels for 2nd-order differencing with 2 ghosts (the
// paper's default with 2 ghost cells, Sec. 3.1 footnote): the y/z pre-pass,
// the fused kernel with runtime strides (schedules 1 and 2), and the fused
// pre-pass kernel specialised for the cubic storage extents n + 4 of common
// block sizes (16, 48, 64, 96, 128).
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {
namespace {
template <int EXT>
cudaError_t go(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  interior_pre_kernel<2, false, 1, false, EXT><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_prepass_f64_order2(const StageArgs &a, const Tile *wtiles, int nwtiles, cudaStream_t st) {
  if (nwtiles <= 0) return cudaSuccess;
  dydz_kernel<2, false><<<nwtiles, dim3(TX, TY), 0, st>>>(a, wtiles);
  return cudaGetLastError();
}

cudaError_t launch_fused_f64_order2(const StageArgs &a, const Tile *tiles, int ntiles, bool pre, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (pre)
    interior_pre_kernel<2, false, 1><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  else
    interior_kernel<2, false><<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}

cudaError_t launch_fused_pre_f64_ext2(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (ext) {
    case 20: return go<20>(a, tiles, ntiles, st);
    case 52: return go<52>(a, tiles, ntiles, st);
    case 68: return go<68>(a, tiles, ntiles, st);
    case 100: return go<100>(a, tiles, ntiles, st);
    case 132: return go<132>(a, tiles, ntiles, st);
    default: return go<0>(a, tiles, ntiles, st);
  }
}
}  // namespace z4c
