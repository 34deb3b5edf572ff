// FP64 instantiations of the interior kernels.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {

cudaError_t launch_prepass_f64(int order, const StageArgs &a, const Tile *wtiles, int nwtiles, cudaStream_t st) {
  if (nwtiles <= 0) return cudaSuccess;
  if (order == 2) return launch_prepass_f64_order2(a, wtiles, nwtiles, st);
  dim3 block(TX, TY);
  if (order == 4)
    dydz_kernel<4, false><<<nwtiles, block, 0, st>>>(a, wtiles);
  else
    dydz_kernel<6, false><<<nwtiles, block, 0, st>>>(a, wtiles);
  return cudaGetLastError();
}

cudaError_t launch_fused_f64(int order, const StageArgs &a, const Tile *tiles, int ntiles, bool pre,
                             cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (order == 2) return launch_fused_f64_order2(a, tiles, ntiles, pre, st);
  dim3 block(TX, TY);
  if (pre) {
    if (order == 4)
      interior_pre_kernel<4, false, 1><<<ntiles, block, 0, st>>>(a, tiles);
    else
      interior_pre_kernel<6, false, 1><<<ntiles, block, 0, st>>>(a, tiles);
  } else if (order == 4) {
    interior_kernel<4, false><<<ntiles, block, 0, st>>>(a, tiles);
  } else {
    interior_kernel<6, false><<<ntiles, block, 0, st>>>(a, tiles);
  }
  return cudaGetLastError();
}

}  // namespace z4c
