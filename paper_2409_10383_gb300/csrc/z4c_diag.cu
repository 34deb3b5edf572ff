// Launchers of the diagnostics kernels (device code in z4c_diag.cuh).
#include <type_traits>

#include "z4c_diag.cuh"

namespace z4c {

cudaError_t launch_indicators(const double *u, const DevBlock *blocks, const Tile *tiles, int ntiles,
                              const int32_t *first, int nb, double *part, double *out, cudaStream_t st) {
  if (ntiles <= 0 || nb <= 0) return cudaSuccess;
  indicator_tile_kernel<<<ntiles, dim3(TX, TY), 0, st>>>(u, blocks, tiles, part);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  indicator_block_kernel<<<(nb + 127) / 128, 128, 0, st>>>(part, first, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_track(const double *u, const DevBlock *blocks, const TrackIn *in, int np, double dt, double *out,
                         cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  track_kernel<<<1, 64, 0, st>>>(u, blocks, in, np, dt, out);
  return cudaGetLastError();
}

cudaError_t launch_psi4(const double *u, const DevBlock *blocks, const Tile *tiles, int ntiles, const double *ds,
                        double *out, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (!ds) return cudaErrorInvalidValue;
  const dim3 block(TX, TY);
  psi4_kernel<2><<<ntiles, block, 0, st>>>(u, blocks, tiles, ds, out);
  psi4_kernel<4><<<ntiles, block, 0, st>>>(u, blocks, tiles, ds, out);
  psi4_kernel<6><<<ntiles, block, 0, st>>>(u, blocks, tiles, ds, out);
  return cudaGetLastError();
}

}  // namespace z4c
