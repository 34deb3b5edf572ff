// Launchers of the auxiliary kernels (device code in z4c_aux.cuh).
#include "z4c_aux.cuh"

namespace z4c {

cudaError_t launch_ghosts_f64(double *reg, const DevBlock *blocks, const GhostCopy *list, int n,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ghost_kernel<double><<<(n + 255) / 256, 256, 0, st>>>(reg, blocks, list, n);
  return cudaGetLastError();
}

cudaError_t launch_ghosts_f32(float *reg, const DevBlock *blocks, const GhostCopy *list, int n,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ghost_kernel<float><<<(n + 255) / 256, 256, 0, st>>>(reg, blocks, list, n);
  return cudaGetLastError();
}

cudaError_t launch_sommerfeld(bool f32, const StageArgs &a, const CellRef *cells, int ncells,
                              cudaStream_t st) {
  if (ncells <= 0) return cudaSuccess;
  const int nb = (ncells + SOMM_CTA - 1) / SOMM_CTA;
  if (f32) {
    sommerfeld_rhs_f32_kernel<<<nb, SOMM_CTA, 0, st>>>(a, cells, ncells);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sommerfeld_update_f32_kernel<<<nb, SOMM_CTA, 0, st>>>(a, cells, ncells);
  } else {
    sommerfeld_kernel<<<nb, SOMM_CTA, 0, st>>>(a, cells, ncells);
  }
  return cudaGetLastError();
}

size_t somm_kbuf_floats(int ncells) { return (size_t)NF * SOMM_CTA * (size_t)((ncells + SOMM_CTA - 1) / SOMM_CTA); }

cudaError_t launch_initial_data(double *u0, const DevBlock *blocks, int nblocks, int max_S, int instance,
                                int kind, const double *par, int npar, cudaStream_t st) {
  IdPar P{};
  for (int q = 0; q < npar && q < 64; ++q) P.v[q] = par[q];
  dim3 grid((max_S + 255) / 256, nblocks);
  initial_data_kernel<<<grid, 256, 0, st>>>(u0, blocks, instance, kind, P);
  return cudaGetLastError();
}

cudaError_t launch_to_shadow(const double *src, float *dst, const DevBlock *blocks, int nblocks,
                             int max_S, cudaStream_t st) {
  dim3 grid((max_S + 255) / 256, nblocks);
  to_shadow_kernel<<<grid, 256, 0, st>>>(src, dst, blocks);
  return cudaGetLastError();
}

cudaError_t launch_constraint_partials(int order, const double *u0, const DevBlock *blocks, const Tile *tiles,
                                       int ntiles, int instance, double r_mask, double *per_cell,
                                       double *partials, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  dim3 block(TX, TY);
  if (order == 2)
    constraints_kernel<2><<<ntiles, block, 0, st>>>(u0, blocks, tiles, instance, r_mask, per_cell, partials);
  else if (order == 4)
    constraints_kernel<4><<<ntiles, block, 0, st>>>(u0, blocks, tiles, instance, r_mask, per_cell, partials);
  else
    constraints_kernel<6><<<ntiles, block, 0, st>>>(u0, blocks, tiles, instance, r_mask, per_cell, partials);
  return cudaGetLastError();
}

cudaError_t launch_constraint_finalize(const double *partials, int n, double *result, cudaStream_t st) {
  constraints_finalize<<<1, 1024, 0, st>>>(partials, n, result);
  return cudaGetLastError();
}

cudaError_t peak_fma(bool f64, cudaStream_t st, double *flops_per_s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8, iters = f64 ? 2048 : 65536;
  void *sink = nullptr;  // kernel never writes (condition never true)
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int rep = 0; rep < 2; ++rep) {  // first launch warms up clocks
    cudaEventRecord(e0, st);
    if (f64)
      fma_peak_kernel<double><<<blocks, threads, 0, st>>>((double *)sink, iters, 0.999999, 1e-7);
    else
      fma_peak_kernel<float><<<blocks, threads, 0, st>>>((float *)sink, iters, 0.9999f, 1e-7f);
    cudaEventRecord(e1, st);
  }
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *flops_per_s = 2.0 * 8.0 * iters * (double)threads * blocks / (ms * 1e-3);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t peak_convert(int mode, cudaStream_t st, double *conv_per_s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8, iters = 2048;
  unsigned long long *sink = nullptr;  // kernel never writes (condition never true)
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int rep = 0; rep < 2; ++rep) {  // first launch warms up clocks
    cudaEventRecord(e0, st);
    if (mode == 0) convert_peak_kernel<0><<<blocks, threads, 0, st>>>(sink, iters);
    else if (mode == 1) convert_peak_kernel<1><<<blocks, threads, 0, st>>>(sink, iters);
    else if (mode == 2) convert_peak_kernel<2><<<blocks, threads, 0, st>>>(sink, iters);
    else convert_peak_kernel<3><<<blocks, threads, 0, st>>>(sink, iters);
    cudaEventRecord(e1, st);
  }
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *conv_per_s = 8.0 * iters * (double)threads * blocks / (ms * 1e-3);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace z4c
