// Launchers of the mesh-refinement transfer kernels (device code in z4c_smr.cuh).
#include "z4c_smr.cuh"

namespace z4c {

cudaError_t launch_restrict(double *reg, const DevBlock *blocks, const RestrictRef *list, int n, const double *wtab,
                            bool to_buffer, double *cb, int ncb, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long tot = (long long)n * NF;
  restrict_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(reg, blocks, list, n, wtab, to_buffer ? 1 : 0, cb,
                                                                  ncb);
  return cudaGetLastError();
}

cudaError_t launch_restrict_blocks(const double *reg, const DevBlock *blocks, const int32_t *rblocks, int nrb,
                                   const double *wtab, const int32_t *krow, double *rb, cudaStream_t st) {
  if (nrb <= 0) return cudaSuccess;
  restrict_block_kernel<<<dim3(nrb, NF), 256, 0, st>>>(reg, blocks, rblocks, wtab, krow, rb);
  return cudaGetLastError();
}

cudaError_t launch_rb_scatter(double *reg, const DevBlock *blocks, const RbCopy *list, int n, const double *rb,
                              double *cb, int ncb, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long tot = (long long)n * NF;
  rb_scatter_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(reg, blocks, list, n, rb, cb, ncb);
  return cudaGetLastError();
}

cudaError_t launch_prolong_boxes(double *reg, const DevBlock *blocks, const PBox *boxes, int nbox,
                                 const int32_t *slots, const int32_t *axtab, const double *cb, int ncb,
                                 const double *pw, cudaStream_t st) {
  if (nbox <= 0) return cudaSuccess;
  prolong_box_kernel<<<dim3(nbox, NF), 128, 0, st>>>(reg, blocks, boxes, slots, axtab, cb, ncb, pw);
  return cudaGetLastError();
}

cudaError_t launch_cb_copy(const double *reg, const DevBlock *blocks, const CbCopy *list, int n, double *cb, int ncb,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cb_copy_kernel<<<(n + 255) / 256, 256, 0, st>>>(reg, blocks, list, n, cb, ncb);
  return cudaGetLastError();
}

cudaError_t launch_prolong(double *reg, const DevBlock *blocks, const ProlongRef *list, int n, const int32_t *idx,
                           const double *cb, int ncb, const double *pw, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long tot = (long long)n * NF;
  prolong_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(reg, blocks, list, n, idx, cb, ncb, pw);
  return cudaGetLastError();
}

}  // namespace z4c
