// FP32-RHS split schedule (4): RHS kernel storing k, then the stage-update
// and enforcement kernel.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {

// Schedule 4, second kernel: the RK stage update and the FP64 enforcement of
// the FP32 RHS stored by interior_pre_kernel<..., SPLIT = true> (same tile
// list, same tile order).  Few registers, so many warps hide the latency of
// the FP64 state loads.
__global__ void __launch_bounds__(TX * TY, 8) split_epilogue_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = a.blocks[t.block];
  const int i = t.i0 + threadIdx.x, j = t.j0 + threadIdx.y, kk = t.k0;
  if (i >= b.n[0] || j >= b.n[1]) return;
  const int g = b.g;
  const int32_t cidx = ((kk + g) * b.e[1] + (j + g)) * b.e[0] + (i + g);
  const float *kt = a.kbuf + (int64_t)blockIdx.x * NF * (TX * TY) + threadIdx.y * TX + threadIdx.x;
  float k[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) k[f] = kt[f * (TX * TY)];
  stage_epilogue<float>(a, t.block, b.off + cidx, b.S, k);
}

cudaError_t launch_split_f32(int order, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  dim3 block(TX, TY);
  if (order == 4)
    interior_pre_kernel<4, true, 4, true><<<ntiles, block, 0, st>>>(a, tiles);
  else
    interior_pre_kernel<6, true, 4, true><<<ntiles, block, 0, st>>>(a, tiles);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  split_epilogue_kernel<<<ntiles, block, 0, st>>>(a, tiles);
  return cudaGetLastError();
}
}  // namespace z4c
