// FP32-RHS split schedule (4): RHS kernel storing k, then the stage-update
// and enforcement kernel.
#include <type_traits>

#include "z4c_interior.cuh"

namespace z4c {

// Schedule 4, second kernel: the RK stage update and the FP64 enforcement of
// the FP32 RHS stored by interior_pre_kernel<..., SPLIT = true> (same tile
// list, same tile order).  Few registers, so many warps hide the latency of
// the FP64 state loads.
// The tile's shape s (bits 28..29 of Tile::block; 0 = 16 x 8) sets which
// cell of the (TX << s) x (TY >> s) tile thread tid = y TX + x updates: the
// one the RHS kernel stored at index tid of the tile's k record.
__global__ void __launch_bounds__(TX * TY, 8) split_epilogue_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  const Tile t = tiles[blockIdx.x];
  const int shape = t.block >> TILE_SHAPE_SHIFT, blk = t.block & TILE_BLOCK_MASK;
  const DevBlock &b = a.blocks[blk];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int i = t.i0 + (tid & ((TX << shape) - 1)), j = t.j0 + (tid >> (4 + shape)), kk = t.k0;
  if (i >= b.n[0] || j >= b.n[1]) return;
  const int g = b.g;
  const int32_t cidx = ((kk + g) * b.e[1] + (j + g)) * b.e[0] + (i + g);
  const float *kt = a.kbuf + (int64_t)blockIdx.x * NF * (TX * TY) + tid;
  float k[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) k[f] = kt[f * (TX * TY)];
  stage_epilogue<float>(a, blk, b.off + cidx, b.S, k);
}

cudaError_t launch_split_epilogue(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  split_epilogue_kernel<<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}

}  // namespace z4c
