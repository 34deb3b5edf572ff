// FP32-RHS split schedule (4): RHS kernel storing k, then the stage-update
// and enforcement kernel.
#include <type_traits>

#include "z4c_interior.cuh"
#include "z4c_tma.cuh"

namespace z4c {

// Schedule 4, second kernel: the RK stage update and the FP64 enforcement of
// the FP32 RHS stored by interior_pre_kernel<..., SPLIT = true> (same tile
// list, same tile order).  Every FP64 operand of the stage (u0 and / or the
// accumulator, 22 values each) and the 22 k values are loaded first, all at
// once, into registers (126 per thread, 4 CTAs per SM): one round trip to
// HBM per cell instead of several.
// The tile's shape s (bits 28..29 of Tile::block; 0 = 16 x 8) sets which
// cell of the (TX << s) x (TY >> s) tile thread tid = y TX + x updates: the
// one the RHS kernel stored at index tid of the tile's k record.
__global__ void __launch_bounds__(TX * TY, 4) split_epilogue_kernel(StageArgs a, const Tile *__restrict__ tiles) {
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
  StageOperands op;
  op.load(a, b.off + cidx, b.S);
  stage_epilogue_preloaded<float>(a, blk, b.off + cidx, b.S, k, op);
}

// The same stage update, persistent and fed by bulk asynchronous copies.
// Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; while it
// updates one tile, the copy engine brings the next tile's k record and its
// u0 / accumulator rows (those the stage reads) into the other of two
// shared-memory stages, so the FP64 arithmetic runs from shared memory
// instead of waiting on HBM with a register file's worth of loads in
// flight.  Requires full tiles (n_x, n_y multiples of the tile's width and
// height) and 16-byte aligned rows: an even ghost width, an even storage
// extent along x and 16-byte aligned registers (the launcher checks).  Every
// wait is bounded: a stage whose copies do not land sets the status word.
constexpr int EPI_K_BYTES = NF * TX * TY * 4;
constexpr int EPI_F_BYTES = NF * TX * TY * 8;
constexpr int EPI_STAGE_BYTES = EPI_K_BYTES + 2 * EPI_F_BYTES;
constexpr int EPI_SMEM = 2 * EPI_STAGE_BYTES + 16;

struct SmemField {
  const double *p;
  __device__ __forceinline__ double operator()(int f) const { return p[f * (TX * TY)]; }
};

__device__ __forceinline__ void epi_issue(const StageArgs &a, const Tile *tiles, int t, unsigned char *stage,
                                          uint64_t *bar, int lane) {
  const Tile T = tiles[t];
  const int shape = T.block >> TILE_SHAPE_SHIFT;
  const DevBlock &b = a.blocks[T.block & TILE_BLOCK_MASK];
  const int txs = TX << shape, tys = TY >> shape;
  const bool use_u0 = a.mode != MODE_S4, use_acc = a.mode != MODE_S1;
  const uint32_t bytes = EPI_K_BYTES + (use_u0 ? EPI_F_BYTES : 0) + (use_acc ? EPI_F_BYTES : 0);
  if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
  __syncwarp();
  if (lane == 0) bulk_g2s(stage, a.kbuf + (int64_t)t * NF * (TX * TY), EPI_K_BYTES, bar);
  const int g = b.g;
  const int nrow = NF * tys;  // (field, row) pairs per array
  for (int q = lane; q < 2 * nrow; q += 32) {
    const int arr = q / nrow, fr = q % nrow, f = fr / tys, jj = fr % tys;
    if ((arr == 0 && !use_u0) || (arr == 1 && !use_acc)) continue;
    const int64_t o = b.off + (int64_t)f * b.S +
                      ((int64_t)(T.k0 + g) * b.e[1] + (T.j0 + jj + g)) * b.e[0] + (T.i0 + g);
    const double *src = (arr == 0 ? a.u0 : a.acc) + o;
    unsigned char *dst = stage + EPI_K_BYTES + arr * EPI_F_BYTES + (f * (TX * TY) + jj * txs) * 8;
    bulk_g2s(dst, src, txs * 8, bar);
  }
}

__global__ void __launch_bounds__(TX * TY, 2) split_epilogue_tma_kernel(StageArgs a, const Tile *__restrict__ tiles,
                                                                       int ntiles) {
  unsigned char *sm = dyn_smem();
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * EPI_STAGE_BYTES);
  const int tid = threadIdx.y * TX + threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid < 32 && (int)blockIdx.x < ntiles) epi_issue(a, tiles, blockIdx.x, sm, &bar[0], tid);
  for (int n = 0;; ++n) {
    const int t = blockIdx.x + n * gridDim.x;
    if (t >= ntiles) break;
    const int s = n & 1;
    // the other stage was last read in iteration n - 1, which every thread
    // has left (barrier at its end): refill it with the next tile
    if (tid < 32 && t + (int)gridDim.x < ntiles) {
      fence_proxy_async_smem();  // the generic reads of that stage before the async writes
      epi_issue(a, tiles, t + gridDim.x, sm + (s ^ 1) * EPI_STAGE_BYTES, &bar[s ^ 1], tid);
    }
    const bool ok = mbar_wait(&bar[s], (n >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      // give the copies in flight a bounded time to land, then stop
      mbar_wait(&bar[s], (n >> 1) & 1, 1u << 16);
      mbar_wait(&bar[s ^ 1], ((n + 1) >> 1) & 1, 1u << 16);
      if (tid == 0 && a.status) atomicOr(a.status, 1);
      return;
    }
    const unsigned char *stg = sm + s * EPI_STAGE_BYTES;
    const Tile T = tiles[t];
    const int shape = T.block >> TILE_SHAPE_SHIFT, blk = T.block & TILE_BLOCK_MASK;
    const DevBlock &b = a.blocks[blk];
    const int i = T.i0 + (tid & ((TX << shape) - 1)), j = T.j0 + (tid >> (4 + shape)), kk = T.k0;
    const int g = b.g;
    const int32_t cidx = ((kk + g) * b.e[1] + (j + g)) * b.e[0] + (i + g);
    const float *ks = reinterpret_cast<const float *>(stg) + tid;
    float k[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) k[f] = ks[f * (TX * TY)];
    const double *su0 = reinterpret_cast<const double *>(stg + EPI_K_BYTES) + tid;
    const double *sacc = reinterpret_cast<const double *>(stg + EPI_K_BYTES + EPI_F_BYTES) + tid;
    stage_epilogue_from<float>(a, blk, b.off + cidx, b.S, k, SmemField{su0}, SmemField{sacc});
    __syncthreads();
  }
}

// Tiles of the list qualify when full and 16-byte aligned (see above).
bool epilogue_tma_ok(const StageArgs &a) {
  return ((uintptr_t)a.u0 % 16 == 0) && ((uintptr_t)a.acc % 16 == 0) && ((uintptr_t)a.kbuf % 16 == 0);
}

cudaError_t launch_split_epilogue_tma(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(split_epilogue_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         EPI_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = ntiles < 2 * nsm ? ntiles : 2 * nsm;
  split_epilogue_tma_kernel<<<grid, dim3(TX, TY), EPI_SMEM, st>>>(a, tiles, ntiles);
  return cudaGetLastError();
}

cudaError_t launch_split_epilogue(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  split_epilogue_kernel<<<ntiles, dim3(TX, TY), 0, st>>>(a, tiles);
  return cudaGetLastError();
}

}  // namespace z4c
