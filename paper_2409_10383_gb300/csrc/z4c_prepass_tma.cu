// FP32 y/z pre-pass (D_y f and D_z f of the eleven fields with mixed second
// derivatives, paper Sec. 2: the second derivatives of the Z4c RHS) walking
// z, fed by TMA tensor copies into a shared-memory ring of plane slabs.
//
// The plane-tiled pre-pass (dydz_kernel) reads each value from L2 about ten
// times: the z-stencil neighbours of a tile live in other CTAs' planes, so no
// L1 keeps them.  Here a CTA of PX x PY threads owns one (x, y) column of the
// widened interior and a group of NQ of the eleven fields, and walks NZ
// planes.  For every storage plane it needs, one thread issues NQ
// cp.async.bulk.tensor copies (one PX x (PY + 2W) box per field, the tile's
// rows with the y halo) into a ring slot; the copy engine stays LA planes
// ahead of the arithmetic.  D_z reads the 2W + 1 slots of the planes around
// the output plane, D_y the rows of its own slot: every shadow value crosses
// from L2 once per CTA, and halo planes are shared by the NZ planes of a
// column.  Field groups keep the ring small (32 KB for NQ = 4, order 6), so
// that 7 CTAs share an SM.
//
// The arithmetic is FD<ORD>::d1 on the same FP32 values as dydz_kernel, in
// the same order, so the stored derivatives are bit-identical to it.
//
// Every mbarrier wait is bounded.  A CTA whose copies do not land waits a
// bounded time for those still in flight, sets the status word and returns.
#include <cuda.h>

#include <type_traits>

#include "z4c_rhs.cuh"
#include "z4c_tma.cuh"

namespace z4c {
namespace {

template <int ORD>
struct PreGeom {
  static constexpr int W = ORD / 2;              // half width of the first derivative
  static constexpr int SR = PRE_TMA_PY + 2 * W;  // rows per field slab
  static constexpr int SLAB = SR * PRE_TMA_PX;   // floats per field slab (one copy)
  static constexpr int NQ = PRE_TMA_NQ;          // fields per CTA (slots q0 .. q0 + NQ - 1)
  static constexpr int PLANE = NQ * SLAB;        // floats per ring slot
  static constexpr int LA = PRE_TMA_LA;          // planes in flight beyond the stencil's
  static constexpr int RING = 2 * W + 1 + LA;
  static constexpr size_t SMEM = sizeof(float) * RING * PLANE + RING * sizeof(uint64_t);
  static_assert((SLAB * sizeof(float)) % 128 == 0, "slabs must stay 128-byte aligned");
};

// field of stored-derivative slot q (the inverse of dslot)
__device__ __forceinline__ int field_of_slot(int q) {
  return q == 0 ? CHI : q <= 6 ? GXX + (q - 1) : q == 7 ? ALPHA : BETAX + (q - 8);
}

// One box of a 4-D tensor map (x, y, z, field) into shared memory; completion
// counted on bar.  x * 4 bytes is a multiple of 16 (the tile's storage x is a
// multiple of PRE_TMA_PX); y may be negative (zero fill, never used).
__device__ __forceinline__ void tma_box4(float *dst, const void *map, int x, int y, int z, int f, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_addr(bar))
      : "memory");
}

// Slab readers for FD<ORD>::d1.  SlabY: the output plane's slot, offsets in
// rows of PX floats.  SlabZ: offset m picks the slot of plane z + m.
struct SlabY {
  const float *p;  // this thread's cell in the field's slab of the output plane
  __device__ __forceinline__ float at(int, int off) const { return p[off]; }
};
template <int W>
struct SlabZ {
  const float *ring;
  int slot[2 * W + 1];  // ring offset (floats) of planes z - W .. z + W
  int cell;             // field slab + this thread's cell
  __device__ __forceinline__ float at(int, int m) const { return ring[slot[m + W] + cell]; }
};

template <int ORD>
__global__ void __launch_bounds__(PRE_TMA_PX *PRE_TMA_PY)
    dydz_tma_kernel(StageArgs a, const Tile *__restrict__ tiles, uint32_t rounds) {
  using G = PreGeom<ORD>;
  constexpr int W = G::W, PX = PRE_TMA_PX;
  float *ring = reinterpret_cast<float *>(dyn_smem());
  uint64_t *bar = reinterpret_cast<uint64_t *>(ring + G::RING * G::PLANE);
  const Tile t = tiles[blockIdx.x];
  const int blk = t.block & TILE_BLOCK_MASK;
  const int q0 = (t.block >> TILE_SHAPE_SHIFT) * G::NQ;   // the CTA's first field slot
  const int nq = min(G::NQ, NDS - q0);
  const DevBlock &b = a.blocks[blk];
  const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(a.tmap32) + blk;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PX + tx;
  const int g = b.g, e0 = b.e[0], e1 = b.e[1];
  const int nz = min(PRE_TMA_NZ, b.n[2] - t.k0);
  const int np = nz + 2 * W;      // planes staged: k0 - W .. k0 + nz - 1 + W
  const int xs = t.i0 + g;        // storage x of the tile (a multiple of PX)
  const int ys = t.j0 + g - W;    // storage y of slab row 0
  const int zs = t.k0 + g - W;    // storage z of staged plane 0

  if (tid == 0) {
    for (int s = 0; s < G::RING; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: plane s into slot s % RING
  auto issue = [&](int s) {
    uint64_t *br = &bar[s % G::RING];
    float *dst = ring + (s % G::RING) * G::PLANE;
    mbar_arrive_expect_tx(br, uint32_t(nq * G::SLAB * sizeof(float)));
#pragma unroll 1
    for (int q = 0; q < nq; ++q) tma_box4(dst + q * G::SLAB, map, xs, ys, zs + s, field_of_slot(q0 + q), br);
  };
  int issued = min(np, G::RING);
  if (tid == 0)
    for (int s = 0; s < issued; ++s) issue(s);

  const int i = t.i0 + tx, j = t.j0 + ty;
  const bool in_x = i >= 0 && i < b.n[0], in_y = j >= 0 && j < b.n[1];
  const bool wide_x = i >= -W && i < b.n[0] + W, wide_y = j >= -W && j < b.n[1] + W;
  const bool need_dy = in_y && wide_x;
  const bool need_dz = (in_y && wide_x) || (in_x && wide_y);
  const float s1 = b.s1f;
  const int cell = (ty + W) * PX + tx;  // this thread's cell in a field slab
  float *out = reinterpret_cast<float *>(a.dstore) + b.off;
  int waited = 0;  // planes [0, waited) have landed

#pragma unroll 1
  for (int o = 0; o < nz; ++o) {
    bool ok = true;
    for (; waited <= o + 2 * W; ++waited) ok = ok && mbar_wait(&bar[waited % G::RING], (waited / G::RING) & 1, rounds);
    if (__syncthreads_or(!ok)) {
      // give every copy still in flight a bounded time to land, then stop
      if (tid == 0) {
        // each slot holds at most one plane in flight: the last RING issued
        for (int s = max(0, issued - G::RING); s < issued; ++s)
          mbar_wait(&bar[s % G::RING], (s / G::RING) & 1, 1u << 16);
        if (a.status) atomicOr(a.status, 1);
      }
      __syncthreads();
      return;
    }
    if (need_dz) {
      const int kk = t.k0 + o;
      const int64_t c = ((int64_t)(kk + g) * e1 + (j + g)) * e0 + (i + g);
      SlabZ<W> sz{ring, {}, cell};
#pragma unroll
      for (int m = 0; m <= 2 * W; ++m) sz.slot[m] = ((o + m) % G::RING) * G::PLANE;
      const float *cur = ring + sz.slot[W] + cell;
#pragma unroll
      for (int q = 0; q < G::NQ; ++q) {
        if (q >= nq) break;
        if (need_dy) out[(int64_t)(q0 + q) * b.S + c] = FD<ORD>::d1(SlabY{cur + q * G::SLAB}, 0, PX) * s1;
        SlabZ<W> zq = sz;
        zq.cell = cell + q * G::SLAB;
        out[(int64_t)(q0 + q + NDS) * b.S + c] = FD<ORD>::d1(zq, 0, 1) * s1;
      }
    }
    // every thread is done with plane o: its slot takes plane o + RING
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && issued < np) issue(issued);
    if (issued < np) ++issued;
  }
}

template <int ORD>
cudaError_t go(const StageArgs &a, const Tile *tiles, int n, uint32_t rounds, cudaStream_t st) {
  constexpr size_t smem = PreGeom<ORD>::SMEM;
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(dydz_tma_kernel<ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dydz_tma_kernel<ORD><<<n, dim3(PRE_TMA_PX, PRE_TMA_PY), smem, st>>>(a, tiles, rounds);
  return cudaGetLastError();
}

}  // namespace

bool prepass_tma_built(int order) { return order == 4 || order == 6; }

cudaError_t launch_prepass_tma_f32(int order, const StageArgs &a, const Tile *ztiles, int n, cudaStream_t st,
                                   uint32_t rounds) {
  if (n <= 0) return cudaSuccess;
  if (order == 6) return go<6>(a, ztiles, n, rounds, st);
  if (order == 4) return go<4>(a, ztiles, n, rounds, st);
  return cudaErrorInvalidValue;
}

}  // namespace z4c
