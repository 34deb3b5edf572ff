// Fused interior stage kernel: Z4c RHS at every interior cell of a tile,
// followed by the RK4 stage update and the algebraic constraint enforcement
// (paper Sec. 3: the RK stage of each MeshBlock; Sec. 2: Z4c RHS).
// One thread per cell, TX x TY cells of one z-plane per CTA; tiles come
// from a work list so blocks of any size (and several blocks per launch,
// the paper's MeshBlockPack) share one launch.
#pragma once

#include "z4c_rhs.cuh"
#include "z4c_tma.cuh"

namespace z4c {

template <int ORD, bool F32>
__global__ void __launch_bounds__(TX * TY) interior_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  using R = typename std::conditional<F32, float, double>::type;
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = a.blocks[t.block];
  const int i = t.i0 + threadIdx.x, j = t.j0 + threadIdx.y, kk = t.k0;
  if (i >= b.n[0] || j >= b.n[1]) return;
  const int g = b.g, e0 = b.e[0], e1 = b.e[1];
  const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
  const int st[3] = {1, e0, e0 * e1};
  const int64_t off = b.off + cidx;
  // 1/chi with the chi floor, always in FP64
  // 1/max(chi, chi_floor), always from the FP64 stage state
  R ichi;
  if constexpr (F32)
    ichi = inv_chi_f32(a.x64[off], b.chi_floor);
  else
    ichi = 1.0 / fmax(a.x64[off], b.chi_floor);
  const Phys<R> p{R(b.kappa1), R(b.kappa2), R(b.eta), b.lapse, b.shift};
  R k[NF];
  if constexpr (F32) {
    const Src<float, true> s{a.x32 + b.off, cidx, b.S};
    const Scales<float> sc = scales_of(b, 0.0f);
    const Direct<ORD, float, Src<float, true>> dv{s, st, sc};
    rhs_point<ORD, float>(s, dv, st, sc, p, ichi, k);
  } else {
    const Src<double, false> s{a.x64 + b.off, cidx, b.S};
    const Scales<double> sc = scales_of(b, 0.0);
    const Direct<ORD, double, Src<double, false>> dv{s, st, sc};
    rhs_point<ORD, double>(s, dv, st, sc, p, ichi, k);
  }
  stage_epilogue<R>(a, t.block, off, b.S, k);
}


// Pre-pass: D_y f and D_z f (times s1) of the eleven fields with mixed
// second derivatives, into the stored-derivative arrays (same layout as a
// register, 22 arrays per block).  D_y f is needed where the cell row is
// interior in y and within W = ORD/2 cells of the interior in x; D_z f on
// that region plus the one interior in x and within W of the interior in y.
// Tiles (a separate list) cover the interior widened by W in x and y.
template <int ORD, bool F32>
__global__ void __launch_bounds__(TX * TY) dydz_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int W = ORD / 2;
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = a.blocks[t.block];
  const int i = t.i0 + threadIdx.x, j = t.j0 + threadIdx.y, kk = t.k0;
  if constexpr (F32) {
    // into L2: the whole storage rows of this tile's rows of the eleven
    // fields PF_PRE planes ahead, from the first tile of the row band
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (t.i0 == -W && tid < NF && dslot(tid) >= 0)
      prefetch_rows<float>(a.x32, tid, b.S, kk + b.g + PF_PRE, t.j0 + b.g, t.j0 + b.g + TY, b.e[0], b.e[1], b.e[2],
                           b.off);
  }
  const bool in_x = i >= 0 && i < b.n[0], in_y = j >= 0 && j < b.n[1];
  const bool wide_x = i >= -W && i < b.n[0] + W, wide_y = j >= -W && j < b.n[1] + W;
  const bool need_dy = in_y && wide_x;
  const bool need_dz = (in_y && wide_x) || (in_x && wide_y);
  if (!need_dz) return;
  const int g = b.g, e0 = b.e[0], e1 = b.e[1];
  const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
  const int64_t off = b.off + cidx;
  R *out = reinterpret_cast<R *>(a.dstore) + off;
  const R s1 = F32 ? R(b.s1f) : R(b.s1);
  const int sy = e0, sz = e0 * e1;
  if constexpr (F32) {
    const Src<float, true> s{a.x32 + b.off, cidx, b.S};
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (dslot(f) < 0) continue;
      if (need_dy) out[(int64_t)dslot(f) * b.S] = FD<ORD>::d1(s, f, sy) * s1;
      out[(int64_t)(dslot(f) + NDS) * b.S] = FD<ORD>::d1(s, f, sz) * s1;
    }
  } else {
    const Src<double, false> s{a.x64 + b.off, cidx, b.S};
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (dslot(f) < 0) continue;
      if (need_dy) out[(int64_t)dslot(f) * b.S] = FD<ORD>::d1(s, f, sy) * s1;
      out[(int64_t)(dslot(f) + NDS) * b.S] = FD<ORD>::d1(s, f, sz) * s1;
    }
  }
}

// Interior stage kernel taking the y/z first derivatives and the mixed
// second derivatives of the eleven fields from the pre-pass arrays.
// OCC = minimum resident CTAs per SM the register allocation must allow
// (1: up to 255 registers per thread; 4: 128), chosen by the autotuner.
// SPLIT (FP32 only): store k in a.kbuf for split_epilogue_kernel instead of
// applying the stage update here (k of tile blockIdx.x at kbuf + blockIdx.x
// NF TX TY; the launcher offsets kbuf for a sub-range of a tile list).
// EXT > 0: every block of the launch has cubic storage EXT^3 (n + 2g = EXT
// along all axes), so all stencil offsets are compile-time constants.
// SHAPE (SPLIT only): tiles of (TX << SHAPE) x (TY >> SHAPE) cells; thread
// tid = y TX + x takes cell (tid % (TX << SHAPE), tid / (TX << SHAPE)), so
// a warp covers one row of 32 cells (SHAPE >= 1) instead of two of 16.
template <int ORD, bool F32, int OCC, bool SPLIT = false, int EXT = 0, int SHAPE = 0>
__global__ void __launch_bounds__(TX * TY, OCC) interior_pre_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  using R = typename std::conditional<F32, float, double>::type;
  static_assert(SHAPE == 0 || SPLIT, "tile shapes other than 16 x 8 are for the split RHS kernel");
  constexpr int TXS = TX << SHAPE;
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = a.blocks[t.block & TILE_BLOCK_MASK];
  const int tid0 = threadIdx.y * TX + threadIdx.x;
  const int i = t.i0 + (SHAPE ? tid0 % TXS : (int)threadIdx.x), j = t.j0 + (SHAPE ? tid0 / TXS : (int)threadIdx.y);
  const int kk = t.k0;
  const int e0 = EXT > 0 ? EXT : b.e[0], e1 = EXT > 0 ? EXT : b.e[1];
  const int32_t S = EXT > 0 ? EXT * EXT * EXT : b.S;
  if constexpr (F32 && SPLIT) {
    // into L2: the shadow fields and stored derivatives of this tile's rows
    // PF_RHS planes ahead (with the ghost rows at the y edges)
    constexpr int ROWS = TY >> SHAPE;
    if (tid0 < 2 * NF)
      prefetch_rows<float>(tid0 < NF ? a.x32 : reinterpret_cast<const float *>(a.dstore), tid0 % NF, S,
                           kk + b.g + PF_RHS, t.j0 == 0 ? 0 : t.j0 + b.g,
                           t.j0 + ROWS >= b.n[1] ? e1 : t.j0 + b.g + ROWS, e0, e1, EXT > 0 ? EXT : b.e[2], b.off);
  }
  if (i >= b.n[0] || j >= b.n[1]) return;
  const int g = b.g;
  const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
  const int st[3] = {1, e0, e0 * e1};
  const int64_t off = b.off + cidx;
  // 1/max(chi, chi_floor), always from the FP64 stage state
  R ichi;
  if constexpr (F32)
    ichi = inv_chi_f32(a.x64[off], b.chi_floor);
  else
    ichi = 1.0 / fmax(a.x64[off], b.chi_floor);
  const Phys<R> p{R(b.kappa1), R(b.kappa2), R(b.eta), b.lapse, b.shift};
  R k[NF];
  const Src<R, false> ds{reinterpret_cast<const R *>(a.dstore) + b.off, cidx, S};
  if constexpr (F32) {
    const Src<float, true> s{a.x32 + b.off, cidx, S};
    const Scales<float> sc = scales_of(b, 0.0f);
    const Pre<ORD, float, Src<float, true>, Src<float, false>> dv{s, ds, st, sc};
    rhs_point<ORD, float>(s, dv, st, sc, p, ichi, k);
    if constexpr (SPLIT) {
      float *kt = a.kbuf + (int64_t)blockIdx.x * NF * (TX * TY) + tid0;
#pragma unroll
      for (int f = 0; f < NF; ++f) kt[f * (TX * TY)] = k[f];
      return;
    }
  } else {
    const Src<double, false> s{a.x64 + b.off, cidx, S};
    const Scales<double> sc = scales_of(b, 0.0);
    const Pre<ORD, double, Src<double, false>, Src<double, false>> dv{s, ds, st, sc};
    rhs_point<ORD, double>(s, dv, st, sc, p, ichi, k);
  }
  stage_epilogue<R>(a, t.block, off, S, k);
}

// FP32-RHS split-schedule RHS kernel computing two neighbouring cells of a
// row per thread on the packed f32x2 instructions (F2), on tiles of shape
// SHAPE: (TX << SHAPE) x (TY >> SHAPE) cells (1: 32 x 4, 2: 64 x 2), 64
// threads; thread (tx, ty) owns cells (i0 + 2 tx, i0 + 2 tx + 1) of row
// j0 + ty, so a warp covers 32 (SHAPE 1: two rows) or 64 cells of a row.
// The same stencils, pre-pass derivatives and algebra as
// interior_pre_kernel<ORD, true, 4, true, EXT>; a warp's loads of a stencil
// point touch few cache lines, and the pair shares its x stencil loads.
// Requires an even storage extent, an even ghost width and n_x a multiple
// of the tile width (the host checks; every cell pair then starts 8-byte
// aligned).  Stores k in a.kbuf like the split RHS kernel, cell (ii, jj) of
// the tile at jj * (TX << SHAPE) + ii.
template <int ORD, int EXT, int SHAPE>
__global__ void __launch_bounds__(TX * TY / 2, 4) interior_pair_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  static_assert(EXT > 0 && EXT % 2 == 0, "pair kernel needs an even compile-time extent");
  constexpr int TXS = TX << SHAPE;
  const Tile t = tiles[blockIdx.x];
  const int blk = t.block & TILE_BLOCK_MASK;
  const DevBlock &b = a.blocks[blk];
  const int i = t.i0 + 2 * threadIdx.x, j = t.j0 + threadIdx.y, kk = t.k0;
  constexpr int e0 = EXT, e1 = EXT;
  constexpr int32_t S = EXT * EXT * EXT;
  {
    // into L2: the shadow fields and stored derivatives of this tile's rows
    // PF_RHS planes ahead (with the ghost rows at the y edges)
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid < 2 * NF)
      prefetch_rows<float>(tid < NF ? a.x32 : reinterpret_cast<const float *>(a.dstore), tid % NF, S,
                           kk + b.g + PF_RHS, t.j0 == 0 ? 0 : t.j0 + b.g,
                           t.j0 + (TY >> SHAPE) >= b.n[1] ? e1 : t.j0 + b.g + (TY >> SHAPE), e0, e1, EXT, b.off);
  }
  if (i >= b.n[0] || j >= b.n[1]) return;
  const int g = b.g;
  const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
  const int st[3] = {1, e0, e0 * e1};
  const int64_t off = b.off + cidx;
  const F2 ichi(inv_chi_f32(a.x64[off], b.chi_floor), inv_chi_f32(a.x64[off + 1], b.chi_floor));
  const Phys<F2> p{F2(b.kappa1), F2(b.kappa2), F2(b.eta), b.lapse, b.shift};
  const Scales<F2> sc{F2(b.s1f), F2(b.s2f), F2(b.smixf), F2(b.slopf), F2(b.skof)};
  const SrcPair<true> s{a.x32 + b.off, cidx, S};
  const SrcPair<false> ds{reinterpret_cast<const float *>(a.dstore) + b.off, cidx, S};
  const Pre<ORD, F2, SrcPair<true>, SrcPair<false>> dv{s, ds, st, sc};
  F2 k[NF];
  rhs_point<ORD, F2>(s, dv, st, sc, p, ichi, k);
  float *kt = a.kbuf + (int64_t)blockIdx.x * NF * (TX * TY) + threadIdx.y * TXS + 2 * threadIdx.x;
#pragma unroll
  for (int f = 0; f < NF; ++f) *reinterpret_cast<float2 *>(kt + f * (TX * TY)) = k[f].v;
}

}  // namespace z4c
