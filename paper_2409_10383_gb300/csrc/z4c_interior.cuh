// Fused interior stage kernel: Z4c RHS at every interior cell of a tile,
// followed by the RK4 stage update and the algebraic constraint enforcement
// (paper Sec. 3: the RK stage of each MeshBlock; Sec. 2: Z4c RHS).
// One thread per cell, TX x TY cells of one z-plane per CTA; tiles come
// from a work list so blocks of any size (and several blocks per launch,
// the paper's MeshBlockPack) share one launch.
#pragma once

#include "z4c_rhs.cuh"

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
template <int ORD, bool F32, int OCC, bool SPLIT = false, int EXT = 0>
__global__ void __launch_bounds__(TX * TY, OCC) interior_pre_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  using R = typename std::conditional<F32, float, double>::type;
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = a.blocks[t.block];
  const int i = t.i0 + threadIdx.x, j = t.j0 + threadIdx.y, kk = t.k0;
  if (i >= b.n[0] || j >= b.n[1]) return;
  const int g = b.g;
  const int e0 = EXT > 0 ? EXT : b.e[0], e1 = EXT > 0 ? EXT : b.e[1];
  const int32_t S = EXT > 0 ? EXT * EXT * EXT : b.S;
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
      float *kt = a.kbuf + (int64_t)blockIdx.x * NF * (TX * TY) + threadIdx.y * TX + threadIdx.x;
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

}  // namespace z4c
