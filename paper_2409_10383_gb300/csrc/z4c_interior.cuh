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
  const double chig = fmax(a.x64[off], b.chi_floor);
  const R ichi = R(1.0 / chig);
  const Phys<R> p{R(b.kappa1), R(b.kappa2), R(b.eta), b.lapse, b.shift};
  R k[NF];
  if constexpr (F32) {
    const Src<float, true> s{a.x32 + off, b.S};
    rhs_point<ORD, float>(s, st, scales_of(b, 0.0f), p, ichi, k);
  } else {
    const Src<double, false> s{a.x64 + off, b.S};
    rhs_point<ORD, double>(s, st, scales_of(b, 0.0), p, ichi, k);
  }
  stage_epilogue<R>(a, off, b.S, k);
}

}  // namespace z4c
