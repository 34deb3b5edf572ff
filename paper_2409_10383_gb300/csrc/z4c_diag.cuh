// Diagnostics beside the RK4 step (paper Sec. 3.2: refinement criteria on
// chi; Sec. 3.3: puncture trackers and the Weyl scalar Psi4), FP64.
// Launchers in z4c_diag.cu.
#pragma once

#include "z4c_rhs.cuh"

namespace z4c {

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Per tile (TX x TY cells of one z-plane): min chi and max |grad chi| over
// its interior cells, the gradient by the block's centred first-derivative
// stencil; part[2 t] = min, part[2 t + 1] = max.
__global__ void __launch_bounds__(TX * TY) indicator_tile_kernel(const double *__restrict__ u,
                                                                 const DevBlock *__restrict__ blocks,
                                                                 const Tile *__restrict__ tiles,
                                                                 double *__restrict__ part) {
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = blocks[t.block];
  const int i = t.i0 + threadIdx.x, j = t.j0 + threadIdx.y, kk = t.k0;
  double mn = INFINITY, mx = 0.0;
  if (i < b.n[0] && j < b.n[1]) {
    const int g = b.g, e0 = b.e[0], e1 = b.e[1];
    const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
    const int st[3] = {1, e0, e0 * e1};
    const Src<double, false> s{u + b.off, cidx, b.S};
    mn = s.at(CHI, 0);
    double sq = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double q = (b.order == 2   ? FD<2>::d1(s, CHI, st[d])
                        : b.order == 4 ? FD<4>::d1(s, CHI, st[d])
                                       : FD<6>::d1(s, CHI, st[d])) *
                       b.s1;
      sq = fma(q, q, sq);
    }
    mx = sqrt(sq);
  }
  __shared__ double red[2][TX * TY / 32];
  const int tid = threadIdx.y * TX + threadIdx.x, lane = tid & 31, warp = tid >> 5;
  mn = warp_min_d(mn);
  mx = warp_max_d(mx);
  if (lane == 0) {
    red[0][warp] = mn;
    red[1][warp] = mx;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < TX * TY / 32; ++w) {
      mn = fmin(mn, red[0][w]);
      mx = fmax(mx, red[1][w]);
    }
    part[2 * (int64_t)blockIdx.x] = mn;
    part[2 * (int64_t)blockIdx.x + 1] = mx;
  }
}

// Per block: min / max over its tiles [first[b], first[b + 1]) of the tile
// list; out[b] = min chi, out[nb + b] = max |grad chi|.
__global__ void indicator_block_kernel(const double *__restrict__ part, const int32_t *__restrict__ first, int nb,
                                       double *__restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double mn = INFINITY, mx = 0.0;
  for (int t = first[b]; t < first[b + 1]; ++t) {
    mn = fmin(mn, part[2 * (int64_t)t]);
    mx = fmax(mx, part[2 * (int64_t)t + 1]);
  }
  out[b] = mn;
  out[nb + b] = mx;
}

// One tracker step per puncture (one thread each): beta at xw by 4-point
// Lagrange interpolation per axis over the cell centres i0 .. i0 + 3,
// i0 = floor((x - lo)/h - 1/2) - 1; out[6 q + d] = x0[d] - dt beta[d],
// out[6 q + 3 + d] = beta[d].
__global__ void track_kernel(const double *__restrict__ u, const DevBlock *__restrict__ blocks,
                             const TrackIn *__restrict__ in, int np, double dt, double *__restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const TrackIn p = in[q];
  const DevBlock &b = blocks[p.block];
  int s0[3];
  double w[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int i0 = (int)floor((p.xw[d] - b.lo[d]) / b.h - 0.5) - 1;
    s0[d] = i0 + b.g;
    double xs[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xs[a] = b.lo[d] + (i0 + a + 0.5) * b.h;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double v = 1.0;
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if (m != a) v *= (p.xw[d] - xs[m]) / (xs[a] - xs[m]);
      w[d][a] = v;
    }
  }
  const int e0 = b.e[0], e1 = b.e[1];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double *f = u + b.off + (int64_t)(BETAX + c) * b.S;
    double v = 0.0;
    for (int kz = 0; kz < 4; ++kz)
      for (int jy = 0; jy < 4; ++jy)
        for (int ix = 0; ix < 4; ++ix)
          v += w[2][kz] * w[1][jy] * w[0][ix] * f[((s0[2] + kz) * e1 + s0[1] + jy) * e0 + s0[0] + ix];
    out[6 * q + c] = p.x0[c] - dt * v;
    out[6 * q + 3 + c] = v;
  }
}

// Psi4 (psi4_point) at every interior cell of the blocks of order ORD, one
// thread per cell over the interior tiles; out holds per block the real part
// and then the imaginary part over the block's storage cells (offset
// 2 off / NF), other cells untouched.  The y/z first derivatives of the
// eleven fields with mixed second derivatives come from ds (the FP64
// pre-pass arrays of u, as in the RHS); every other stencil reads u.
template <int ORD>
__global__ void __launch_bounds__(TX * TY) psi4_kernel(const double *__restrict__ u,
                                                       const DevBlock *__restrict__ blocks,
                                                       const Tile *__restrict__ tiles, const double *__restrict__ ds,
                                                       double *__restrict__ out) {
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = blocks[t.block];
  const int i = t.i0 + threadIdx.x, j = t.j0 + threadIdx.y, kk = t.k0;
  if (b.order != ORD || i >= b.n[0] || j >= b.n[1]) return;
  const int g = b.g, e0 = b.e[0], e1 = b.e[1];
  const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
  const int st[3] = {1, e0, e0 * e1};
  const Src<double, false> s{u + b.off, cidx, b.S};
  const Scales<double> sc = scales_of(b, 0.0);
  const double ichi = 1.0 / fmax(s.at(CHI, 0), b.chi_floor);
  const double x[3] = {b.lo[0] + (i + 0.5) * b.h, b.lo[1] + (j + 0.5) * b.h, b.lo[2] + (kk + 0.5) * b.h};
  double v[2];
  const Src<double, false> d{ds + b.off, cidx, b.S};
  const Pre<ORD, double, Src<double, false>, Src<double, false>> dv{s, d, st, sc};
  psi4_point<ORD>(s, dv, ichi, x, v);
  double *o = out + b.off / NF * 2 + cidx;
  o[0] = v[0];
  o[b.S] = v[1];
}

}  // namespace z4c
