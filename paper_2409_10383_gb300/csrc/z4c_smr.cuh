// Mesh-refinement ghost transfer kernels (paper Sec. 3.1): restriction by
// 5-point Lagrange interpolation per axis (3D tensor product) over fine
// active cells, and prolongation by 5-point Lagrange interpolation per axis
// from a coarse buffer.  Both are evaluated separably (x, then y, then z).
// One thread per (list entry, field), entries fastest: the threads of a warp
// work on neighbouring entries of one field, so their stencils overlap in
// memory and the loads coalesce.  FP64 registers.  Launchers in z4c_smr.cu.
#pragma once

#include "z4c_internal.cuh"

namespace z4c {

__global__ void restrict_kernel(double *__restrict__ reg, const DevBlock *__restrict__ blocks,
                                const RestrictRef *__restrict__ list, int n, const double *__restrict__ wtab,
                                int to_buffer, double *__restrict__ cb, int ncb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NF) return;
  const int e = t % n, f = t / n;
  const RestrictRef r = list[e];
  const DevBlock &F = blocks[r.src];
  const int e0 = F.e[0], e01 = F.e[0] * F.e[1];
  const double *src = reg + F.off + (int64_t)f * F.S + r.s;
  const double *wx = wtab + 5 * r.wp[0], *wy = wtab + 5 * r.wp[1], *wz = wtab + 5 * r.wp[2];
  double v = 0.0;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double vy = 0.0;
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const double *row = src + c * e01 + b * e0;
      double vx = 0.0;
#pragma unroll
      for (int a = 0; a < 5; ++a) vx = fma(wx[a], __ldg(row + a), vx);
      vy = fma(wy[b], vx, vy);
    }
    v = fma(wz[c], vy, v);
  }
  if (to_buffer) {
    cb[(int64_t)f * ncb + r.didx] = v;
  } else {
    const DevBlock &D = blocks[r.dst];
    reg[D.off + (int64_t)f * D.S + r.didx] = v;
  }
}

// Restriction of every coarse cell of one fine block (blockIdx.x indexes
// rblocks) for one field (blockIdx.y), by three passes over the block's
// active cells staged in shared memory: x, then y, then z, each the 5-point
// Lagrange sum with the same start rule, weights and evaluation order as
// restrict_kernel, so the results are identical; a coarse cell's x-pass
// partial sums are shared by every coarse cell in its (y, z) neighbourhood.
// krow[key + 4] = wtab row of the weight pattern key = start - 2c.
__global__ void __launch_bounds__(256) restrict_block_kernel(const double *__restrict__ reg,
                                                             const DevBlock *__restrict__ blocks,
                                                             const int32_t *__restrict__ rblocks,
                                                             const double *__restrict__ wtab,
                                                             const int32_t *__restrict__ krow,
                                                             double *__restrict__ rb) {
  __shared__ double fine[RB_NMAX * RB_NMAX * RB_NMAX];       // then the y-pass output
  __shared__ double rx[RB_NMAX * RB_NMAX * (RB_NMAX / 2)];   // x-pass output
  const DevBlock &B = blocks[rblocks[blockIdx.x]];
  const int f = blockIdx.y;
  const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const int g = B.g, e0 = B.e[0], e1 = B.e[1];
  const double *src = reg + B.off + (int64_t)f * B.S;
  // 5-point window start s of coarse cell c and its krow index; with 2
  // ghosts the 3-point stencil from 2c (lower half) or 2c-1 (upper half),
  // clamped into the block, at offset off inside the window
  const bool np3 = B.g == 2;
  auto start = [np3](int c, int n, int &kr) {
    const int nc = n / 2;
    if (!np3) {
      int s = c < nc / 2 ? 2 * c - 1 : 2 * c - 2;
      s = s < 0 ? 0 : s > n - 5 ? n - 5 : s;
      kr = s - 2 * c + 4;
      return s;
    }
    int s3 = c < nc / 2 ? 2 * c : 2 * c - 1;
    s3 = s3 < 0 ? 0 : s3 > n - 3 ? n - 3 : s3;
    const int s = s3 - 1 < 0 ? 0 : s3 - 1 > n - 5 ? n - 5 : s3 - 1;
    kr = 8 + 3 * (s - 2 * c + 4) + (s3 - s);
    return s;
  };
  for (int q = threadIdx.x; q < nx * ny * nz; q += blockDim.x) {
    const int i = q % nx, j = (q / nx) % ny, k = q / (nx * ny);
    fine[q] = src[((k + g) * e1 + (j + g)) * e0 + (i + g)];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < cx * ny * nz; q += blockDim.x) {  // (c_x, j, k)
    const int c = q % cx, jk = q / cx;
    int kr;
    const int s = start(c, nx, kr);
    const double *w = wtab + 5 * krow[kr];
    const double *row = fine + jk * nx + s;
    double v = 0.0;
#pragma unroll
    for (int a = 0; a < 5; ++a) v = fma(w[a], row[a], v);
    rx[q] = v;
  }
  __syncthreads();
  double *ry = fine;
  for (int q = threadIdx.x; q < cx * cy * nz; q += blockDim.x) {  // (c_x, c_y, k)
    const int c0 = q % cx, c = (q / cx) % cy, k = q / (cx * cy);
    int kr;
    const int s = start(c, ny, kr);
    const double *w = wtab + 5 * krow[kr];
    double v = 0.0;
#pragma unroll
    for (int b = 0; b < 5; ++b) v = fma(w[b], rx[(k * ny + s + b) * cx + c0], v);
    ry[q] = v;
  }
  __syncthreads();
  double *out = rb + ((int64_t)blockIdx.x * NF + f) * RB_NC3;
  for (int q = threadIdx.x; q < cx * cy * cz; q += blockDim.x) {  // (c_x, c_y, c_z)
    const int cxy = q % (cx * cy), c = q / (cx * cy);
    int kr;
    const int s = start(c, nz, kr);
    const double *w = wtab + 5 * krow[kr];
    double v = 0.0;
#pragma unroll
    for (int cc = 0; cc < 5; ++cc) v = fma(w[cc], ry[(s + cc) * cx * cy + cxy], v);
    out[q] = v;
  }
}

// Scatter of block-restricted values to coarse ghost cells and coarse-buffer
// slots; one thread per (entry, field), entries fastest.
__global__ void rb_scatter_kernel(double *__restrict__ reg, const DevBlock *__restrict__ blocks,
                                  const RbCopy *__restrict__ list, int n, const double *__restrict__ rb,
                                  double *__restrict__ cb, int ncb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NF) return;
  const int e = t % n, f = t / n;
  const RbCopy r = list[e];
  const double v = rb[((int64_t)r.rb * NF + f) * RB_NC3 + r.ci];
  if (r.dst >= 0) {
    const DevBlock &D = blocks[r.dst];
    reg[D.off + (int64_t)f * D.S + r.didx] = v;
  } else {
    cb[(int64_t)f * ncb + r.didx] = v;
  }
}

__global__ void cb_copy_kernel(const double *__restrict__ reg, const DevBlock *__restrict__ blocks,
                               const CbCopy *__restrict__ list, int n, double *__restrict__ cb, int ncb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const CbCopy c = list[t];
  const DevBlock &S = blocks[c.src];
#pragma unroll
  for (int f = 0; f < NF; ++f) cb[(int64_t)f * ncb + c.slot] = reg[S.off + (int64_t)f * S.S + c.scidx];
}

// pw[(5 * c + a)]: weight of the a-th of the 5 coarse points for child c
// (0: offset -1/4, 1: +1/4) with stencil shift code s (shift + 2) at
// pw + 10 * s; the 3-point stencils of 2 ghosts (zero weights on two of the
// five points) at pw + 50 + 10 * s
__global__ void prolong_kernel(double *__restrict__ reg, const DevBlock *__restrict__ blocks,
                               const ProlongRef *__restrict__ list, int n, const int32_t *__restrict__ idx,
                               const double *__restrict__ cb, int ncb, const double *__restrict__ pw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NF) return;
  const int e = t % n, f = t / n;
  const ProlongRef p = list[e];
  const int32_t *ix = idx + e;  // slot q of entry e at ix[q * n]
  const double *cf = cb + (int64_t)f * ncb;
  double wx[2][5], wy[2][5], wz[2][5];
  {
    const double *pb = pw + 50 * ((p.mask >> PROLONG_NP3_BIT) & 1);
    const double *px = pb + 10 * ((p.mask >> PROLONG_SHIFT_BIT) & 7);
    const double *py = pb + 10 * ((p.mask >> (PROLONG_SHIFT_BIT + 3)) & 7);
    const double *pz = pb + 10 * ((p.mask >> (PROLONG_SHIFT_BIT + 6)) & 7);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      wx[q / 5][q % 5] = px[q];
      wy[q / 5][q % 5] = py[q];
      wz[q / 5][q % 5] = pz[q];
    }
  }
  double acc[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};  // [z child][y child][x child]
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double ry[2][2] = {{0, 0}, {0, 0}};  // [y child][x child]
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      double rx[2] = {0, 0};
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        const double v = __ldg(cf + __ldg(ix + (int64_t)((c * 5 + b) * 5 + a) * n));
        rx[0] = fma(wx[0][a], v, rx[0]);
        rx[1] = fma(wx[1][a], v, rx[1]);
      }
#pragma unroll
      for (int yc = 0; yc < 2; ++yc) {
        ry[yc][0] = fma(wy[yc][b], rx[0], ry[yc][0]);
        ry[yc][1] = fma(wy[yc][b], rx[1], ry[yc][1]);
      }
    }
#pragma unroll
    for (int zc = 0; zc < 2; ++zc)
#pragma unroll
      for (int yc = 0; yc < 2; ++yc) {
        acc[zc][yc][0] = fma(wz[zc][c], ry[yc][0], acc[zc][yc][0]);
        acc[zc][yc][1] = fma(wz[zc][c], ry[yc][1], acc[zc][yc][1]);
      }
  }
  const DevBlock &D = blocks[p.dst];
  double *out = reg + D.off + (int64_t)f * D.S + p.cidx0;
  const int e0 = D.e[0], e01 = D.e[0] * D.e[1];
#pragma unroll
  for (int zc = 0; zc < 2; ++zc)
#pragma unroll
    for (int yc = 0; yc < 2; ++yc)
#pragma unroll
      for (int xc = 0; xc < 2; ++xc)
        if (p.mask >> (xc + 2 * yc + 4 * zc) & 1) out[zc * e01 + yc * e0 + xc] = acc[zc][yc][xc];
}

// Prolongation of whole ghost regions (one CTA per box and field): the box's
// coarse values gathered into shared memory, then x, y and z passes of the
// 5-point Lagrange sums; the x-pass partial sums are shared by every fine
// cell with the same x, the y-pass ones by every fine cell with the same
// (x, y).  Per fine cell the same weights, stencil shift and evaluation order
// as prolong_kernel, so the values are identical.
__global__ void __launch_bounds__(128) prolong_box_kernel(double *__restrict__ reg,
                                                          const DevBlock *__restrict__ blocks,
                                                          const PBox *__restrict__ boxes,
                                                          const int32_t *__restrict__ slots,
                                                          const int32_t *__restrict__ axtab,
                                                          const double *__restrict__ cb, int ncb,
                                                          const double *__restrict__ pw) {
  __shared__ double CY[PB_Y > PB_C ? PB_Y : PB_C];  // coarse box, then the y-pass output
  __shared__ double X[PB_X];
  const PBox B = boxes[blockIdx.x];
  const int f = blockIdx.y;
  const int f0 = B.nf[0], f1 = B.nf[1], f2 = B.nf[2];
  const int c0 = B.nc[0], c1 = B.nc[1], c2 = B.nc[2];
  const double *cf = cb + (int64_t)f * ncb;
  const int32_t *ax = axtab + B.ax;
  for (int q = threadIdx.x; q < c0 * c1 * c2; q += blockDim.x) CY[q] = cf[slots[B.tab + q]];
  __syncthreads();
  for (int q = threadIdx.x; q < f0 * c1 * c2; q += blockDim.x) {  // [z'][y'][i]
    const int i = q % f0, r = q / f0;
    const int32_t e = ax[i];
    const double *w = pw + (e >> 16);
    const double *row = CY + r * c0 + (e & 0xffff);
    double v = 0.0;
#pragma unroll
    for (int a = 0; a < 5; ++a) v = fma(w[a], row[a], v);
    X[q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < f0 * f1 * c2; q += blockDim.x) {  // [z'][j][i]
    const int i = q % f0, j = (q / f0) % f1, z = q / (f0 * f1);
    const int32_t e = ax[f0 + j];
    const double *w = pw + (e >> 16);
    const int s = e & 0xffff;
    double v = 0.0;
#pragma unroll
    for (int b = 0; b < 5; ++b) v = fma(w[b], X[(z * c1 + s + b) * f0 + i], v);
    CY[q] = v;
  }
  __syncthreads();
  const DevBlock &D = blocks[B.dst];
  double *out = reg + D.off + (int64_t)f * D.S;
  const int e0 = D.e[0], e1 = D.e[1];
  for (int q = threadIdx.x; q < f0 * f1 * f2; q += blockDim.x) {
    const int i = q % f0, j = (q / f0) % f1, k = q / (f0 * f1);
    const int32_t e = ax[f0 + f1 + k];
    const double *w = pw + (e >> 16);
    const int s = e & 0xffff;
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 5; ++c) v = fma(w[c], CY[((s + c) * f1 + j) * f0 + i], v);
    out[((B.o[2] + k) * e1 + (B.o[1] + j)) * e0 + (B.o[0] + i)] = v;
  }
}

}  // namespace z4c
