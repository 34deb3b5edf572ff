// Context creation and binding (C ABI, include/z4c.h).  Validates each
// instance's Mesh of MeshBlocks (paper Sec. 3: an oct-tree of equal blocks,
// neighbours at most one refinement level apart), builds the per-block
// descriptors, the interior tile lists of every (order, precision) group, the
// Sommerfeld cell lists and the ghost-fill lists: same-level copies and, at
// refinement boundaries (Sec. 3.1), restrictions, coarse-buffer copies and
// prolongations.  Everything is laid out in the caller's scratch buffer.  No
// CUDA call happens before z4c_bind.
#include <algorithm>
#include <climits>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "z4c_ctx.cuh"

using namespace z4c;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The block's FP32 shadow as a 4-D tensor (x, y, z, field) with boxes of one
// field's PRE_TMA_PX x (PRE_TMA_PY + order) rows of one plane; out-of-range
// box parts read as zero.  False if the encoder is missing or refuses.
bool encode_shadow_map(CUtensorMap *m, const float *base, const DevBlock &D, int order) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dim[4] = {(cuuint64_t)D.e[0], (cuuint64_t)D.e[1], (cuuint64_t)D.e[2], (cuuint64_t)NF};
  const cuuint64_t stride[3] = {(cuuint64_t)D.e[0] * 4, (cuuint64_t)D.e[0] * D.e[1] * 4, (cuuint64_t)D.S * 4};
  const cuuint32_t box[4] = {(cuuint32_t)PRE_TMA_PX, (cuuint32_t)(PRE_TMA_PY + order), 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dim, stride, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
long long iround(double v) { return (long long)std::llround(v); }
long long ifloor(double v) { return (long long)std::floor(v); }

// Lagrange basis polynomial l_i(x) over the points xs[0..np-1] (Sec. 3.1.1)
double lagrange(const double *xs, int np, int i, double x) {
  double w = 1.0;
  for (int q = 0; q < np; ++q)
    if (q != i) w *= (x - xs[q]) / (xs[i] - xs[q]);
  return w;
}
double lagrange5(const double xs[5], int i, double x) { return lagrange(xs, 5, i, x); }

// Points per axis of the transfer stencils: N_g + 1 = 3 with 2 ghosts
// (Sec. 3.1.1, the 3rd-order transfer of 2nd-order differencing), else 5.
// Every table and kernel works on 5-point windows; a 3-point stencil is
// stored as the 5-point window that contains it (kept inside the active
// region or the domain), with zero weights on the two other points.
int transfer_points(int ghosts) { return ghosts == 2 ? 3 : 5; }

// 5 restriction weights: window start key = s5 - 2c (fine cells, relative to
// the coarse cell's first child); np == 3 puts the 3-point weights of the
// cells s5 + off .. s5 + off + 2 at positions off .. off + 2.
void restriction_row(int key, int np, int off, double w[5]) {
  for (int q = 0; q < 5; ++q) w[q] = 0.0;
  double xs[5];
  const int o = np == 5 ? 0 : off;
  for (int q = 0; q < np; ++q) xs[q] = key + o + q - 0.5;  // fine centres, relative to the coarse centre
  for (int q = 0; q < np; ++q) w[o + q] = lagrange(xs, np, q, 0.0);
}

// Restriction stencil along one axis (Sec. 3.1.1, readings R12 and R19):
// coarse cell c of a fine block of n cells; returns the 5-point window start
// s5 and, for np == 3, the offset of the 3-point stencil inside it.
void restriction_start(int c, int n, int np, int &s5, int &off) {
  const int nc = n / 2;
  if (np == 5) {
    s5 = std::min(std::max(c < nc / 2 ? 2 * c - 1 : 2 * c - 2, 0), n - 5);
    off = 0;
    return;
  }
  const int s3 = std::min(std::max(c < nc / 2 ? 2 * c : 2 * c - 1, 0), n - 3);
  s5 = std::min(std::max(s3 - 1, 0), n - 5);
  off = s3 - s5;
}

int check_instance(const z4c_instance &I) {
  const z4c_params &p = I.params;
  if (I.fd_order != 2 && I.fd_order != 4 && I.fd_order != 6) return Z4C_ERR_UNSUPPORTED;
  if (I.ghosts < I.fd_order / 2 + 1 || I.ghosts > 8) return Z4C_ERR_UNSUPPORTED;
  if (p.rhs_precision != 64 && p.rhs_precision != 32) return Z4C_ERR_UNSUPPORTED;
  if (p.lapse < 0 || p.lapse > 1 || p.shift < 0 || p.shift > 1) return Z4C_ERR_BAD_ARG;
  if (!(p.chi_floor > 0.0)) return Z4C_ERR_BAD_ARG;
  if (p.schedule < 0 || p.schedule > 6) return Z4C_ERR_BAD_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(I.mesh.hi[d] > I.mesh.lo[d])) return Z4C_ERR_BAD_MESH;
  return Z4C_OK;
}

// The blocks of one instance: equal n, spacing h0 / 2^level, aligned to their
// level's block lattice, tiling the mesh without overlap.  The owner map
// records the block covering each cell of the finest block lattice.
struct Layout {
  int n[3] = {0, 0, 0};
  double h0 = 0.0;
  int lmax = 0;
  double unit[3] = {0, 0, 0};     // finest block width per axis
  long long M[3] = {0, 0, 0};     // finest lattice cells per axis
  std::vector<int> owner;         // local block index per finest lattice cell
  std::vector<std::array<long long, 3>> go;  // first interior cell, global index at the block's level
};

int make_layout(const z4c_instance &I, const z4c_block *blocks, int count, Layout &Lo) {
  for (int d = 0; d < 3; ++d) Lo.n[d] = blocks[0].n[d];
  Lo.h0 = blocks[0].h * std::ldexp(1.0, blocks[0].level);
  if (!(Lo.h0 > 0.0)) return Z4C_ERR_BAD_MESH;
  for (int b = 0; b < count; ++b) {
    const z4c_block &B = blocks[b];
    if (B.level < 0 || B.level > 20) return Z4C_ERR_BAD_MESH;
    for (int d = 0; d < 3; ++d)
      if (B.n[d] != Lo.n[d]) return Z4C_ERR_BAD_MESH;
    if (std::fabs(B.h * std::ldexp(1.0, B.level) - Lo.h0) > 1e-12 * Lo.h0) return Z4C_ERR_BAD_MESH;
    Lo.lmax = std::max(Lo.lmax, B.level);
  }
  for (int d = 0; d < 3; ++d)
    if (Lo.n[d] < I.ghosts) return Z4C_ERR_UNSUPPORTED;  // a ghost region must come from one neighbour
  if (Lo.lmax > 0)  // restriction stencils: 5 fine cells inside an even block
    for (int d = 0; d < 3; ++d)
      if (Lo.n[d] < 8 || Lo.n[d] % 2) return Z4C_ERR_UNSUPPORTED;
  long long total = 1;
  for (int d = 0; d < 3; ++d) {
    Lo.unit[d] = Lo.n[d] * Lo.h0 / std::ldexp(1.0, Lo.lmax);
    const double v = (I.mesh.hi[d] - I.mesh.lo[d]) / Lo.unit[d];
    Lo.M[d] = iround(v);
    if (Lo.M[d] < 1 || std::fabs(v - Lo.M[d]) > 1e-8 * std::max(1.0, v)) return Z4C_ERR_BAD_MESH;
    total *= Lo.M[d];
  }
  if (total > (1LL << 28)) return Z4C_ERR_UNSUPPORTED;
  Lo.owner.assign((size_t)total, -1);
  Lo.go.resize(count);
  for (int b = 0; b < count; ++b) {
    const z4c_block &B = blocks[b];
    const long long span = 1LL << (Lo.lmax - B.level);  // finest cells per block
    long long o[3];
    for (int d = 0; d < 3; ++d) {
      const double v = (B.lo[d] - I.mesh.lo[d]) / Lo.unit[d];
      o[d] = iround(v);
      if (std::fabs(v - o[d]) > 1e-8 * std::max(1.0, std::fabs(v))) return Z4C_ERR_BAD_MESH;
      if (o[d] < 0 || o[d] % span != 0 || o[d] + span > Lo.M[d]) return Z4C_ERR_BAD_MESH;
      Lo.go[b][d] = o[d] / span * Lo.n[d];
    }
    for (long long k = o[2]; k < o[2] + span; ++k)
      for (long long j = o[1]; j < o[1] + span; ++j)
        for (long long i = o[0]; i < o[0] + span; ++i) {
          int &c = Lo.owner[(size_t)((k * Lo.M[1] + j) * Lo.M[0] + i)];
          if (c != -1) return Z4C_ERR_BAD_MESH;  // overlap
          c = b;
        }
  }
  for (int c : Lo.owner)
    if (c == -1) return Z4C_ERR_BAD_MESH;  // gap
  return Z4C_OK;
}

// Builder of one instance's ghost-fill lists.
struct GhostBuilder {
  z4c_ctx *ctx;
  const Instance &I;
  const Layout &Lo;
  int p;  // precision slot
  std::map<int, int> wpat;  // restriction pattern key -> row of ctx->wtab
  std::map<std::array<long long, 4>, int> slot;  // (level, wrapped coarse cell) -> coarse-buffer slot

  const z4c_block &blk(int lb) const { return ctx->blocks[I.first + lb]; }
  double hb(int lb) const { return blk(lb).h; }

  // wrap into a periodic domain; false if outside a non-periodic one
  bool inside(double x[3]) const {
    for (int d = 0; d < 3; ++d) {
      if (I.mesh.periodic) {
        const double L = I.mesh.hi[d] - I.mesh.lo[d];
        while (x[d] < I.mesh.lo[d]) x[d] += L;
        while (x[d] >= I.mesh.hi[d]) x[d] -= L;
      } else if (x[d] < I.mesh.lo[d] || x[d] > I.mesh.hi[d]) {
        return false;
      }
    }
    return true;
  }

  int owner_of(const double x[3]) const {
    long long u[3];
    for (int d = 0; d < 3; ++d) {
      u[d] = ifloor((x[d] - I.mesh.lo[d]) / Lo.unit[d]);
      u[d] = std::min(std::max(u[d], 0LL), Lo.M[d] - 1);
    }
    return Lo.owner[(size_t)((u[2] * Lo.M[1] + u[1]) * Lo.M[0] + u[0])];
  }

  int storage_index(int lb, const long long q[3]) const {
    const int g = I.ghosts;
    const long long e0 = Lo.n[0] + 2 * g, e1 = Lo.n[1] + 2 * g;
    return (int)((q[2] * e1 + q[1]) * e0 + q[0]);
  }

  // storage index in block lb of the cell whose centre is x
  int cell_in(int lb, const double x[3]) const {
    long long q[3];
    for (int d = 0; d < 3; ++d) q[d] = ifloor((x[d] - blk(lb).lo[d]) / hb(lb)) + I.ghosts;
    return storage_index(lb, q);
  }

  int pattern(int key, int np, int off) {
    const int k = 16 * key + 4 * (np == 3) + off;
    auto it = wpat.find(k);
    if (it != wpat.end()) return it->second;
    double w[5];
    restriction_row(key, np, off, w);
    const int row = (int)(ctx->wtab.size() / 5);
    for (int q = 0; q < 5; ++q) ctx->wtab.push_back(w[q]);
    wpat[k] = row;
    return row;
  }

  // restriction of fine block nb at the coarse cell centred at x (Sec. 3.1.1):
  // 5 fine cells per axis, start 2c-1 (lower half of the block) or 2c-2
  // (upper half); with 2 ghosts 3 cells from 2c or 2c-1; clamped into the
  // active region
  RestrictRef restriction(int nb, const double x[3]) {
    RestrictRef r{};
    long long st[3];
    const int np = transfer_points(I.ghosts);
    for (int d = 0; d < 3; ++d) {
      const long long c = ifloor((x[d] - blk(nb).lo[d]) / (2.0 * hb(nb)));
      int s, off;
      restriction_start((int)c, Lo.n[d], np, s, off);
      r.wp[d] = pattern((int)(s - 2 * c), np, off);
      st[d] = s + I.ghosts;
      r.cc |= (int32_t)(c << (8 * d));
    }
    r.src = I.first + nb;
    r.s = storage_index(nb, st);
    return r;
  }

  // coarse-buffer slot of the level-lc cell with global index q (unwrapped)
  int coarse_slot(int lc, const long long q[3], int &err) {
    double x[3];
    const double hc = Lo.h0 / std::ldexp(1.0, lc);
    for (int d = 0; d < 3; ++d) x[d] = I.mesh.lo[d] + (q[d] + 0.5) * hc;
    if (!inside(x)) {
      err = 1;
      return 0;
    }
    long long w[3];
    for (int d = 0; d < 3; ++d) w[d] = ifloor((x[d] - I.mesh.lo[d]) / hc);
    const std::array<long long, 4> key = {lc, w[0], w[1], w[2]};
    auto it = slot.find(key);
    if (it != slot.end()) return it->second;
    const int nb = owner_of(x);
    const int s = ctx->ncb++;
    if (blk(nb).level == lc) {
      ctx->cbcopy.push_back(CbCopy{s, I.first + nb, cell_in(nb, x), 0});
    } else if (blk(nb).level == lc + 1) {
      RestrictRef r = restriction(nb, x);
      r.dst = -1;
      r.didx = s;
      ctx->rbuf.push_back(r);
    } else {
      err = 1;  // two levels apart
    }
    slot[key] = s;
    return s;
  }

  // Stencil start (global level-(L-1) index, shifted into a non-periodic
  // domain) and pw row of the fine cell with global level-L index gi.
  void stencil_of(long long gi, double hc, int d, long long &start, int &row) const {
    const long long P = gi >= 0 ? gi / 2 : -((-gi + 1) / 2);  // floor(gi / 2)
    long long sh = 0;
    if (!I.mesh.periodic) {
      const long long nd = iround((I.mesh.hi[d] - I.mesh.lo[d]) / hc);
      sh = std::max<long long>(std::min<long long>(P - 2, nd - 5), 0) - (P - 2);
    }
    start = P - 2 + sh;
    row = (int)(10 * (sh + 2) + 5 * (gi - 2 * P)) + (transfer_points(I.ghosts) == 3 ? 50 : 0);
  }

  // Ghost regions of block lb (index r0 + 3 r1 + 9 r2 with r_d = 0 below,
  // 1 beside, 2 above the interior along d) that lie inside the domain and
  // wholly in coarser blocks become PBox entries, when the ghost width is
  // even (no parent straddles two regions), at most 4, and the block has at
  // most 16 cells per axis.
  void boxes(int lb, bool boxed[27], int &err) {
    const int g = I.ghosts, L = blk(lb).level;
    if (g % 2 != 0 || g > 4 || L == 0) return;
    for (int d = 0; d < 3; ++d)
      if (Lo.n[d] > 16) return;
    const double h = hb(lb), hc = 2.0 * h;
    const int e[3] = {Lo.n[0] + 2 * g, Lo.n[1] + 2 * g, Lo.n[2] + 2 * g};
    for (int r = 0; r < 27; ++r) {
      if (r == 13) continue;  // the interior
      int lo[3], hi[3];
      for (int d = 0, q = r; d < 3; ++d, q /= 3) {
        const int rd = q % 3;
        lo[d] = rd == 0 ? 0 : rd == 1 ? g : g + Lo.n[d];
        hi[d] = rd == 0 ? g : rd == 1 ? g + Lo.n[d] : e[d];
      }
      bool all = true;
      for (int k = lo[2]; k < hi[2] && all; ++k)
        for (int j = lo[1]; j < hi[1] && all; ++j)
          for (int i = lo[0]; i < hi[0] && all; ++i) {
            const int idx[3] = {i, j, k};
            double x[3];
            for (int d = 0; d < 3; ++d) x[d] = blk(lb).lo[d] + (idx[d] - g + 0.5) * h;
            all = inside(x) && blk(owner_of(x)).level == L - 1;
          }
      if (!all) continue;
      PBox B{};
      B.dst = I.first + lb;
      B.ax = (int)ctx->paxtab.size();
      long long cmin[3], cmax[3];
      for (int d = 0; d < 3; ++d) {
        B.o[d] = (int16_t)lo[d];
        B.nf[d] = (uint8_t)(hi[d] - lo[d]);
        cmin[d] = LLONG_MAX;
        cmax[d] = LLONG_MIN;
        for (int s = lo[d]; s < hi[d]; ++s) {
          long long st;
          int row;
          stencil_of(Lo.go[lb][d] + s - g, hc, d, st, row);
          cmin[d] = std::min(cmin[d], st);
          cmax[d] = std::max(cmax[d], st + 4);
        }
        B.nc[d] = (uint8_t)(cmax[d] - cmin[d] + 1);
      }
      const int ncb = B.nc[0] * B.nc[1] * B.nc[2];
      if (ncb > PB_C || B.nf[0] * B.nc[1] * B.nc[2] > PB_X || B.nf[0] * B.nf[1] * B.nc[2] > PB_Y) continue;
      for (int d = 0; d < 3; ++d)
        for (int s = lo[d]; s < hi[d]; ++s) {
          long long st;
          int row;
          stencil_of(Lo.go[lb][d] + s - g, hc, d, st, row);
          ctx->paxtab.push_back((int32_t)((row << 16) | (int)(st - cmin[d])));
        }
      B.tab = (int)ctx->pslots.size();
      for (long long z = cmin[2]; z <= cmax[2]; ++z)
        for (long long y = cmin[1]; y <= cmax[1]; ++y)
          for (long long x = cmin[0]; x <= cmax[0]; ++x) {
            const long long q[3] = {x, y, z};
            ctx->pslots.push_back(coarse_slot(L - 1, q, err));
          }
      ctx->pbox.push_back(B);
      boxed[r] = true;
    }
  }

  int build() {
    const int g = I.ghosts;
    const int e[3] = {Lo.n[0] + 2 * g, Lo.n[1] + 2 * g, Lo.n[2] + 2 * g};
    int err = 0;
    for (int lb = 0; lb < I.count; ++lb) {
      const int b = I.first + lb, L = blk(lb).level;
      const double h = hb(lb);
      std::map<std::array<long long, 3>, int> parents;  // prolongation parents already listed
      bool boxed[27] = {false};
      boxes(lb, boxed, err);
      auto region_of = [&](const int idx[3]) {
        int r = 0;
        for (int d = 2; d >= 0; --d) r = 3 * r + (idx[d] < g ? 0 : idx[d] < Lo.n[d] + g ? 1 : 2);
        return r;
      };
      for (int k = 0; k < e[2]; ++k)
        for (int j = 0; j < e[1]; ++j)
          for (int i = 0; i < e[0]; ++i) {
            const int idx[3] = {i, j, k};
            bool interior = true;
            for (int d = 0; d < 3; ++d) interior &= idx[d] >= g && idx[d] < Lo.n[d] + g;
            if (interior) continue;
            double x[3], xw[3];
            for (int d = 0; d < 3; ++d) xw[d] = x[d] = blk(lb).lo[d] + (idx[d] - g + 0.5) * h;
            const int cidx = (k * e[1] + j) * e[0] + i;
            if (!inside(xw)) {
              CellRef c{b, cidx, (int16_t)i, (int16_t)j, (int16_t)k, 0};
              for (int d = 0; d < 3; ++d) {
                const int kind = idx[d] < g ? SOMM_FORWARD : idx[d] >= Lo.n[d] + g ? SOMM_BACKWARD : SOMM_CENTRED;
                c.code |= (uint16_t)(kind << (2 * d));
              }
              ctx->somm[p].push_back(c);
              continue;
            }
            const int nb = owner_of(xw);
            const int ln = blk(nb).level;
            if (ln == L) {
              ctx->gcopy[p].push_back(GhostCopy{b, cidx, I.first + nb, cell_in(nb, xw)});
            } else if (ln == L + 1) {
              RestrictRef r = restriction(nb, xw);
              r.dst = b;
              r.didx = cidx;
              ctx->rghost.push_back(r);
            } else if (ln == L - 1) {
              if (boxed[region_of(idx)]) continue;  // filled by prolong_box_kernel
              // parent coarse cell (global index at level L-1, unwrapped)
              std::array<long long, 3> pc;
              const double hc = 2.0 * h;
              for (int d = 0; d < 3; ++d) pc[d] = ifloor((x[d] - I.mesh.lo[d]) / hc);
              if (parents.count(pc)) continue;
              parents[pc] = 1;
              long long child[3];
              int ok[3][2];
              for (int d = 0; d < 3; ++d) {
                child[d] = 2 * pc[d] - Lo.go[lb][d] + g;  // storage index of the lower child
                ok[d][0] = child[d] >= 0 && child[d] < e[d];
                ok[d][1] = child[d] + 1 >= 0 && child[d] + 1 < e[d];
              }
              int mask = 0;
              for (int q = 0; q < 8; ++q)
                if (ok[0][q & 1] && ok[1][(q >> 1) & 1] && ok[2][(q >> 2) & 1]) mask |= 1 << q;
              // stencil shift into a non-periodic domain: cells pc-2+sh .. pc+2+sh
              // must lie in [0, nd) with nd the level-(L-1) cells across the domain
              long long sh[3] = {0, 0, 0};
              if (!I.mesh.periodic)
                for (int d = 0; d < 3; ++d) {
                  const long long nd = iround((I.mesh.hi[d] - I.mesh.lo[d]) / hc);
                  const long long s0 = std::max<long long>(std::min<long long>(pc[d] - 2, nd - 5), 0);
                  sh[d] = s0 - (pc[d] - 2);
                }
              for (int d = 0; d < 3; ++d) {
                if (sh[d] < -2 || sh[d] > 2) err = 1;  // domain narrower than 5 coarse cells
                else mask |= (int)(sh[d] + 2) << (PROLONG_SHIFT_BIT + 3 * d);
              }
              if (transfer_points(g) == 3) mask |= 1 << PROLONG_NP3_BIT;
              // the lower child may lie before the storage (odd ghost width): address
              // children relative to an index that can be negative; the kernel only
              // touches the masked ones
              ProlongRef pr{b, (int)((child[2] * e[1] + child[1]) * e[0] + child[0]), (int)ctx->pidx.size(), mask};
              for (int c = 0; c < 5; ++c)
                for (int bb = 0; bb < 5; ++bb)
                  for (int a = 0; a < 5; ++a) {
                    const long long q[3] = {pc[0] + sh[0] + a - 2, pc[1] + sh[1] + bb - 2, pc[2] + sh[2] + c - 2};
                    ctx->pidx.push_back(coarse_slot(L - 1, q, err));
                  }
              ctx->prol.push_back(pr);
            } else {
              err = 1;  // neighbours more than one level apart
            }
          }
    }
    return err ? Z4C_ERR_BAD_MESH : Z4C_OK;
  }
};

}  // namespace

extern "C" {

int z4c_create_batch(const z4c_instance *instances, int ninstances, const z4c_block *blocks, int nblocks,
                     z4c_ctx **out) {
  if (!out) return Z4C_ERR_BAD_ARG;
  *out = nullptr;
  if (!instances || !blocks || ninstances <= 0 || nblocks <= 0) return Z4C_ERR_BAD_ARG;
  // blocks grouped by instance, in instance order
  std::vector<int> first(ninstances, -1), count(ninstances, 0);
  for (int b = 0; b < nblocks; ++b) {
    const int i = blocks[b].instance;
    if (i < 0 || i >= ninstances) return Z4C_ERR_BAD_ARG;
    if (b > 0 && i < blocks[b - 1].instance) return Z4C_ERR_BAD_ARG;
    if (first[i] < 0) first[i] = b;
    ++count[i];
  }
  for (int i = 0; i < ninstances; ++i) {
    if (count[i] == 0) return Z4C_ERR_BAD_ARG;
    const int r = check_instance(instances[i]);
    if (r) return r;
  }

  z4c_ctx *ctx = new z4c_ctx();
  auto bail = [&](int code) {
    delete ctx;
    return code;
  };
  ctx->blocks.assign(blocks, blocks + nblocks);
  int64_t off = 0;
  bool sched_set[2] = {false, false};
  // prolongation weights: coarse points at shift-2..shift+2 (coarse
  // spacing) from the parent centre, evaluated at the children's offsets
  // -1/4 and +1/4, for shift = -2..2.  pw[50..99]: the 3-point stencils of
  // 2 ghosts in the same 5-point windows.  The window shift fixes where the
  // parent lies in it (2 - shift) and so the 3-point start inside it,
  // clamp(parent - 1, 0, 2): parent-1..parent+1, moved by at most one cell
  // into the domain like the window (readings R13, R19).
  for (int sh = -2; sh <= 2; ++sh) {
    double xs[5];
    for (int q = 0; q < 5; ++q) xs[q] = sh + q - 2;
    for (int q = 0; q < 5; ++q) {
      ctx->pw[10 * (sh + 2) + q] = lagrange5(xs, q, -0.25);
      ctx->pw[10 * (sh + 2) + 5 + q] = lagrange5(xs, q, 0.25);
    }
    const int s3 = std::min(std::max(2 - sh - 1, 0), 2);
    double x3[3];
    for (int a = 0; a < 3; ++a) x3[a] = sh - 2 + s3 + a;
    for (int a = 0; a < 3; ++a) {
      ctx->pw[50 + 10 * (sh + 2) + s3 + a] = lagrange(x3, 3, a, -0.25);
      ctx->pw[50 + 10 * (sh + 2) + 5 + s3 + a] = lagrange(x3, 3, a, 0.25);
    }
  }
  for (int i = 0; i < ninstances; ++i) {
    const z4c_instance &I = instances[i];
    Layout Lo;
    int r = make_layout(I, blocks + first[i], count[i], Lo);
    if (r) return bail(r);
    const bool f32 = I.params.rhs_precision == 32;
    if (f32 && Lo.lmax > 0) return bail(Z4C_ERR_UNSUPPORTED);  // refinement transfer is FP64 only
    Instance in;
    in.mesh = I.mesh;
    in.params = I.params;
    in.ghosts = I.ghosts;
    in.order = I.fd_order;
    in.first = first[i];
    in.count = count[i];
    ctx->inst.push_back(in);
    const int p = f32 ? 1 : 0;
    ctx->has[p] = true;
    if (!sched_set[p]) {
      // default (0): FP64 pre-pass + fused kernel; FP32-RHS split schedule 4
      const int sc = I.params.schedule;
      ctx->sched[p] = sc == 1 ? 1 : sc == 2 ? 2 : !f32 ? 2 : sc == 0 ? 4 : sc;
      sched_set[p] = true;
    }
    const int g = I.ghosts, ord = I.fd_order;
    const int *n = Lo.n;
    const int e[3] = {n[0] + 2 * g, n[1] + 2 * g, n[2] + 2 * g};
    const long long S = (long long)e[0] * e[1] * e[2];
    if (S * NF >= (1LL << 31)) return bail(Z4C_ERR_UNSUPPORTED);
    ctx->max_S = std::max(ctx->max_S, (int)S);
    // stencil denominators: 2h, h^2 (2nd order); 12h, 12h^2 (4th); 60h, 180h^2 (6th)
    const double den1 = ord == 2 ? 2.0 : ord == 4 ? 12.0 : 60.0, den2 = ord == 2 ? 1.0 : ord == 4 ? 12.0 : 180.0;
    // KO: (-1)^(N+1) / 2^(2N), N = order/2 + 1
    const double kosg = ord == 2 ? -1.0 / 16.0 : ord == 4 ? 1.0 / 64.0 : -1.0 / 256.0;
    Group &G = ctx->grp[group_of(ord, f32)];
    G.order = ord;
    G.f32 = f32;
    const int W = ord / 2;
    for (int lb = 0; lb < count[i]; ++lb) {
      const int b = first[i] + lb;
      const double h = blocks[b].h;
      DevBlock D{};
      for (int d = 0; d < 3; ++d) {
        D.n[d] = n[d];
        D.e[d] = e[d];
        D.lo[d] = blocks[b].lo[d];
      }
      D.g = g;
      D.order = ord;
      D.S = (int32_t)S;
      D.off = off;
      off += NF * S;
      D.h = h;
      D.s1 = 1.0 / (den1 * h);
      D.s2 = 1.0 / (den2 * h * h);
      D.smix = 1.0 / (den1 * den1 * h * h);
      D.slop = 1.0 / (den1 * h);
      D.sko = kosg * I.params.ko_sigma / h;
      D.s1f = (float)D.s1;
      D.s2f = (float)D.s2;
      D.smixf = (float)D.smix;
      D.slopf = (float)D.slop;
      D.skof = (float)D.sko;
      D.hf = (float)h;
      D.kappa1 = I.params.kappa1;
      D.kappa2 = I.params.kappa2;
      D.eta = I.params.eta;
      D.chi_floor = I.params.chi_floor;
      D.lapse = I.params.lapse;
      D.shift = I.params.shift;
      D.instance = i;
      D.f32 = f32 ? 1 : 0;
      ctx->dblocks.push_back(D);
      ctx->dt_host.push_back(0.0);
      // the staged FP32 kernel copies 24-float rows from x = i0 with 16-byte
      // aligned bulk copies and assumes full tiles
      const bool staged = f32 && ord == 6 && g == 4 && n[0] % TX == 0 && n[1] % TY == 0 && e[0] % 4 == 0 &&
                          D.off % 4 == 0;
      for (int k = 0; k < n[2]; ++k) {
        for (int j0 = 0; j0 < n[1]; j0 += TY)
          for (int i0 = 0; i0 < n[0]; i0 += TX) {
            G.tiles.push_back(Tile{b, i0, j0, k});
            ctx->ctiles.push_back(Tile{b, i0, j0, k});
            if (f32 && ord == 6) (staged ? G.stiles : G.rtiles).push_back(Tile{b, i0, j0, k});
          }
        for (int j0 = -W; j0 < n[1] + W; j0 += TY)
          for (int i0 = -W; i0 < n[0] + W; i0 += TX) G.wtiles.push_back(Tile{b, i0, j0, k});
      }
    }
    GhostBuilder gb{ctx, ctx->inst.back(), Lo, p, {}, {}};
    r = gb.build();
    if (r) return bail(r);
  }
  ctx->reg_elems = (size_t)off;
  // block-structured restriction when every fine block that is restricted
  // has at most RB_NMAX cells per axis
  {
    bool ok = !(ctx->rghost.empty() && ctx->rbuf.empty());
    for (const auto *lst : {&ctx->rghost, &ctx->rbuf})
      for (const RestrictRef &r : *lst)
        for (int d = 0; d < 3; ++d) ok &= ctx->blocks[r.src].n[d] <= RB_NMAX;
    if (ok) {
      ctx->rb_mode = true;
      // the same weights as GhostBuilder::pattern: krow[key + 4] for 5
      // points, krow[8 + 3 (key + 4) + off] for 3 points at offset off
      for (int key = -4; key < 4; ++key)
        for (int v = 0; v < 4; ++v) {
          double w[5];
          restriction_row(key, v == 0 ? 5 : 3, v == 0 ? 0 : v - 1, w);
          ctx->krow[v == 0 ? key + 4 : 8 + 3 * (key + 4) + v - 1] = (int32_t)(ctx->wtab.size() / 5);
          for (int q = 0; q < 5; ++q) ctx->wtab.push_back(w[q]);
        }
      std::map<int, int> rbi;
      auto add = [&](const RestrictRef &r, int32_t dst, int32_t didx) {
        auto it = rbi.find(r.src);
        if (it == rbi.end()) {
          it = rbi.emplace(r.src, (int)ctx->rblocks.size()).first;
          ctx->rblocks.push_back(r.src);
        }
        const z4c_block &B = ctx->blocks[r.src];
        const int c0 = r.cc & 255, c1 = (r.cc >> 8) & 255, c2 = (r.cc >> 16) & 255;
        ctx->rbcopy.push_back(RbCopy{dst, didx, it->second, (c2 * (B.n[1] / 2) + c1) * (B.n[0] / 2) + c0});
      };
      for (const RestrictRef &r : ctx->rghost) add(r, r.dst, r.didx);
      for (const RestrictRef &r : ctx->rbuf) add(r, -1, r.didx);
    }
  }
  // tiles sorted by the cubic storage extent of their block (stable, so the
  // order within a block is kept), one range per extent
  for (Group &G : ctx->grp) {
    if (G.tiles.empty()) continue;
    auto ext_of = [&](const Tile &t) {
      const DevBlock &D = ctx->dblocks[t.block];
      return (D.e[0] == D.e[1] && D.e[1] == D.e[2]) ? D.e[0] : 0;
    };
    std::stable_sort(G.tiles.begin(), G.tiles.end(),
                     [&](const Tile &x, const Tile &y) { return ext_of(x) < ext_of(y); });
    for (int q = 0; q < (int)G.tiles.size(); ++q) {
      const int e = ext_of(G.tiles[q]);
      if (G.eranges.empty() || G.eranges.back().ext != e) G.eranges.push_back({e, q, 0, true});
      ++G.eranges.back().count;
      // two cells per thread: even ghost width and interior width, even
      // block offset (8-byte aligned cell pairs in every array)
      const DevBlock &D = ctx->dblocks[G.tiles[q].block];
      G.eranges.back().pair = G.eranges.back().pair && G.f32 && D.g % 2 == 0 && D.n[0] % 2 == 0 &&
                              D.off % 2 == 0 && D.S % 2 == 0;
    }
    if (!G.f32) continue;
    ctx->wide_shape.resize(ctx->dblocks.size(), 0);
    ctx->wide_pair.resize(ctx->dblocks.size(), 0);
    // schedule-5/6 list: wide tiles (a warp along one row) where n_x is a
    // multiple of 64 (shape 2) or 32 (shape 1) and a kernel is built
    for (const Group::ExtRange &r : G.eranges) {
      const int n0 = ctx->dblocks[G.tiles[r.first].block].n[0];
      const int shape = !wide_ext_built(G.order, r.ext) ? 0 : n0 % 64 == 0 ? 2 : n0 % 32 == 0 ? 1 : 0;
      Group::ExtRange pr{r.ext, (int)G.ptiles.size(), 0, r.pair && shape > 0, shape};
      if (shape == 0) {
        G.ptiles.insert(G.ptiles.end(), G.tiles.begin() + r.first, G.tiles.begin() + r.first + r.count);
      } else {
        const int txs = TX << shape, tys = TY >> shape;
        int last = -1;
        for (int q = r.first; q < r.first + r.count; ++q) {
          const int b = G.tiles[q].block;
          if (b == last) continue;  // a block's tiles are contiguous in the sorted list
          last = b;
          ctx->wide_shape[b] = (int8_t)shape;
          ctx->wide_pair[b] = (int8_t)(r.pair ? 1 : 0);
          const DevBlock &D = ctx->dblocks[b];
          for (int k = 0; k < D.n[2]; ++k)
            for (int j0 = 0; j0 < D.n[1]; j0 += tys)
              for (int i0 = 0; i0 < D.n[0]; i0 += txs)
                G.ptiles.push_back(Tile{b | (shape << TILE_SHAPE_SHIFT), i0, j0, k});
        }
      }
      pr.count = (int)G.ptiles.size() - pr.first;
      G.peranges.push_back(pr);
    }
    // full, 16-byte aligned tiles for the bulk-copy stage update
    auto full_of = [&](const std::vector<Tile> &tl, Group::ExtRange &r) {
      r.full = true;
      for (int q = r.first; q < r.first + r.count; ++q) {
        const int sh = tl[q].block >> TILE_SHAPE_SHIFT;
        const DevBlock &D = ctx->dblocks[tl[q].block & TILE_BLOCK_MASK];
        r.full = r.full && D.n[0] % (TX << sh) == 0 && D.n[1] % (TY >> sh) == 0 && D.g % 2 == 0 &&
                 D.e[0] % 2 == 0 && D.e[1] % 2 == 0 && D.off % 2 == 0 && D.S % 2 == 0;
      }
    };
    for (Group::ExtRange &r : G.eranges) full_of(G.tiles, r);
    for (Group::ExtRange &r : G.peranges) full_of(G.ptiles, r);
    // the z-walking pre-pass fed by TMA: 16-byte aligned rows and fields in
    // every block of the group; tiles whose storage x is a multiple of
    // PRE_TMA_PX, covering the interior widened by W in x and y, each
    // walking PRE_TMA_NZ planes (z chunks outermost)
    if (prepass_tma_built(G.order)) {
      const int W = G.order / 2;
      std::vector<int> gb;
      for (const Tile &t : G.tiles)
        if (gb.empty() || gb.back() != t.block) gb.push_back(t.block);
      std::sort(gb.begin(), gb.end());
      gb.erase(std::unique(gb.begin(), gb.end()), gb.end());
      bool ok = !gb.empty();
      for (int b : gb) {
        const DevBlock &D = ctx->dblocks[b];
        ok = ok && D.e[0] % 4 == 0 && D.S % 4 == 0 && D.off % 4 == 0 && D.g >= W;
      }
      if (ok) {
        G.tma_pre = true;
        for (int b : gb) {
          const DevBlock &D = ctx->dblocks[b];
          for (int k0 = 0; k0 < D.n[2]; k0 += PRE_TMA_NZ)
            for (int j0 = -W; j0 < D.n[1] + W; j0 += PRE_TMA_PY)
              for (int xs = 0; xs < D.g + D.n[0] + W; xs += PRE_TMA_PX)
                if (xs + PRE_TMA_PX > D.g - W)
                  for (int fg = 0; fg * PRE_TMA_NQ < NDS; ++fg)
                    G.ztiles.push_back(Tile{b | (fg << TILE_SHAPE_SHIFT), xs - D.g, j0, k0});
        }
      }
    }
  }
  // prolongation slots transposed to [125][entries] so that the threads of a
  // warp (neighbouring entries) read consecutive words
  {
    const size_t ne = ctx->prol.size();
    std::vector<int32_t> tr(ctx->pidx.size());
    for (size_t e = 0; e < ne; ++e)
      for (size_t q = 0; q < 125; ++q) tr[q * ne + e] = ctx->pidx[e * 125 + q];
    ctx->pidx.swap(tr);
  }

  // scratch layout
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + std::max<size_t>(bytes, 1));
    return at;
  };
  ctx->o_blocks = take(sizeof(DevBlock) * ctx->dblocks.size());
  for (Group &G : ctx->grp) {
    G.o_tiles = take(sizeof(Tile) * G.tiles.size());
    G.o_wtiles = take(sizeof(Tile) * G.wtiles.size());
    G.o_stiles = take(sizeof(Tile) * G.stiles.size());
    G.o_rtiles = take(sizeof(Tile) * G.rtiles.size());
    G.o_ptiles = take(sizeof(Tile) * G.ptiles.size());
    G.o_ztiles = take(sizeof(Tile) * G.ztiles.size());
  }
  for (int p = 0; p < 2; ++p) {
    ctx->o_somm[p] = take(sizeof(CellRef) * ctx->somm[p].size());
    ctx->o_gcopy[p] = take(sizeof(GhostCopy) * ctx->gcopy[p].size());
  }
  ctx->o_rghost = take(sizeof(RestrictRef) * ctx->rghost.size());
  ctx->o_rbuf = take(sizeof(RestrictRef) * ctx->rbuf.size());
  ctx->o_rblocks = take(sizeof(int32_t) * ctx->rblocks.size());
  ctx->o_rbcopy = take(sizeof(RbCopy) * ctx->rbcopy.size());
  ctx->o_krow = take(sizeof ctx->krow);
  ctx->o_rb = take(sizeof(double) * NF * RB_NC3 * ctx->rblocks.size());
  ctx->o_cbcopy = take(sizeof(CbCopy) * ctx->cbcopy.size());
  ctx->o_prol = take(sizeof(ProlongRef) * ctx->prol.size());
  ctx->o_pbox = take(sizeof(PBox) * ctx->pbox.size());
  ctx->o_pslots = take(sizeof(int32_t) * ctx->pslots.size());
  ctx->o_paxtab = take(sizeof(int32_t) * ctx->paxtab.size());
  ctx->o_pidx = take(sizeof(int32_t) * ctx->pidx.size());
  ctx->o_wtab = take(sizeof(double) * ctx->wtab.size());
  ctx->o_pw = take(sizeof ctx->pw);
  ctx->o_cb = take(sizeof(double) * NF * (size_t)ctx->ncb);
  ctx->o_ctiles = take(sizeof(Tile) * ctx->ctiles.size());
  ctx->cfirst.assign(ctx->blocks.size() + 1, 0);
  for (const Tile &t : ctx->ctiles) ++ctx->cfirst[t.block + 1];
  for (size_t b = 0; b < ctx->blocks.size(); ++b) ctx->cfirst[b + 1] += ctx->cfirst[b];
  ctx->o_cfirst = take(sizeof(int32_t) * ctx->cfirst.size());
  // diagnostics: per-block indicator outputs, tracker inputs and outputs
  ctx->o_diag = take(std::max(sizeof(double) * 2 * ctx->blocks.size(),
                              (sizeof(TrackIn) + sizeof(double) * 6) * Z4C_MAX_PUNCTURES));
  ctx->o_part = take(sizeof(double) * 8 * 3 * ctx->ctiles.size());  // order-4, -6 and -2 records
  ctx->o_res = take(sizeof(double) * 8);
  ctx->o_dt = take(sizeof(double) * ctx->dblocks.size());
  if (ctx->has[1]) {
    ctx->o_sh0 = take(sizeof(float) * ctx->reg_elems + z4c_ctx::F32_SHIFT);
    ctx->o_sh1 = take(sizeof(float) * ctx->reg_elems + z4c_ctx::F32_SHIFT);
    ctx->o_ds32 = take(sizeof(float) * ctx->reg_elems + z4c_ctx::F32_SHIFT);
  }
  if (ctx->has[0]) ctx->o_ds64 = take(sizeof(double) * ctx->reg_elems);
  ctx->o_status = take(sizeof(int32_t));
  {  // schedule 4: the FP32 RHS of the largest FP32 group's tiles
    size_t nt = 0;
    for (const Group &G : ctx->grp)
      if (G.f32) nt = std::max(nt, std::max(G.tiles.size(), G.ptiles.size()));
    ctx->o_kbuf = take(sizeof(float) * NF * TX * TY * nt);
  }
  // the FP32-RHS Sommerfeld cells' k records (their own: the Sommerfeld
  // kernels may run beside the interior ones)
  ctx->o_kbuf_somm = take(sizeof(float) * somm_kbuf_floats((int)ctx->somm[1].size()));
  // tensor maps of the two FP32 shadows, per block (written at bind)
  if (ctx->has[1]) ctx->o_tmap = take(2 * 128 * ctx->dblocks.size());
  ctx->scratch_total = o;
  *out = ctx;
  return Z4C_OK;
}

int z4c_create(const z4c_mesh *mesh, const z4c_block *blocks, int nblocks, int ghosts, int fd_order,
               const z4c_params *params, z4c_ctx **out) {
  if (!out) return Z4C_ERR_BAD_ARG;
  *out = nullptr;
  if (!mesh || !blocks || !params || nblocks <= 0) return Z4C_ERR_BAD_ARG;
  for (int b = 0; b < nblocks; ++b)
    if (blocks[b].instance != 0) return Z4C_ERR_UNSUPPORTED;
  z4c_instance I;
  I.mesh = *mesh;
  I.params = *params;
  I.ghosts = ghosts;
  I.fd_order = fd_order;
  return z4c_create_batch(&I, 1, blocks, nblocks, out);
}

int z4c_state_bytes(const z4c_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return Z4C_ERR_BAD_ARG;
  *bytes = ctx->reg_elems * sizeof(double);
  return Z4C_OK;
}

int z4c_scratch_bytes(const z4c_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return Z4C_ERR_BAD_ARG;
  *bytes = ctx->scratch_total;
  return Z4C_OK;
}

int z4c_bind(z4c_ctx *ctx, void *u0, void *stage_a, void *stage_b, void *acc, void *scratch,
             void *cuda_stream) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  void *ptrs[5] = {u0, stage_a, stage_b, acc, scratch};
  for (void *p : ptrs)
    if (!p || ((uintptr_t)p & 255)) return fail(ctx, Z4C_ERR_BAD_ARG, "null or unaligned buffer");
  ctx->reg[0] = (double *)u0;
  ctx->reg[1] = (double *)stage_a;
  ctx->reg[2] = (double *)stage_b;
  ctx->reg[3] = (double *)acc;
  ctx->scratch = (char *)scratch;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->drop_graph();
  cudaStream_t st = ctx->stream;
  auto up = [&](size_t at, const void *src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(ctx->scratch + at, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  CK(up(ctx->o_blocks, ctx->dblocks.data(), sizeof(DevBlock) * ctx->dblocks.size()));
  for (const Group &G : ctx->grp) {
    CK(up(G.o_tiles, G.tiles.data(), sizeof(Tile) * G.tiles.size()));
    CK(up(G.o_wtiles, G.wtiles.data(), sizeof(Tile) * G.wtiles.size()));
    CK(up(G.o_stiles, G.stiles.data(), sizeof(Tile) * G.stiles.size()));
    CK(up(G.o_rtiles, G.rtiles.data(), sizeof(Tile) * G.rtiles.size()));
    CK(up(G.o_ptiles, G.ptiles.data(), sizeof(Tile) * G.ptiles.size()));
    CK(up(G.o_ztiles, G.ztiles.data(), sizeof(Tile) * G.ztiles.size()));
  }
  // tensor maps for the TMA-fed pre-pass: per block of a qualifying group
  // and shadow q, the 4-D tensor (x, y, z, field) of the block's FP32
  // shadow with boxes of PRE_TMA_PX x (PRE_TMA_PY + order) x 1 x 1
  if (ctx->has[1]) {
    const size_t nb = ctx->dblocks.size();
    std::vector<CUtensorMap> maps(2 * nb);
    std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
    std::vector<char> done(nb, 0);
    for (Group &G : ctx->grp) {
      if (!G.tma_pre) continue;
      for (const Tile &t : G.ztiles) {
        const int blk = t.block & TILE_BLOCK_MASK;
        if (done[blk]) continue;
        done[blk] = 1;
        const DevBlock &D = ctx->dblocks[blk];
        for (int q = 0; q < 2; ++q)
          if (!encode_shadow_map(&maps[q * nb + blk], ctx->d_sh(q) + D.off, D, G.order)) G.tma_pre = false;
      }
    }
    CK(up(ctx->o_tmap, maps.data(), sizeof(CUtensorMap) * maps.size()));
  }
  for (int p = 0; p < 2; ++p) {
    CK(up(ctx->o_somm[p], ctx->somm[p].data(), sizeof(CellRef) * ctx->somm[p].size()));
    CK(up(ctx->o_gcopy[p], ctx->gcopy[p].data(), sizeof(GhostCopy) * ctx->gcopy[p].size()));
  }
  CK(up(ctx->o_rghost, ctx->rghost.data(), sizeof(RestrictRef) * ctx->rghost.size()));
  CK(up(ctx->o_rbuf, ctx->rbuf.data(), sizeof(RestrictRef) * ctx->rbuf.size()));
  CK(up(ctx->o_rblocks, ctx->rblocks.data(), sizeof(int32_t) * ctx->rblocks.size()));
  CK(up(ctx->o_rbcopy, ctx->rbcopy.data(), sizeof(RbCopy) * ctx->rbcopy.size()));
  CK(up(ctx->o_krow, ctx->krow, sizeof ctx->krow));
  CK(up(ctx->o_cbcopy, ctx->cbcopy.data(), sizeof(CbCopy) * ctx->cbcopy.size()));
  CK(up(ctx->o_prol, ctx->prol.data(), sizeof(ProlongRef) * ctx->prol.size()));
  CK(up(ctx->o_pbox, ctx->pbox.data(), sizeof(PBox) * ctx->pbox.size()));
  CK(up(ctx->o_pslots, ctx->pslots.data(), sizeof(int32_t) * ctx->pslots.size()));
  CK(up(ctx->o_paxtab, ctx->paxtab.data(), sizeof(int32_t) * ctx->paxtab.size()));
  CK(up(ctx->o_pidx, ctx->pidx.data(), sizeof(int32_t) * ctx->pidx.size()));
  CK(up(ctx->o_wtab, ctx->wtab.data(), sizeof(double) * ctx->wtab.size()));
  CK(up(ctx->o_pw, ctx->pw, sizeof ctx->pw));
  CK(up(ctx->o_ctiles, ctx->ctiles.data(), sizeof(Tile) * ctx->ctiles.size()));
  CK(up(ctx->o_cfirst, ctx->cfirst.data(), sizeof(int32_t) * ctx->cfirst.size()));
  CK(cudaMemsetAsync(ctx->d_status(), 0, sizeof(int32_t), st));
  // the tables live in host vectors owned by ctx; wait so the copies are done
  CK(cudaStreamSynchronize(st));
  ctx->bound = true;
  ctx->shadow_valid = false;
  ctx->dt_dirty = true;
  return Z4C_OK;
}

}  // extern "C"
