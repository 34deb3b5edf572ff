// Context creation and binding (C ABI, include/z4c.h): validates each
// instance's Mesh of MeshBlocks (paper Sec. 3), builds the per-block
// descriptors, the interior tile lists of every (order, precision) group, the
// same-level ghost-copy lists and the Sommerfeld cell lists, and lays them out
// in the caller's scratch buffer.  No CUDA call happens before z4c_bind.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "z4c_ctx.cuh"

using namespace z4c;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
long long iround(double v) { return (long long)std::llround(v); }

int check_instance(const z4c_instance &I) {
  const z4c_params &p = I.params;
  if (I.fd_order != 4 && I.fd_order != 6) return Z4C_ERR_UNSUPPORTED;
  if (I.ghosts < I.fd_order / 2 + 1 || I.ghosts > 8) return Z4C_ERR_UNSUPPORTED;
  if (p.rhs_precision != 64 && p.rhs_precision != 32) return Z4C_ERR_UNSUPPORTED;
  if (p.lapse < 0 || p.lapse > 1 || p.shift < 0 || p.shift > 1) return Z4C_ERR_BAD_ARG;
  if (!(p.chi_floor > 0.0)) return Z4C_ERR_BAD_ARG;
  if (p.schedule < 0 || p.schedule > 2) return Z4C_ERR_BAD_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(I.mesh.hi[d] > I.mesh.lo[d])) return Z4C_ERR_BAD_MESH;
  return Z4C_OK;
}

// Blocks of one instance: one spacing and one size, tiling the mesh on a
// lattice.  Fills the global integer origin of each block and the lattice
// (block index per lattice cell, relative to the instance).
int check_blocks(const z4c_instance &I, const z4c_block *blocks, int count, std::vector<int> &lattice,
                 std::vector<std::array<long long, 3>> &go, long long N[3], long long nb[3]) {
  const double h = blocks[0].h;
  const int *n = blocks[0].n;
  if (!(h > 0.0)) return Z4C_ERR_BAD_MESH;
  for (int d = 0; d < 3; ++d)
    if (n[d] < I.ghosts) return Z4C_ERR_UNSUPPORTED;  // a ghost region must come from one neighbour
  for (int d = 0; d < 3; ++d) {
    const double v = (I.mesh.hi[d] - I.mesh.lo[d]) / h;
    N[d] = iround(v);
    if (std::fabs(v - N[d]) > 1e-8 * std::max(1.0, v) || N[d] % n[d] != 0) return Z4C_ERR_BAD_MESH;
    nb[d] = N[d] / n[d];
  }
  if (nb[0] * nb[1] * nb[2] != count) return Z4C_ERR_BAD_MESH;
  lattice.assign(count, -1);
  go.resize(count);
  for (int b = 0; b < count; ++b) {
    const z4c_block &B = blocks[b];
    if (B.level != 0) return Z4C_ERR_UNSUPPORTED;
    if (std::fabs(B.h - h) > 1e-12 * h) return Z4C_ERR_BAD_MESH;
    long long L[3];
    for (int d = 0; d < 3; ++d) {
      if (B.n[d] != n[d]) return Z4C_ERR_BAD_MESH;
      const double v = (B.lo[d] - I.mesh.lo[d]) / h;
      go[b][d] = iround(v);
      if (std::fabs(v - go[b][d]) > 1e-8 * std::max(1.0, std::fabs(v))) return Z4C_ERR_BAD_MESH;
      if (go[b][d] < 0 || go[b][d] % n[d] != 0) return Z4C_ERR_BAD_MESH;
      L[d] = go[b][d] / n[d];
      if (L[d] >= nb[d]) return Z4C_ERR_BAD_MESH;
    }
    const long long li = (L[2] * nb[1] + L[1]) * nb[0] + L[0];
    if (lattice[li] != -1) return Z4C_ERR_BAD_MESH;  // overlap
    lattice[li] = b;
  }
  return Z4C_OK;
}

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
  ctx->blocks.assign(blocks, blocks + nblocks);
  int64_t off = 0;
  bool sched_set[2] = {false, false};
  for (int i = 0; i < ninstances; ++i) {
    const z4c_instance &I = instances[i];
    std::vector<int> lattice;
    std::vector<std::array<long long, 3>> go;
    long long N[3], nb[3];
    const int r = check_blocks(I, blocks + first[i], count[i], lattice, go, N, nb);
    if (r) {
      delete ctx;
      return r;
    }
    Instance in;
    in.mesh = I.mesh;
    in.params = I.params;
    in.ghosts = I.ghosts;
    in.order = I.fd_order;
    in.first = first[i];
    in.count = count[i];
    ctx->inst.push_back(in);
    const bool f32 = I.params.rhs_precision == 32;
    const int p = f32 ? 1 : 0;
    ctx->has[p] = true;
    if (!sched_set[p]) {
      ctx->sched[p] = I.params.schedule == 1 ? 1 : 2;
      sched_set[p] = true;
    }
    const int g = I.ghosts, ord = I.fd_order;
    const int *n = blocks[first[i]].n;
    const double h = blocks[first[i]].h;
    const int e[3] = {n[0] + 2 * g, n[1] + 2 * g, n[2] + 2 * g};
    const long long S = (long long)e[0] * e[1] * e[2];
    if (S * NF >= (1LL << 31)) {
      delete ctx;
      return Z4C_ERR_UNSUPPORTED;
    }
    ctx->max_S = std::max(ctx->max_S, (int)S);
    const double den1 = ord == 4 ? 12.0 : 60.0, den2 = ord == 4 ? 12.0 : 180.0;
    const double kosg = ord == 4 ? 1.0 / 64.0 : -1.0 / 256.0;  // (-1)^(N+1) / 2^(2N)
    Group &G = ctx->grp[2 * (ord == 6) + (f32 ? 1 : 0)];
    G.order = ord;
    G.f32 = f32;
    for (int lb = 0; lb < count[i]; ++lb) {
      const int b = first[i] + lb;
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
      // interior tiles (fused kernel, constraints) and widened tiles (pre-pass)
      const int W = ord / 2;
      for (int k = 0; k < n[2]; ++k) {
        for (int j0 = 0; j0 < n[1]; j0 += TY)
          for (int i0 = 0; i0 < n[0]; i0 += TX) {
            G.tiles.push_back(Tile{b, i0, j0, k});
            ctx->ctiles.push_back(Tile{b, i0, j0, k});
          }
        for (int j0 = -W; j0 < n[1] + W; j0 += TY)
          for (int i0 = -W; i0 < n[0] + W; i0 += TX) G.wtiles.push_back(Tile{b, i0, j0, k});
      }
      // ghost cells: copies from the lattice neighbour, or Sommerfeld cells
      for (int k = 0; k < e[2]; ++k)
        for (int j = 0; j < e[1]; ++j)
          for (int ii = 0; ii < e[0]; ++ii) {
            const int idx[3] = {ii, j, k};
            bool interior = true;
            for (int d = 0; d < 3; ++d) interior &= idx[d] >= g && idx[d] < n[d] + g;
            if (interior) continue;
            long long Gc[3];
            bool outside = false;
            for (int d = 0; d < 3; ++d) {
              Gc[d] = go[lb][d] + idx[d] - g;
              if (I.mesh.periodic)
                Gc[d] = ((Gc[d] % N[d]) + N[d]) % N[d];
              else if (Gc[d] < 0 || Gc[d] >= N[d])
                outside = true;
            }
            const int cidx = (k * e[1] + j) * e[0] + ii;
            if (outside) {
              ctx->somm[p].push_back(CellRef{b, cidx});
              continue;
            }
            long long L[3], q[3];
            for (int d = 0; d < 3; ++d) {
              L[d] = Gc[d] / n[d];
              q[d] = Gc[d] - L[d] * n[d] + g;
            }
            const int src = first[i] + lattice[(L[2] * nb[1] + L[1]) * nb[0] + L[0]];
            const int scidx = (int)((q[2] * e[1] + q[1]) * e[0] + q[0]);
            ctx->gcopy[p].push_back(GhostCopy{b, cidx, src, scidx});
          }
    }
  }
  ctx->reg_elems = (size_t)off;

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
  }
  for (int p = 0; p < 2; ++p) {
    ctx->o_somm[p] = take(sizeof(CellRef) * ctx->somm[p].size());
    ctx->o_gcopy[p] = take(sizeof(GhostCopy) * ctx->gcopy[p].size());
  }
  ctx->o_ctiles = take(sizeof(Tile) * ctx->ctiles.size());
  ctx->o_part = take(sizeof(double) * 8 * 2 * ctx->ctiles.size());  // order-4 and order-6 records
  ctx->o_res = take(sizeof(double) * 8);
  ctx->o_dt = take(sizeof(double) * ctx->dblocks.size());
  if (ctx->has[1]) {
    ctx->o_sh0 = take(sizeof(float) * ctx->reg_elems);
    ctx->o_sh1 = take(sizeof(float) * ctx->reg_elems);
    ctx->o_ds32 = take(sizeof(float) * ctx->reg_elems);
  }
  if (ctx->has[0]) ctx->o_ds64 = take(sizeof(double) * ctx->reg_elems);
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
  }
  for (int p = 0; p < 2; ++p) {
    CK(up(ctx->o_somm[p], ctx->somm[p].data(), sizeof(CellRef) * ctx->somm[p].size()));
    CK(up(ctx->o_gcopy[p], ctx->gcopy[p].data(), sizeof(GhostCopy) * ctx->gcopy[p].size()));
  }
  CK(up(ctx->o_ctiles, ctx->ctiles.data(), sizeof(Tile) * ctx->ctiles.size()));
  // the tables live in host vectors owned by ctx; wait so the copies are done
  CK(cudaStreamSynchronize(st));
  ctx->bound = true;
  ctx->shadow_valid = false;
  ctx->dt_dirty = true;
  return Z4C_OK;
}

}  // extern "C"
