// Host side of the C ABI declared in include/z4c.h.
//
// The context owns only host-side descriptors and CUDA graphs; every device
// buffer (state registers, scratch holding the descriptor tables and work
// lists) belongs to the caller.  All work is enqueued on the caller's stream.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "z4c.h"
#include "z4c_internal.cuh"

using namespace z4c;

struct z4c_ctx {
  z4c_mesh mesh;
  z4c_params params;
  int ghosts = 0, order = 0, nblocks = 0;
  std::vector<z4c_block> blocks;
  std::vector<DevBlock> dblocks;
  std::vector<Tile> tiles;
  std::vector<Tile> wtiles;  // interior widened by order/2 in x and y (pre-pass)
  std::vector<CellRef> somm;
  std::vector<GhostCopy> gcopy;
  size_t reg_elems = 0;
  int max_S = 0;
  // scratch layout (byte offsets)
  size_t o_blocks = 0, o_tiles = 0, o_wtiles = 0, o_somm = 0, o_gcopy = 0, o_part = 0, o_res = 0,
         o_sh0 = 0, o_sh1 = 0, o_dstore = 0, scratch_total = 0;
  // bound buffers
  double *reg[4] = {nullptr, nullptr, nullptr, nullptr};
  char *scratch = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  bool shadow_valid = false;
  // graph of one RK4 step
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  std::string err;

  int sched = 2;  // 1 single fused kernel, 2 pre-pass + fused kernel
  int occ = 1;    // resident CTAs per SM the fused kernel is compiled for (1, 2, 4)
  bool f32() const { return params.rhs_precision == 32; }
  bool pre() const { return sched == 2; }
  const Tile *d_wtiles() const { return (const Tile *)(scratch + o_wtiles); }
  void *d_dstore() const { return pre() ? (void *)(scratch + o_dstore) : nullptr; }
  const DevBlock *d_blocks() const { return (const DevBlock *)(scratch + o_blocks); }
  const Tile *d_tiles() const { return (const Tile *)(scratch + o_tiles); }
  const CellRef *d_somm() const { return (const CellRef *)(scratch + o_somm); }
  const GhostCopy *d_gcopy() const { return (const GhostCopy *)(scratch + o_gcopy); }
  double *d_part() const { return (double *)(scratch + o_part); }
  double *d_res() const { return (double *)(scratch + o_res); }
  float *d_sh(int q) const { return (float *)(scratch + (q == 0 ? o_sh0 : o_sh1)); }
};

namespace {

int fail(z4c_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, Z4C_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                 \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

long long iround(double v) { return (long long)std::llround(v); }

}  // namespace

extern "C" {

int z4c_create(const z4c_mesh *mesh, const z4c_block *blocks, int nblocks, int ghosts, int fd_order,
               const z4c_params *params, z4c_ctx **out) {
  if (!out) return Z4C_ERR_BAD_ARG;
  *out = nullptr;
  if (!mesh || !blocks || !params || nblocks <= 0) return Z4C_ERR_BAD_ARG;
  if (fd_order != 4 && fd_order != 6) return Z4C_ERR_UNSUPPORTED;
  if (ghosts < fd_order / 2 + 1 || ghosts > 8) return Z4C_ERR_UNSUPPORTED;
  if (params->rhs_precision != 64 && params->rhs_precision != 32) return Z4C_ERR_UNSUPPORTED;
  if (params->lapse < 0 || params->lapse > 1 || params->shift < 0 || params->shift > 1) return Z4C_ERR_BAD_ARG;
  if (!(params->chi_floor > 0.0)) return Z4C_ERR_BAD_ARG;
  if (params->schedule < 0 || params->schedule > 2) return Z4C_ERR_BAD_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(mesh->hi[d] > mesh->lo[d])) return Z4C_ERR_BAD_MESH;

  // all blocks on one level with one spacing and one size
  const double h = blocks[0].h;
  int n[3] = {blocks[0].n[0], blocks[0].n[1], blocks[0].n[2]};
  if (!(h > 0.0)) return Z4C_ERR_BAD_MESH;
  for (int d = 0; d < 3; ++d)
    if (n[d] < ghosts) return Z4C_ERR_UNSUPPORTED;  // a ghost region must come from one neighbour
  long long N[3];
  for (int d = 0; d < 3; ++d) {
    double v = (mesh->hi[d] - mesh->lo[d]) / h;
    N[d] = iround(v);
    if (std::fabs(v - N[d]) > 1e-8 * std::max(1.0, v) || N[d] % n[d] != 0) return Z4C_ERR_BAD_MESH;
  }
  const long long nb[3] = {N[0] / n[0], N[1] / n[1], N[2] / n[2]};
  if (nb[0] * nb[1] * nb[2] != nblocks) return Z4C_ERR_BAD_MESH;
  std::vector<int> lattice(nblocks, -1);
  std::vector<std::array<long long, 3>> go(nblocks);
  for (int b = 0; b < nblocks; ++b) {
    const z4c_block &B = blocks[b];
    if (B.level != 0 || B.instance != 0) return Z4C_ERR_UNSUPPORTED;
    if (std::fabs(B.h - h) > 1e-12 * h) return Z4C_ERR_BAD_MESH;
    long long L[3];
    for (int d = 0; d < 3; ++d) {
      if (B.n[d] != n[d]) return Z4C_ERR_BAD_MESH;
      double v = (B.lo[d] - mesh->lo[d]) / h;
      go[b][d] = iround(v);
      if (std::fabs(v - go[b][d]) > 1e-8 * std::max(1.0, std::fabs(v))) return Z4C_ERR_BAD_MESH;
      if (go[b][d] < 0 || go[b][d] % n[d] != 0) return Z4C_ERR_BAD_MESH;
      L[d] = go[b][d] / n[d];
      if (L[d] >= nb[d]) return Z4C_ERR_BAD_MESH;
    }
    long long li = (L[2] * nb[1] + L[1]) * nb[0] + L[0];
    if (lattice[li] != -1) return Z4C_ERR_BAD_MESH;  // overlap
    lattice[li] = b;
  }

  z4c_ctx *ctx = new z4c_ctx();
  ctx->mesh = *mesh;
  ctx->params = *params;
  ctx->ghosts = ghosts;
  ctx->order = fd_order;
  ctx->nblocks = nblocks;
  ctx->blocks.assign(blocks, blocks + nblocks);

  const int g = ghosts;
  const int e[3] = {n[0] + 2 * g, n[1] + 2 * g, n[2] + 2 * g};
  const int S = e[0] * e[1] * e[2];
  if ((long long)S * NF >= (1LL << 31)) {
    delete ctx;
    return Z4C_ERR_UNSUPPORTED;
  }
  ctx->max_S = S;
  const double den1 = fd_order == 4 ? 12.0 : 60.0;
  const double den2 = fd_order == 4 ? 12.0 : 180.0;
  const double kosg = fd_order == 4 ? 1.0 / 64.0 : -1.0 / 256.0;  // (-1)^(N+1) / 2^(2N)
  for (int b = 0; b < nblocks; ++b) {
    DevBlock D{};
    for (int d = 0; d < 3; ++d) {
      D.n[d] = n[d];
      D.e[d] = e[d];
      D.lo[d] = blocks[b].lo[d];
    }
    D.g = g;
    D.order = fd_order;
    D.S = S;
    D.off = (int64_t)b * NF * S;
    D.h = h;
    D.s1 = 1.0 / (den1 * h);
    D.s2 = 1.0 / (den2 * h * h);
    D.smix = 1.0 / (den1 * den1 * h * h);
    D.slop = 1.0 / (den1 * h);
    D.sko = kosg * params->ko_sigma / h;
    D.s1f = (float)D.s1;
    D.s2f = (float)D.s2;
    D.smixf = (float)D.smix;
    D.slopf = (float)D.slop;
    D.skof = (float)D.sko;
    D.hf = (float)h;
    D.kappa1 = params->kappa1;
    D.kappa2 = params->kappa2;
    D.eta = params->eta;
    D.chi_floor = params->chi_floor;
    D.lapse = params->lapse;
    D.shift = params->shift;
    ctx->dblocks.push_back(D);
  }
  ctx->reg_elems = (size_t)nblocks * NF * S;

  // work lists: interior tiles, Sommerfeld cells, ghost copies
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < n[2]; ++k)
      for (int j0 = 0; j0 < n[1]; j0 += TY)
        for (int i0 = 0; i0 < n[0]; i0 += TX) ctx->tiles.push_back(Tile{b, i0, j0, k});
  // schedule: 0 = default (the pre-pass, faster for both precisions),
  // 1 = single fused kernel, 2 = y/z pre-pass + fused kernel.  The tables
  // of both are built so that z4c_autotune can switch.
  ctx->sched = params->schedule == 1 ? 1 : 2;
  ctx->occ = params->rhs_precision == 32 ? 4 : 1;
  {
    const int W = fd_order / 2;
    for (int b = 0; b < nblocks; ++b)
      for (int k = 0; k < n[2]; ++k)
        for (int j0 = -W; j0 < n[1] + W; j0 += TY)
          for (int i0 = -W; i0 < n[0] + W; i0 += TX) ctx->wtiles.push_back(Tile{b, i0, j0, k});
  }
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < e[2]; ++k)
      for (int j = 0; j < e[1]; ++j)
        for (int i = 0; i < e[0]; ++i) {
          const int idx[3] = {i, j, k};
          bool interior = true;
          for (int d = 0; d < 3; ++d) interior &= idx[d] >= g && idx[d] < n[d] + g;
          if (interior) continue;
          long long G[3];
          bool outside = false;
          for (int d = 0; d < 3; ++d) {
            G[d] = go[b][d] + idx[d] - g;
            if (mesh->periodic) {
              G[d] = ((G[d] % N[d]) + N[d]) % N[d];
            } else if (G[d] < 0 || G[d] >= N[d]) {
              outside = true;
            }
          }
          const int cidx = (k * e[1] + j) * e[0] + i;
          if (outside) {
            ctx->somm.push_back(CellRef{b, cidx});
            continue;
          }
          long long L[3], q[3];
          for (int d = 0; d < 3; ++d) {
            L[d] = G[d] / n[d];
            q[d] = G[d] - L[d] * n[d] + g;
          }
          const int src = lattice[(L[2] * nb[1] + L[1]) * nb[0] + L[0]];
          const int scidx = (int)((q[2] * e[1] + q[1]) * e[0] + q[0]);
          ctx->gcopy.push_back(GhostCopy{b, cidx, src, scidx});
        }

  // scratch layout
  size_t o = 0;
  ctx->o_blocks = o;
  o = align256(o + sizeof(DevBlock) * ctx->dblocks.size());
  ctx->o_tiles = o;
  o = align256(o + sizeof(Tile) * ctx->tiles.size());
  ctx->o_wtiles = o;
  o = align256(o + sizeof(Tile) * ctx->wtiles.size());
  ctx->o_somm = o;
  o = align256(o + sizeof(CellRef) * std::max<size_t>(1, ctx->somm.size()));
  ctx->o_gcopy = o;
  o = align256(o + sizeof(GhostCopy) * std::max<size_t>(1, ctx->gcopy.size()));
  ctx->o_part = o;
  o = align256(o + sizeof(double) * 8 * ctx->tiles.size());
  ctx->o_res = o;
  o = align256(o + sizeof(double) * 8);
  if (ctx->f32()) {
    ctx->o_sh0 = o;
    o = align256(o + sizeof(float) * ctx->reg_elems);
    ctx->o_sh1 = o;
    o = align256(o + sizeof(float) * ctx->reg_elems);
  }
  {
    ctx->o_dstore = o;
    o = align256(o + (ctx->f32() ? sizeof(float) : sizeof(double)) * ctx->reg_elems);
  }
  ctx->scratch_total = o;
  *out = ctx;
  return Z4C_OK;
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
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->scratch + ctx->o_blocks, ctx->dblocks.data(),
                     sizeof(DevBlock) * ctx->dblocks.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->scratch + ctx->o_tiles, ctx->tiles.data(), sizeof(Tile) * ctx->tiles.size(),
                     cudaMemcpyHostToDevice, st));
  if (!ctx->wtiles.empty())
    CK(cudaMemcpyAsync(ctx->scratch + ctx->o_wtiles, ctx->wtiles.data(), sizeof(Tile) * ctx->wtiles.size(),
                       cudaMemcpyHostToDevice, st));
  if (!ctx->somm.empty())
    CK(cudaMemcpyAsync(ctx->scratch + ctx->o_somm, ctx->somm.data(), sizeof(CellRef) * ctx->somm.size(),
                       cudaMemcpyHostToDevice, st));
  if (!ctx->gcopy.empty())
    CK(cudaMemcpyAsync(ctx->scratch + ctx->o_gcopy, ctx->gcopy.data(),
                       sizeof(GhostCopy) * ctx->gcopy.size(), cudaMemcpyHostToDevice, st));
  // the tables live in host vectors owned by ctx; wait so the copies are done
  CK(cudaStreamSynchronize(st));
  ctx->bound = true;
  ctx->shadow_valid = false;
  return Z4C_OK;
}

}  // extern "C"

namespace {

int ensure_bound(z4c_ctx *ctx) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  if (!ctx->bound) return fail(ctx, Z4C_ERR_NOT_BOUND, "z4c_bind has not been called");
  return Z4C_OK;
}

int fill_ghosts_f64(z4c_ctx *ctx, double *reg) {
  CK(launch_ghosts_f64(reg, ctx->d_blocks(), ctx->d_gcopy(), (int)ctx->gcopy.size(), ctx->stream));
  return Z4C_OK;
}

int fill_ghosts_f32(z4c_ctx *ctx, float *reg) {
  CK(launch_ghosts_f32(reg, ctx->d_blocks(), ctx->d_gcopy(), (int)ctx->gcopy.size(), ctx->stream));
  return Z4C_OK;
}

int launch_prepass(z4c_ctx *ctx, const StageArgs &a) {
  if (!ctx->pre()) return Z4C_OK;
  const int nw = (int)ctx->wtiles.size();
  CK(ctx->f32() ? launch_prepass_f32(ctx->order, a, ctx->d_wtiles(), nw, ctx->stream)
                : launch_prepass_f64(ctx->order, a, ctx->d_wtiles(), nw, ctx->stream));
  return Z4C_OK;
}

int launch_fused(z4c_ctx *ctx, const StageArgs &a) {
  const int nt = (int)ctx->tiles.size();
  if (!ctx->f32()) {
    CK(launch_fused_f64(ctx->order, a, ctx->d_tiles(), nt, ctx->pre(), ctx->stream));
  } else if (ctx->pre() && ctx->occ == 4) {
    CK(launch_fused_pre_f32_occ4(ctx->order, a, ctx->d_tiles(), nt, ctx->stream));
  } else if (ctx->pre() && ctx->occ == 2) {
    CK(launch_fused_pre_f32_occ2(ctx->order, a, ctx->d_tiles(), nt, ctx->stream));
  } else {
    CK(launch_fused_f32(ctx->order, a, ctx->d_tiles(), nt, ctx->pre(), ctx->stream));
  }
  return Z4C_OK;
}

int launch_stage(z4c_ctx *ctx, StageArgs a) {
  a.dstore = ctx->d_dstore();
  int r = launch_prepass(ctx, a);
  if (r) return r;
  r = launch_fused(ctx, a);
  if (r) return r;
  CK(launch_sommerfeld(ctx->f32(), a, ctx->d_somm(), (int)ctx->somm.size(), ctx->stream));
  return Z4C_OK;
}

// Enqueue one classic RK4 step (paper Sec. 3: ghost fill at every stage).
// Registers: X = (U0, A, B, A) are the stage states, next = (A, B, A, U0).
int enqueue_step(z4c_ctx *ctx, double dt) {
  double *U0 = ctx->reg[0], *SA = ctx->reg[1], *SB = ctx->reg[2], *ACC = ctx->reg[3];
  double *X[4] = {U0, SA, SB, SA};
  double *NX[4] = {SA, SB, SA, U0};
  const double ca[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  const double cb[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
  const int mode[4] = {MODE_S1, MODE_S23, MODE_S23, MODE_S4};
  for (int s = 0; s < 4; ++s) {
    StageArgs a{};
    a.blocks = ctx->d_blocks();
    a.x64 = X[s];
    a.u0 = U0;
    a.acc = ACC;
    a.next = NX[s];
    a.ca = ca[s];
    a.cb = cb[s];
    a.caf = (float)ca[s];
    a.cbf = (float)cb[s];
    a.mode = mode[s];
    if (ctx->f32()) {
      float *sh = ctx->d_sh(s % 2), *nsh = ctx->d_sh((s + 1) % 2);
      int r = fill_ghosts_f32(ctx, sh);
      if (r) return r;
      a.x32 = sh;
      a.next32 = nsh;
      a.next_full = s == 3;
    } else {
      int r = fill_ghosts_f64(ctx, X[s]);
      if (r) return r;
    }
    int r = launch_stage(ctx, a);
    if (r) return r;
  }
  return Z4C_OK;
}

int ensure_shadow(z4c_ctx *ctx) {
  if (!ctx->f32() || ctx->shadow_valid) return Z4C_OK;
  CK(launch_to_shadow(ctx->reg[0], ctx->d_sh(0), ctx->d_blocks(), ctx->nblocks, ctx->max_S, ctx->stream));
  ctx->shadow_valid = true;
  return Z4C_OK;
}

}  // namespace

extern "C" {

int z4c_set_initial_data(z4c_ctx *ctx, int kind, const double *params, int nparams) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (kind < 0 || kind > 4 || nparams < 0 || nparams > 64 || (nparams > 0 && !params))
    return fail(ctx, Z4C_ERR_BAD_ARG, "bad initial-data kind or parameters");
  const int need[5] = {0, 3, 3, 2, 1};
  if (nparams < need[kind]) return fail(ctx, Z4C_ERR_BAD_ARG, "too few initial-data parameters");
  if (kind == 4 && nparams < 1 + 4 * (int)params[0])
    return fail(ctx, Z4C_ERR_BAD_ARG, "too few Brill-Lindquist parameters");
  CK(launch_initial_data(ctx->reg[0], ctx->d_blocks(), ctx->nblocks, ctx->max_S, kind, params, nparams,
                         ctx->stream));
  ctx->shadow_valid = false;
  return Z4C_OK;
}

int z4c_fill_ghosts(z4c_ctx *ctx, int reg) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3) return fail(ctx, Z4C_ERR_BAD_ARG, "register index out of range");
  if (reg == 0) ctx->shadow_valid = false;
  return fill_ghosts_f64(ctx, ctx->reg[reg]);
}

int z4c_rhs(z4c_ctx *ctx, int reg, void *rhs_out) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3 || !rhs_out) return fail(ctx, Z4C_ERR_BAD_ARG, "bad register or output");
  CK(cudaMemsetAsync(rhs_out, 0, ctx->reg_elems * sizeof(double), ctx->stream));
  StageArgs a{};
  a.blocks = ctx->d_blocks();
  a.x64 = ctx->reg[reg];
  a.rhs_out = (double *)rhs_out;
  a.mode = MODE_RHS;
  if (ctx->f32()) {
    // shadow of the register in the second shadow buffer (the first may hold U0's)
    CK(launch_to_shadow(ctx->reg[reg], ctx->d_sh(1), ctx->d_blocks(), ctx->nblocks, ctx->max_S,
                        ctx->stream));
    a.x32 = ctx->d_sh(1);
  }
  return launch_stage(ctx, a);
}

int z4c_rk4_step(z4c_ctx *ctx, double dt, int nsteps) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (nsteps < 0 || !std::isfinite(dt)) return fail(ctx, Z4C_ERR_BAD_ARG, "bad dt or nsteps");
  if (nsteps == 0) return Z4C_OK;
  r = ensure_shadow(ctx);
  if (r) return r;
  if (ctx->stream == nullptr) {  // legacy default stream: no capture, plain launches
    for (int s = 0; s < nsteps; ++s) {
      r = enqueue_step(ctx, dt);
      if (r) return r;
    }
    return Z4C_OK;
  }
  if (!ctx->graph || ctx->graph_dt != dt) {
    if (ctx->graph) {
      cudaGraphExecDestroy(ctx->graph);
      ctx->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    r = enqueue_step(ctx, dt);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (r) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    CK(e);
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    ctx->graph_dt = dt;
  }
  for (int s = 0; s < nsteps; ++s) CK(cudaGraphLaunch(ctx->graph, ctx->stream));
  return Z4C_OK;
}

int z4c_constraints(z4c_ctx *ctx, double r_mask, double *norms, void *per_cell_out) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (!norms) return fail(ctx, Z4C_ERR_BAD_ARG, "norms is null");
  r = fill_ghosts_f64(ctx, ctx->reg[0]);
  if (r) return r;
  if (per_cell_out)
    CK(cudaMemsetAsync(per_cell_out, 0, ctx->reg_elems / NF * 4 * sizeof(double), ctx->stream));
  CK(launch_constraints(ctx->order, ctx->reg[0], ctx->d_blocks(), ctx->d_tiles(), (int)ctx->tiles.size(),
                        r_mask, (double *)per_cell_out, ctx->d_part(), ctx->d_res(), ctx->stream));
  double res[6];
  CK(cudaMemcpyAsync(res, ctx->d_res(), sizeof res, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < 6; ++q) norms[q] = res[q];
  for (int q = 0; q < 6; ++q)
    if (std::isnan(res[q])) return fail(ctx, Z4C_ERR_NAN, "constraint norm %d is NaN", q);
  return Z4C_OK;
}

int z4c_get_state(z4c_ctx *ctx, int reg, void *host, size_t bytes) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3 || !host || bytes != ctx->reg_elems * sizeof(double))
    return fail(ctx, Z4C_ERR_BAD_ARG, "bad register, pointer or size");
  CK(cudaMemcpyAsync(host, ctx->reg[reg], bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return Z4C_OK;
}

int z4c_set_state(z4c_ctx *ctx, int reg, const void *host, size_t bytes) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3 || !host || bytes != ctx->reg_elems * sizeof(double))
    return fail(ctx, Z4C_ERR_BAD_ARG, "bad register, pointer or size");
  CK(cudaMemcpyAsync(ctx->reg[reg], host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (reg == 0) ctx->shadow_valid = false;
  return Z4C_OK;
}

int z4c_evolve_host(z4c_ctx *ctx, const void *host_in, void *host_out, size_t bytes, double dt,
                    int nsteps) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (!host_in || !host_out || bytes != ctx->reg_elems * sizeof(double))
    return fail(ctx, Z4C_ERR_BAD_ARG, "bad host buffers or size");
  CK(cudaMemcpyAsync(ctx->reg[0], host_in, bytes, cudaMemcpyHostToDevice, ctx->stream));
  ctx->shadow_valid = false;
  r = z4c_rk4_step(ctx, dt, nsteps);
  if (r) return r;
  CK(cudaMemcpyAsync(host_out, ctx->reg[0], bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return Z4C_OK;
}

int z4c_sync(z4c_ctx *ctx) {
  int r = ensure_bound(ctx);
  if (r) return r;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  return Z4C_OK;
}

int z4c_profile_steps(z4c_ctx *ctx, double dt, int nsteps, double *ms) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (!ms || nsteps <= 0 || !std::isfinite(dt)) return fail(ctx, Z4C_ERR_BAD_ARG, "bad arguments");
  r = ensure_shadow(ctx);
  if (r) return r;
  cudaEvent_t ev[2];
  CK(cudaEventCreate(&ev[0]));
  CK(cudaEventCreate(&ev[1]));
  double acc[4] = {0, 0, 0, 0};
  double *U0 = ctx->reg[0], *SA = ctx->reg[1], *SB = ctx->reg[2], *ACC = ctx->reg[3];
  double *X[4] = {U0, SA, SB, SA};
  double *NX[4] = {SA, SB, SA, U0};
  const double ca[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  const double cb[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
  const int mode[4] = {MODE_S1, MODE_S23, MODE_S23, MODE_S4};
  auto timed = [&](int kind, auto &&launch) -> int {
    CK(cudaEventRecord(ev[0], ctx->stream));
    CK(launch());
    CK(cudaEventRecord(ev[1], ctx->stream));
    CK(cudaEventSynchronize(ev[1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ev[0], ev[1]));
    acc[kind] += t;
    return Z4C_OK;
  };
  for (int step = 0; step < nsteps; ++step)
    for (int s = 0; s < 4; ++s) {
      StageArgs a{};
      a.blocks = ctx->d_blocks();
      a.x64 = X[s];
      a.u0 = U0;
      a.acc = ACC;
      a.next = NX[s];
      a.ca = ca[s];
      a.cb = cb[s];
      a.caf = (float)ca[s];
      a.cbf = (float)cb[s];
      a.mode = mode[s];
      float *sh = nullptr;
      if (ctx->f32()) {
        sh = ctx->d_sh(s % 2);
        a.x32 = sh;
        a.next32 = ctx->d_sh((s + 1) % 2);
        a.next_full = s == 3;
      }
      const int ng = (int)ctx->gcopy.size(), nt = (int)ctx->tiles.size(), ns = (int)ctx->somm.size();
      if (ng) {
        r = timed(0, [&] {
          return ctx->f32() ? launch_ghosts_f32(sh, ctx->d_blocks(), ctx->d_gcopy(), ng, ctx->stream)
                            : launch_ghosts_f64(X[s], ctx->d_blocks(), ctx->d_gcopy(), ng, ctx->stream);
        });
        if (r) return r;
      }
      a.dstore = ctx->d_dstore();
      if (ctx->pre()) {
        r = timed(3, [&] { return launch_prepass(ctx, a) ? cudaErrorUnknown : cudaSuccess; });
        if (r) return r;
      }
      r = timed(1, [&] { return launch_fused(ctx, a) ? cudaErrorUnknown : cudaSuccess; });
      if (r) return r;
      if (ns) {
        r = timed(2, [&] { return launch_sommerfeld(ctx->f32(), a, ctx->d_somm(), ns, ctx->stream); });
        if (r) return r;
      }
    }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  for (int q = 0; q < 4; ++q) ms[q] = acc[q] / nsteps;
  return Z4C_OK;
}

int z4c_set_variant(z4c_ctx *ctx, int schedule, int occupancy) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  if (schedule != 1 && schedule != 2) return fail(ctx, Z4C_ERR_BAD_ARG, "schedule must be 1 or 2");
  const bool ok = occupancy == 1 || (ctx->f32() && schedule == 2 && (occupancy == 2 || occupancy == 4));
  if (!ok) return fail(ctx, Z4C_ERR_UNSUPPORTED, "no kernel built for this schedule/occupancy");
  ctx->sched = schedule;
  ctx->occ = occupancy;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return Z4C_OK;
}

int z4c_autotune(z4c_ctx *ctx, int reps, int *schedule_out, int *occupancy_out) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reps < 1) return fail(ctx, Z4C_ERR_BAD_ARG, "reps must be >= 1");
  r = ensure_shadow(ctx);
  if (r) return r;
  // stage 1 reads U0 (and its FP32 shadow) and writes ACC and stage A only
  StageArgs a{};
  a.blocks = ctx->d_blocks();
  a.x64 = ctx->reg[0];
  a.u0 = ctx->reg[0];
  a.acc = ctx->reg[3];
  a.next = ctx->reg[1];
  a.ca = a.cb = 0.0;
  a.caf = a.cbf = 0.0f;
  a.mode = MODE_S1;
  if (ctx->f32()) {
    a.x32 = ctx->d_sh(0);
    a.next32 = ctx->d_sh(1);
  }
  struct Cand { int sched, occ; };
  std::vector<Cand> cands = {{1, 1}, {2, 1}};
  if (ctx->f32()) {
    cands.push_back({2, 2});
    cands.push_back({2, 4});
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  Cand pick = {ctx->sched, ctx->occ};
  for (const Cand &c : cands) {
    ctx->sched = c.sched;
    ctx->occ = c.occ;
    for (int rep = 0; rep <= reps; ++rep) {  // first pass untimed
      if (rep == 1) CK(cudaEventRecord(e0, ctx->stream));
      r = ctx->f32() ? fill_ghosts_f32(ctx, ctx->d_sh(0)) : fill_ghosts_f64(ctx, ctx->reg[0]);
      if (r) return r;
      r = launch_stage(ctx, a);
      if (r) return r;
    }
    CK(cudaEventRecord(e1, ctx->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->sched = pick.sched;
  ctx->occ = pick.occ;
  if (ctx->graph) {  // the next z4c_rk4_step captures the chosen kernels
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (schedule_out) *schedule_out = pick.sched;
  if (occupancy_out) *occupancy_out = pick.occ;
  return Z4C_OK;
}

int z4c_peak_fma(int fp64, void *cuda_stream, double *flops_per_s) {
  if (!flops_per_s) return Z4C_ERR_BAD_ARG;
  z4c_ctx *ctx = nullptr;
  CK(peak_fma(fp64 != 0, (cudaStream_t)cuda_stream, flops_per_s));
  return Z4C_OK;
}

int z4c_launches_per_step(const z4c_ctx *ctx) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  const int per_stage = (ctx->gcopy.empty() ? 0 : 1) + (ctx->pre() ? 2 : 1) + (ctx->somm.empty() ? 0 : 1);
  return 4 * per_stage;
}

const char *z4c_last_error(const z4c_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void z4c_destroy(z4c_ctx *ctx) {
  if (!ctx) return;
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  delete ctx;
}

}  // extern "C"
