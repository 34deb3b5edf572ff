// The C ABI calls that enqueue GPU work (include/z4c.h): initial data, ghost
// fill, right-hand side, RK4 steps through a CUDA graph, constraints, state
// copies, measurement aids and the kernel-variant tuner.  Context creation
// and binding are in z4c_build.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "z4c_ctx.cuh"

using namespace z4c;

namespace {

// classic RK4: next = base + FA[s] dt k_s, acc = acc + FB[s] dt k_s
constexpr double FA[4] = {0.5, 0.5, 1.0, 0.0};
constexpr double FB[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
constexpr int MODES[4] = {MODE_S1, MODE_S23, MODE_S23, MODE_S4};

int ensure_bound(z4c_ctx *ctx) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  if (!ctx->bound) return fail(ctx, Z4C_ERR_NOT_BOUND, "z4c_bind has not been called");
  return Z4C_OK;
}

// ghost fill of a stage state: FP64 blocks in the FP64 register, FP32-RHS
// blocks in their FP32 shadow (sh == nullptr: every block in the FP64 register)
int fill_ghosts(z4c_ctx *ctx, double *reg, float *sh) {
  for (int p = 0; p < 2; ++p) {
    const int n = (int)ctx->gcopy[p].size();
    if (!n) continue;
    if (p == 1 && sh)
      CK(launch_ghosts_f32(sh, ctx->d_blocks(), ctx->d_gcopy(1), n, ctx->stream));
    else
      CK(launch_ghosts_f64(reg, ctx->d_blocks(), ctx->d_gcopy(p), n, ctx->stream));
  }
  if (ctx->smr()) {  // refinement boundaries (FP64 instances only)
    const DevBlock *B = ctx->d_blocks();
    const double *wtab = ctx->at<double>(ctx->o_wtab);
    // phase 1: everything reads active cells only
    if (ctx->rb_mode) {
      double *rb = (double *)(ctx->scratch + ctx->o_rb);
      CK(launch_restrict_blocks(reg, B, ctx->at<int32_t>(ctx->o_rblocks), (int)ctx->rblocks.size(), wtab,
                                ctx->at<int32_t>(ctx->o_krow), rb, ctx->stream));
      CK(launch_rb_scatter(reg, B, ctx->at<RbCopy>(ctx->o_rbcopy), (int)ctx->rbcopy.size(), rb, ctx->d_cb(),
                           ctx->ncb, ctx->stream));
    } else {
      CK(launch_restrict(reg, B, ctx->at<RestrictRef>(ctx->o_rghost), (int)ctx->rghost.size(), wtab, false,
                         ctx->d_cb(), ctx->ncb, ctx->stream));
      CK(launch_restrict(reg, B, ctx->at<RestrictRef>(ctx->o_rbuf), (int)ctx->rbuf.size(), wtab, true,
                         ctx->d_cb(), ctx->ncb, ctx->stream));
    }
    CK(launch_cb_copy(reg, B, ctx->at<CbCopy>(ctx->o_cbcopy), (int)ctx->cbcopy.size(), ctx->d_cb(), ctx->ncb,
                      ctx->stream));
    // phase 2: prolongation from the coarse buffer (whole ghost regions as
    // boxes, the other parents one by one)
    CK(launch_prolong_boxes(reg, B, ctx->at<PBox>(ctx->o_pbox), (int)ctx->pbox.size(),
                            ctx->at<int32_t>(ctx->o_pslots), ctx->at<int32_t>(ctx->o_paxtab), ctx->d_cb(),
                            ctx->ncb, ctx->at<double>(ctx->o_pw), ctx->stream));
    CK(launch_prolong(reg, B, ctx->at<ProlongRef>(ctx->o_prol), (int)ctx->prol.size(),
                      ctx->at<int32_t>(ctx->o_pidx), ctx->d_cb(), ctx->ncb, ctx->at<double>(ctx->o_pw),
                      ctx->stream));
  }
  return Z4C_OK;
}

// A kernel whose bounded device-side wait gave up has set the status word:
// report it (once) after the stream has drained.
int status_check(z4c_ctx *ctx) {
  int32_t st = 0;
  CK(cudaMemcpyAsync(&st, ctx->d_status(), sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st == 0) return Z4C_OK;
  CK(cudaMemsetAsync(ctx->d_status(), 0, sizeof(int32_t), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return fail(ctx, Z4C_ERR_TIMEOUT,
              "a bounded wait on bulk copies (mbarrier) gave up in a kernel; results of that launch are invalid");
}

// The side stream and events of the Sommerfeld branch (created once).
int ensure_side(z4c_ctx *ctx) {
  if (!ctx->fork_somm || ctx->side) return Z4C_OK;
  CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  return Z4C_OK;
}

StageArgs group_args(const z4c_ctx *ctx, StageArgs a, bool f32) {
  if (!f32) {
    a.x32 = nullptr;
    a.next32 = nullptr;
  }
  a.dstore = ctx->d_dstore(f32);
  return a;
}

int launch_prepass_group(z4c_ctx *ctx, int g, const StageArgs &a) {
  const Group &G = ctx->grp[g];
  const int p = G.f32 ? 1 : 0;
  if (G.empty() || ctx->sched[p] < 2) return Z4C_OK;
  if (G.f32 && G.tma_pre && ctx->pre_tma) {
    // the TMA-fed kernel, with the tensor maps of the shadow being read
    const int q = a.x32 == ctx->d_sh(0) ? 0 : a.x32 == ctx->d_sh(1) ? 1 : -1;
    if (q >= 0) {
      StageArgs at = a;
      at.tmap32 = ctx->d_tmap(q);
      CK(launch_prepass_tma_f32(G.order, at, ctx->at<Tile>(G.o_ztiles), (int)G.ztiles.size(), ctx->stream));
      return Z4C_OK;
    }
  }
  const int nw = (int)G.wtiles.size();
  CK(G.f32 ? launch_prepass_f32(G.order, a, ctx->d_wtiles(g), nw, ctx->stream)
           : launch_prepass_f64(G.order, a, ctx->d_wtiles(g), nw, ctx->stream));
  return Z4C_OK;
}

int launch_fused_group(z4c_ctx *ctx, int g, const StageArgs &a) {
  const Group &G = ctx->grp[g];
  if (G.empty()) return Z4C_OK;
  const int p = G.f32 ? 1 : 0;
  const bool pre = ctx->sched[p] >= 2;
  const Tile *tl = ctx->d_tiles(g);
  int nt = (int)G.tiles.size();
  if (G.f32 && ctx->sched[1] >= 4) {
    // 4: split RHS kernels + one stage-update kernel; 5: the same on the
    // wide-tile list (one cell per thread); 6: as 5, two cells per thread
    // where the blocks allow it
    const int sc = ctx->sched[1];
    if (sc >= 5) {
      tl = ctx->at<Tile>(G.o_ptiles);
      nt = (int)G.ptiles.size();
    }
    const std::vector<Group::ExtRange> &rs = sc >= 5 ? G.peranges : G.eranges;
    for (const Group::ExtRange &e : rs) {
      StageArgs ar = a;
      ar.kbuf = a.kbuf + (size_t)e.first * NF * TX * TY;
      if (e.shape > 0)
        CK(launch_wide_rhs_f32(G.order, e.ext, e.shape, sc == 6 && e.pair, ar, tl + e.first, e.count,
                               ctx->stream));
      else
        CK(launch_split_rhs_f32(G.order, e.ext, ar, tl + e.first, e.count, ctx->stream));
    }
    // the stage update: fed by bulk copies where the tiles allow it (not for
    // a plain RHS evaluation), else one plain launch over the rest
    const bool tma = ctx->epi_tma && a.mode != MODE_RHS && epilogue_tma_ok(a);
    bool all = tma;
    for (const Group::ExtRange &e : rs) all = all && e.full;
    if (!tma || all) {
      CK(all ? launch_split_epilogue_tma(a, tl, nt, ctx->stream) : launch_split_epilogue(a, tl, nt, ctx->stream));
      return Z4C_OK;
    }
    for (const Group::ExtRange &e : rs) {
      StageArgs ar = a;
      ar.kbuf = a.kbuf + (size_t)e.first * NF * TX * TY;
      CK(e.full ? launch_split_epilogue_tma(ar, tl + e.first, e.count, ctx->stream)
                : launch_split_epilogue(ar, tl + e.first, e.count, ctx->stream));
    }
    return Z4C_OK;
  }
  if (G.f32 && ctx->sched[1] == 3 && !G.stiles.empty()) {
    // staged kernel on the qualifying blocks, the pre-pass schedule on the rest
    CK(launch_staged_f32(G.order, a, ctx->d_stiles(g), (int)G.stiles.size(), ctx->stream));
    tl = ctx->d_rtiles(g);
    nt = (int)G.rtiles.size();
    if (!nt) return Z4C_OK;
  }
  if (!G.f32 && pre) {
    for (const Group::ExtRange &e : G.eranges)
      CK(G.order == 6   ? launch_fused_pre_f64_ext6(e.ext, a, tl + e.first, e.count, ctx->stream)
         : G.order == 4 ? launch_fused_pre_f64_ext4(e.ext, a, tl + e.first, e.count, ctx->stream)
                        : launch_fused_pre_f64_ext2(e.ext, a, tl + e.first, e.count, ctx->stream));
  } else if (!G.f32)
    CK(launch_fused_f64(G.order, a, tl, nt, pre, ctx->stream));
  else if (pre && ctx->occ[1] == 4)
    CK(launch_fused_pre_f32_occ4(G.order, a, tl, nt, ctx->stream));
  else if (pre && ctx->occ[1] == 2)
    CK(launch_fused_pre_f32_occ2(G.order, a, tl, nt, ctx->stream));
  else
    CK(launch_fused_f32(G.order, a, tl, nt, pre, ctx->stream));
  return Z4C_OK;
}

int launch_sommerfeld_p(z4c_ctx *ctx, int p, const StageArgs &a, cudaStream_t st) {
  const int n = (int)ctx->somm[p].size();
  if (!n) return Z4C_OK;
  StageArgs as = a;
  as.kbuf = ctx->d_kbuf_somm();
  CK(launch_sommerfeld(p == 1, as, ctx->d_somm(p), n, st));
  return Z4C_OK;
}

// RHS + stage update of every group, and the Sommerfeld cells.  The
// Sommerfeld kernel reads the stage state (its cells and their neighbours)
// and writes the next state, accumulator and shadow at its own cells only;
// the interior kernels write only interior cells and their own scratch.  So
// with fork set (a captured step) the Sommerfeld cells run on the side
// stream beside the interior RHS and stage-update kernels, from the end of
// the y/z pre-passes (which write only their derivative arrays) to the end
// of the stage; else they follow on the context's stream.
int launch_stage(z4c_ctx *ctx, const StageArgs &base, bool fork = false) {
  const bool any_somm = !ctx->somm[0].empty() || !ctx->somm[1].empty();
  fork = fork && any_somm && ctx->stream != nullptr && ctx->side != nullptr;
  for (int g = 0; g < NGRP; ++g) {
    const int r = launch_prepass_group(ctx, g, group_args(ctx, base, ctx->grp[g].f32));
    if (r) return r;
  }
  if (fork) {
    CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    for (int p = 0; p < 2; ++p) {
      const int r = launch_sommerfeld_p(ctx, p, group_args(ctx, base, p == 1), ctx->side);
      if (r) return r;
    }
    CK(cudaEventRecord(ctx->ev_join, ctx->side));
  }
  for (int g = 0; g < NGRP; ++g) {
    const int r = launch_fused_group(ctx, g, group_args(ctx, base, ctx->grp[g].f32));
    if (r) return r;
  }
  if (fork) {
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    return Z4C_OK;
  }
  for (int p = 0; p < 2; ++p) {
    const int r = launch_sommerfeld_p(ctx, p, group_args(ctx, base, p == 1), ctx->stream);
    if (r) return r;
  }
  return Z4C_OK;
}

// arguments of stage s (0..3) of classic RK4.  Registers: X = (U0, A, B, A)
// are the stage states, next = (A, B, A, U0); FP32 shadows alternate.
StageArgs stage_args(z4c_ctx *ctx, int s) {
  double *U0 = ctx->reg[0], *SA = ctx->reg[1], *SB = ctx->reg[2], *ACC = ctx->reg[3];
  double *X[4] = {U0, SA, SB, SA};
  double *NX[4] = {SA, SB, SA, U0};
  StageArgs a{};
  a.blocks = ctx->d_blocks();
  a.x64 = X[s];
  a.u0 = U0;
  a.acc = ACC;
  a.next = NX[s];
  a.dts = ctx->d_dt();
  a.fa = FA[s];
  a.fb = FB[s];
  a.mode = MODES[s];
  a.status = ctx->d_status();
  a.kbuf = ctx->d_kbuf();
  if (ctx->has[1]) {
    a.x32 = ctx->d_sh(s % 2);
    a.next32 = ctx->d_sh((s + 1) % 2);
    a.next_full = s == 3;
  }
  return a;
}

// One RK4 step; fork: run each stage's Sommerfeld cells on the side stream
// (the captured graph's branch)
int enqueue_step(z4c_ctx *ctx, bool fork = false) {
  for (int s = 0; s < 4; ++s) {
    const StageArgs a = stage_args(ctx, s);
    int r = fill_ghosts(ctx, const_cast<double *>(a.x64), ctx->has[1] ? ctx->d_sh(s % 2) : nullptr);
    if (r) return r;
    r = launch_stage(ctx, a, fork);
    if (r) return r;
  }
  return Z4C_OK;
}

int ensure_shadow(z4c_ctx *ctx) {
  if (!ctx->has[1] || ctx->shadow_valid) return Z4C_OK;
  CK(launch_to_shadow(ctx->reg[0], ctx->d_sh(0), ctx->d_blocks(), (int)ctx->dblocks.size(), ctx->max_S,
                      ctx->stream));
  ctx->shadow_valid = true;
  return Z4C_OK;
}

int upload_dt(z4c_ctx *ctx) {
  if (!ctx->dt_dirty) return Z4C_OK;
  // pageable source: the copy is staged before the call returns
  CK(cudaMemcpyAsync(ctx->d_dt(), ctx->dt_host.data(), sizeof(double) * ctx->dt_host.size(),
                     cudaMemcpyHostToDevice, ctx->stream));
  ctx->dt_dirty = false;
  return Z4C_OK;
}

int set_dt(z4c_ctx *ctx, const double *dt_per_instance) {
  for (size_t i = 0; i < ctx->inst.size(); ++i) {
    const double dt = dt_per_instance[i];
    if (!std::isfinite(dt)) return fail(ctx, Z4C_ERR_BAD_ARG, "non-finite dt for instance %zu", i);
    const Instance &I = ctx->inst[i];
    for (int b = I.first; b < I.first + I.count; ++b)
      if (ctx->dt_host[b] != dt) {
        ctx->dt_host[b] = dt;
        ctx->dt_dirty = true;
      }
  }
  return Z4C_OK;
}

}  // namespace

extern "C" {

int z4c_set_initial_data_instance(z4c_ctx *ctx, int instance, int kind, const double *params, int nparams) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (instance < -1 || instance >= (int)ctx->inst.size()) return fail(ctx, Z4C_ERR_BAD_ARG, "bad instance");
  if (kind < 0 || kind > 4 || nparams < 0 || nparams > 64 || (nparams > 0 && !params))
    return fail(ctx, Z4C_ERR_BAD_ARG, "bad initial-data kind or parameters");
  const int need[5] = {0, 3, 3, 2, 1};
  if (nparams < need[kind]) return fail(ctx, Z4C_ERR_BAD_ARG, "too few initial-data parameters");
  if (kind == 4 && (params[0] < 0 || nparams < 1 + 4 * (int)params[0]))
    return fail(ctx, Z4C_ERR_BAD_ARG, "too few Brill-Lindquist parameters");
  CK(launch_initial_data(ctx->reg[0], ctx->d_blocks(), (int)ctx->dblocks.size(), ctx->max_S, instance, kind,
                         params, nparams, ctx->stream));
  ctx->shadow_valid = false;
  return Z4C_OK;
}

int z4c_set_initial_data(z4c_ctx *ctx, int kind, const double *params, int nparams) {
  return z4c_set_initial_data_instance(ctx, -1, kind, params, nparams);
}

int z4c_fill_ghosts(z4c_ctx *ctx, int reg) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3) return fail(ctx, Z4C_ERR_BAD_ARG, "register index out of range");
  if (reg == 0) ctx->shadow_valid = false;
  return fill_ghosts(ctx, ctx->reg[reg], nullptr);
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
  a.status = ctx->d_status();
  a.kbuf = ctx->d_kbuf();
  if (ctx->has[1]) {
    // shadow of the register in the second shadow buffer (the first may hold U0's)
    CK(launch_to_shadow(ctx->reg[reg], ctx->d_sh(1), ctx->d_blocks(), (int)ctx->dblocks.size(), ctx->max_S,
                        ctx->stream));
    a.x32 = ctx->d_sh(1);
  }
  return launch_stage(ctx, a);
}

int z4c_rk4_step_batch(z4c_ctx *ctx, const double *dt_per_instance, int nsteps) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (nsteps < 0 || !dt_per_instance) return fail(ctx, Z4C_ERR_BAD_ARG, "bad dt or nsteps");
  r = set_dt(ctx, dt_per_instance);
  if (r) return r;
  if (nsteps == 0) return Z4C_OK;
  r = ensure_shadow(ctx);
  if (r) return r;
  r = upload_dt(ctx);
  if (r) return r;
  if (ctx->stream == nullptr) {  // legacy default stream: no capture, plain launches
    for (int s = 0; s < nsteps; ++s) {
      r = enqueue_step(ctx);
      if (r) return r;
    }
    return Z4C_OK;
  }
  if (!ctx->graph) {  // the step reads dt from the device table: one graph serves every dt
    cudaGraph_t g = nullptr;
    r = ensure_side(ctx);  // before the capture begins
    if (r) return r;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    r = enqueue_step(ctx, ctx->fork_somm);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (r) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    CK(e);
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    CK(e);
  }
  for (int s = 0; s < nsteps; ++s) CK(cudaGraphLaunch(ctx->graph, ctx->stream));
  return Z4C_OK;
}

int z4c_rk4_step(z4c_ctx *ctx, double dt, int nsteps) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  std::vector<double> dts(ctx->inst.size(), dt);
  return z4c_rk4_step_batch(ctx, dts.data(), nsteps);
}

int z4c_constraints_instance(z4c_ctx *ctx, int instance, double r_mask, double *norms, void *per_cell_out) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (!norms) return fail(ctx, Z4C_ERR_BAD_ARG, "norms is null");
  if (instance < -1 || instance >= (int)ctx->inst.size()) return fail(ctx, Z4C_ERR_BAD_ARG, "bad instance");
  r = fill_ghosts(ctx, ctx->reg[0], nullptr);
  if (r) return r;
  if (per_cell_out)
    CK(cudaMemsetAsync(per_cell_out, 0, ctx->reg_elems / NF * 4 * sizeof(double), ctx->stream));
  const int nt = (int)ctx->ctiles.size();
  for (int q = 0; q < 3; ++q)  // order-4 records first, then order-6, then order-2 records
    CK(launch_constraint_partials(q == 0 ? 4 : q == 1 ? 6 : 2, ctx->reg[0], ctx->d_blocks(), ctx->d_ctiles(), nt,
                                  instance, r_mask, (double *)per_cell_out, ctx->d_part() + (size_t)q * 8 * nt,
                                  ctx->stream));
  CK(launch_constraint_finalize(ctx->d_part(), 3 * nt, ctx->d_res(), ctx->stream));
  double res[6];
  CK(cudaMemcpyAsync(res, ctx->d_res(), sizeof res, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < 6; ++q) norms[q] = res[q];
  for (int q = 0; q < 6; ++q)
    if (std::isnan(res[q])) return fail(ctx, Z4C_ERR_NAN, "constraint norm %d is NaN", q);
  return Z4C_OK;
}

int z4c_constraints(z4c_ctx *ctx, double r_mask, double *norms, void *per_cell_out) {
  return z4c_constraints_instance(ctx, -1, r_mask, norms, per_cell_out);
}

int z4c_get_state(z4c_ctx *ctx, int reg, void *host, size_t bytes) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3 || !host || bytes != ctx->reg_elems * sizeof(double))
    return fail(ctx, Z4C_ERR_BAD_ARG, "bad register, pointer or size");
  CK(cudaMemcpyAsync(host, ctx->reg[reg], bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return status_check(ctx);
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
  return status_check(ctx);
}

int z4c_sync(z4c_ctx *ctx) {
  int r = ensure_bound(ctx);
  if (r) return r;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  return status_check(ctx);
}

int z4c_test_wait_timeout(z4c_ctx *ctx, int rounds) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (rounds < 1 || rounds > (1 << 16)) return fail(ctx, Z4C_ERR_BAD_ARG, "rounds must be in 1..65536");
  CK(launch_wait_probe(ctx->d_status(), rounds, ctx->stream));
  return z4c_sync(ctx);
}

int z4c_test_prepass_timeout(z4c_ctx *ctx) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (z4c_prepass_tma_blocks(ctx) <= 0)
    return fail(ctx, Z4C_ERR_UNSUPPORTED, "no block runs the TMA-fed pre-pass in this context");
  r = ensure_shadow(ctx);
  if (r) return r;
  // stage 1 reads U0's shadow; the pre-pass writes only its derivative arrays
  const StageArgs base = stage_args(ctx, 0);
  for (int g = 0; g < NGRP; ++g) {
    const Group &G = ctx->grp[g];
    if (G.empty() || !G.f32 || !G.tma_pre) continue;
    StageArgs a = group_args(ctx, base, true);
    a.tmap32 = ctx->d_tmap(0);
    CK(launch_prepass_tma_f32(G.order, a, ctx->at<Tile>(G.o_ztiles), (int)G.ztiles.size(), ctx->stream, 0u));
  }
  return z4c_sync(ctx);
}

int z4c_profile_steps(z4c_ctx *ctx, double dt, int nsteps, double *ms) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (!ms || nsteps <= 0 || !std::isfinite(dt)) return fail(ctx, Z4C_ERR_BAD_ARG, "bad arguments");
  std::vector<double> dts(ctx->inst.size(), dt);
  r = set_dt(ctx, dts.data());
  if (r) return r;
  r = ensure_shadow(ctx);
  if (r) return r;
  r = upload_dt(ctx);
  if (r) return r;
  cudaEvent_t ev[2];
  CK(cudaEventCreate(&ev[0]));
  CK(cudaEventCreate(&ev[1]));
  double acc[4] = {0, 0, 0, 0};
  // kind: 0 ghost fill, 1 fused interior, 2 Sommerfeld, 3 pre-pass
  auto timed = [&](int kind, auto &&launch) -> int {
    CK(cudaEventRecord(ev[0], ctx->stream));
    const int rr = launch();
    if (rr) return rr;
    CK(cudaEventRecord(ev[1], ctx->stream));
    CK(cudaEventSynchronize(ev[1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ev[0], ev[1]));
    acc[kind] += t;
    return Z4C_OK;
  };
  for (int step = 0; step < nsteps; ++step)
    for (int s = 0; s < 4; ++s) {
      const StageArgs a = stage_args(ctx, s);
      r = timed(0, [&] {
        return fill_ghosts(ctx, const_cast<double *>(a.x64), ctx->has[1] ? ctx->d_sh(s % 2) : nullptr);
      });
      if (r) return r;
      r = timed(3, [&] {
        for (int g = 0; g < NGRP; ++g) {
          const int rr = launch_prepass_group(ctx, g, group_args(ctx, a, ctx->grp[g].f32));
          if (rr) return rr;
        }
        return (int)Z4C_OK;
      });
      if (r) return r;
      r = timed(1, [&] {
        for (int g = 0; g < NGRP; ++g) {
          const int rr = launch_fused_group(ctx, g, group_args(ctx, a, ctx->grp[g].f32));
          if (rr) return rr;
        }
        return (int)Z4C_OK;
      });
      if (r) return r;
      r = timed(2, [&] {
        for (int p = 0; p < 2; ++p) {
          const int rr = launch_sommerfeld_p(ctx, p, group_args(ctx, a, p == 1), ctx->stream);
          if (rr) return rr;
        }
        return (int)Z4C_OK;
      });
      if (r) return r;
    }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  for (int q = 0; q < 4; ++q) ms[q] = acc[q] / nsteps;
  return status_check(ctx);
}

int z4c_set_variant(z4c_ctx *ctx, int schedule, int occupancy) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  if (schedule < 1 || schedule > 6) return fail(ctx, Z4C_ERR_BAD_ARG, "schedule must be 1 to 6");
  const bool ok = (schedule >= 3 ? ctx->has[1] : true) &&
                  (schedule >= 4 ? occupancy == 4
                                 : occupancy == 1 || (ctx->has[1] && schedule >= 2 && (occupancy == 2 || occupancy == 4)));
  if (!ok) return fail(ctx, Z4C_ERR_UNSUPPORTED, "no kernel built for this schedule/occupancy");
  ctx->sched[0] = schedule >= 3 ? 2 : schedule;  // schedules 3 to 6 are FP32-only
  ctx->sched[1] = schedule;
  ctx->occ[1] = occupancy;
  ctx->drop_graph();
  return Z4C_OK;
}

int z4c_set_epilogue(z4c_ctx *ctx, int kind) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  if (kind != 0 && kind != 1) return fail(ctx, Z4C_ERR_BAD_ARG, "epilogue kind must be 0 or 1");
  ctx->epi_tma = kind == 1;
  ctx->drop_graph();
  return Z4C_OK;
}

int z4c_set_prepass(z4c_ctx *ctx, int kind) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  if (kind != 0 && kind != 1) return fail(ctx, Z4C_ERR_BAD_ARG, "pre-pass kind must be 0 or 1");
  ctx->pre_tma = kind == 1;
  ctx->drop_graph();
  return Z4C_OK;
}

int z4c_prepass_tma_blocks(const z4c_ctx *ctx) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  if (!ctx->pre_tma) return 0;
  int n = 0;
  for (const Group &G : ctx->grp) {
    if (!G.f32 || !G.tma_pre) continue;
    int last = -1;
    for (const Tile &t : G.ztiles) {
      const int b = t.block & TILE_BLOCK_MASK;
      if (b != last) ++n;  // a block's tiles are contiguous
      last = b;
    }
  }
  return n;
}

int z4c_autotune(z4c_ctx *ctx, int reps, int *schedule_out, int *occupancy_out) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reps < 1) return fail(ctx, Z4C_ERR_BAD_ARG, "reps must be >= 1");
  r = ensure_shadow(ctx);
  if (r) return r;
  r = upload_dt(ctx);
  if (r) return r;
  // stage 1 reads U0 (and its FP32 shadow) and writes ACC and stage A only;
  // timed as the captured step runs it, the Sommerfeld cells on the side
  // stream beside the interior kernels
  StageArgs a = stage_args(ctx, 0);
  r = ensure_side(ctx);
  if (r) return r;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  struct Cand {
    int sched, occ;
    bool tma = true;   // the bulk-copy stage update (split schedules)
    bool pre = true;   // the y/z pre-pass fed by TMA (where blocks qualify)
  };
  bool any_tma_pre = false;
  for (const Group &G : ctx->grp) any_tma_pre = any_tma_pre || (G.f32 && G.tma_pre);
  for (int p = 0; p < 2; ++p) {  // tune each precision with the other fixed
    if (!ctx->has[p]) continue;
    std::vector<Cand> cands = {{1, 1}, {2, 1}};
    if (p == 1) {
      cands.push_back({2, 2});
      cands.push_back({2, 4});
      if (ctx->has_staged()) cands.push_back({3, 4});
      cands.push_back({4, 4, false});
      cands.push_back({4, 4, true});
      if (ctx->has_wide()) {
        cands.push_back({5, 4, false});
        cands.push_back({5, 4, true});
      }
      if (ctx->has_pair()) {
        cands.push_back({6, 4, false});
        cands.push_back({6, 4, true});
      }
      // every candidate with a pre-pass, also with the plane-tiled one
      if (any_tma_pre) {
        const size_t n = cands.size();
        for (size_t q = 0; q < n; ++q)
          if (cands[q].sched >= 2) {
            Cand c = cands[q];
            c.pre = false;
            cands.push_back(c);
          }
      }
    }
    float best = 1e30f;
    Cand pick = {ctx->sched[p], p == 1 ? ctx->occ[1] : 1, ctx->epi_tma, ctx->pre_tma};
    for (const Cand &c : cands) {
      ctx->sched[p] = c.sched;
      if (p == 1) {
        ctx->occ[1] = c.occ;
        ctx->epi_tma = c.tma;
        ctx->pre_tma = c.pre;
      }
      for (int rep = 0; rep <= reps; ++rep) {  // first pass untimed
        if (rep == 1) CK(cudaEventRecord(e0, ctx->stream));
        r = fill_ghosts(ctx, ctx->reg[0], ctx->has[1] ? ctx->d_sh(0) : nullptr);
        if (r) return r;
        r = launch_stage(ctx, a, ctx->fork_somm);
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
    ctx->sched[p] = pick.sched;
    if (p == 1) {
      ctx->occ[1] = pick.occ;
      ctx->epi_tma = pick.tma;
      ctx->pre_tma = pick.pre;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  r = status_check(ctx);
  if (r) return r;
  ctx->drop_graph();  // the next z4c_rk4_step captures the chosen kernels
  const int p = ctx->has[1] ? 1 : 0;
  if (schedule_out) *schedule_out = ctx->sched[p];
  if (occupancy_out) *occupancy_out = p == 1 ? ctx->occ[1] : 1;
  return Z4C_OK;
}

int z4c_block_indicators(z4c_ctx *ctx, int reg, double *chi_min, double *dchi_max) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3 || !chi_min || !dchi_max) return fail(ctx, Z4C_ERR_BAD_ARG, "bad register or output");
  r = fill_ghosts(ctx, ctx->reg[reg], nullptr);
  if (r) return r;
  const int nb = (int)ctx->blocks.size();
  double *out = (double *)(ctx->scratch + ctx->o_diag);
  CK(launch_indicators(ctx->reg[reg], ctx->d_blocks(), ctx->d_ctiles(), (int)ctx->ctiles.size(),
                       ctx->at<int32_t>(ctx->o_cfirst), nb, ctx->d_part(), out, ctx->stream));
  CK(cudaMemcpyAsync(chi_min, out, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(dchi_max, out + nb, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return status_check(ctx);
}

int z4c_psi4(z4c_ctx *ctx, int reg, void *out_device) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3 || !out_device) return fail(ctx, Z4C_ERR_BAD_ARG, "bad register or output");
  r = fill_ghosts(ctx, ctx->reg[reg], nullptr);
  if (r) return r;
  CK(cudaMemsetAsync(out_device, 0, ctx->reg_elems / NF * 2 * sizeof(double), ctx->stream));
  // the y/z first derivatives of every block (FP64 and FP32-RHS alike) from
  // the FP64 register, as the RHS takes them, into the FP64 pre-pass store;
  // a context without one (FP32-RHS blocks only) uses the accumulator
  // register, which has the store's layout and is free between steps (or
  // stage register A when reg is the accumulator)
  void *store = ctx->has[0] ? ctx->d_dstore(false) : ctx->reg[reg == Z4C_REG_ACC ? Z4C_REG_STAGE_A : Z4C_REG_ACC];
  {
    StageArgs a{};
    a.blocks = ctx->d_blocks();
    a.x64 = ctx->reg[reg];
    a.dstore = store;
    for (int g = 0; g < NGRP; ++g) {
      const Group &G = ctx->grp[g];
      if (!G.empty()) CK(launch_prepass_f64(G.order, a, ctx->d_wtiles(g), (int)G.wtiles.size(), ctx->stream));
    }
  }
  const double *ds = (const double *)store;
  CK(launch_psi4(ctx->reg[reg], ctx->d_blocks(), ctx->d_ctiles(), (int)ctx->ctiles.size(), ds,
                 (double *)out_device, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return status_check(ctx);
}

int z4c_track_punctures(z4c_ctx *ctx, int reg, int np, double *xyz, double dt, double *beta_out) {
  int r = ensure_bound(ctx);
  if (r) return r;
  if (reg < 0 || reg > 3 || np < 0 || np > Z4C_MAX_PUNCTURES || (np > 0 && !xyz) || !std::isfinite(dt))
    return fail(ctx, Z4C_ERR_BAD_ARG, "bad register, puncture count, positions or dt");
  if (ctx->inst.size() != 1) return fail(ctx, Z4C_ERR_UNSUPPORTED, "the tracker needs a single-instance context");
  if (np == 0) return Z4C_OK;
  const z4c_mesh &M = ctx->inst[0].mesh;
  std::vector<TrackIn> in(np);
  for (int q = 0; q < np; ++q) {
    TrackIn &p = in[q];
    for (int d = 0; d < 3; ++d) {
      p.x0[d] = p.xw[d] = xyz[3 * q + d];
      if (M.periodic) {
        const double L = M.hi[d] - M.lo[d];
        while (p.xw[d] < M.lo[d]) p.xw[d] += L;
        while (p.xw[d] >= M.hi[d]) p.xw[d] -= L;
      }
    }
    p.block = -1;
    for (size_t b = 0; b < ctx->blocks.size() && p.block < 0; ++b) {  // first block whose closed box holds x
      const z4c_block &B = ctx->blocks[b];
      bool inb = true;
      for (int d = 0; d < 3; ++d) {
        const double t = (p.xw[d] - B.lo[d]) / B.h;
        inb &= t >= -1e-12 && t <= B.n[d] + 1e-12;
      }
      if (inb) p.block = (int32_t)b;
    }
    if (p.block < 0) return fail(ctx, Z4C_ERR_BAD_ARG, "puncture %d lies in no block", q);
  }
  r = fill_ghosts(ctx, ctx->reg[reg], nullptr);
  if (r) return r;
  TrackIn *d_in = (TrackIn *)(ctx->scratch + ctx->o_diag);
  double *d_out = (double *)(d_in + Z4C_MAX_PUNCTURES);
  std::vector<double> out(6 * (size_t)np);
  CK(cudaMemcpyAsync(d_in, in.data(), sizeof(TrackIn) * np, cudaMemcpyHostToDevice, ctx->stream));
  CK(launch_track(ctx->reg[reg], ctx->d_blocks(), d_in, np, dt, d_out, ctx->stream));
  CK(cudaMemcpyAsync(out.data(), d_out, sizeof(double) * 6 * np, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < np; ++q)
    for (int d = 0; d < 3; ++d) {
      xyz[3 * q + d] = out[6 * q + d];
      if (beta_out) beta_out[3 * q + d] = out[6 * q + 3 + d];
    }
  return status_check(ctx);
}

int z4c_peak_fma(int fp64, void *cuda_stream, double *flops_per_s) {
  if (!flops_per_s) return Z4C_ERR_BAD_ARG;
  z4c_ctx *ctx = nullptr;
  CK(peak_fma(fp64 != 0, (cudaStream_t)cuda_stream, flops_per_s));
  return Z4C_OK;
}

int z4c_peak_convert(int mode, void *cuda_stream, double *conv_per_s) {
  if (!conv_per_s || mode < 0 || mode > 3) return Z4C_ERR_BAD_ARG;
  z4c_ctx *ctx = nullptr;
  CK(peak_convert(mode, (cudaStream_t)cuda_stream, conv_per_s));
  return Z4C_OK;
}

int z4c_tile_shape(const z4c_ctx *ctx, int block, int *tx, int *ty, int *cells_per_thread) {
  if (!ctx || !tx || !ty || !cells_per_thread || block < 0 || block >= (int)ctx->dblocks.size())
    return Z4C_ERR_BAD_ARG;
  const bool f32 = ctx->dblocks[block].f32 != 0;
  const int sc = ctx->sched[f32 ? 1 : 0];
  int shape = 0, pair = 0;
  if (f32 && sc >= 5 && block < (int)ctx->wide_shape.size()) {
    shape = ctx->wide_shape[block];
    pair = sc == 6 && shape > 0 ? ctx->wide_pair[block] : 0;
  }
  *tx = TX << shape;
  *ty = TY >> shape;
  *cells_per_thread = pair ? 2 : 1;
  return Z4C_OK;
}

int z4c_launches_per_step(const z4c_ctx *ctx) {
  if (!ctx) return Z4C_ERR_BAD_ARG;
  int per_stage = 0;
  // FP32-RHS Sommerfeld cells take two kernels (RHS, then the stage update)
  for (int p = 0; p < 2; ++p) per_stage += (ctx->gcopy[p].empty() ? 0 : 1) + (ctx->somm[p].empty() ? 0 : p + 1);
  if (ctx->rb_mode)
    per_stage += 2;  // block restriction + scatter
  else
    per_stage += (ctx->rghost.empty() ? 0 : 1) + (ctx->rbuf.empty() ? 0 : 1);
  per_stage += (ctx->cbcopy.empty() ? 0 : 1) + (ctx->prol.empty() ? 0 : 1) + (ctx->pbox.empty() ? 0 : 1);
  for (const Group &G : ctx->grp) {
    if (G.empty()) continue;
    const int sc = ctx->sched[G.f32 ? 1 : 0];
    if (sc == 3 && G.f32 && !G.stiles.empty())
      per_stage += 2 + (G.rtiles.empty() ? 0 : 1);
    else if (sc == 4 && G.f32)
      per_stage += 2 + (int)G.eranges.size();
    else if (sc >= 5 && G.f32)
      per_stage += 2 + (int)G.peranges.size();
    else if (sc >= 2 && !G.f32)
      per_stage += 1 + (int)G.eranges.size();
    else
      per_stage += sc >= 2 ? 2 : 1;
  }
  return 4 * per_stage;
}

const char *z4c_last_error(const z4c_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void z4c_destroy(z4c_ctx *ctx) {
  if (!ctx) return;
  ctx->drop_graph();
  ctx->drop_side();
  delete ctx;
}

}  // extern "C"
