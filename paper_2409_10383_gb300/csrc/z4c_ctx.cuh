// Host-side context of the C ABI: descriptors, work lists and the scratch
// layout.  Shared by z4c_build.cu (creation, binding) and z4c_api.cu (the
// calls that enqueue GPU work).  Not part of the C ABI.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "z4c.h"
#include "z4c_internal.cuh"

namespace z4c {

// One independent problem: a Mesh of equal MeshBlocks on one level.
struct Instance {
  z4c_mesh mesh;
  z4c_params params;
  int ghosts = 0, order = 0;
  int first = 0, count = 0;  // its blocks are [first, first + count)
};

// Kernels are templated on (order, precision): one work list per group.
// Group index = 2 * (order == 6) + f32.
struct Group {
  int order = 4;
  bool f32 = false;
  std::vector<Tile> tiles;   // interior tiles of the group's blocks
  std::vector<Tile> wtiles;  // interior widened by order/2 in x and y (pre-pass)
  // FP32 order 6: the tiles split by whether their block qualifies for the
  // shared-memory staged kernel (schedule 3)
  std::vector<Tile> stiles, rtiles;
  // tiles are sorted by their block's cubic storage extent (0: not cubic);
  // ranges [first, first + count) of one extent, for the kernels
  // specialised on it (FP64 pre-pass schedule, FP32 split schedule)
  struct ExtRange {
    int ext, first, count;
    bool pair;      // the two-cells-per-thread RHS kernel applies (FP32)
    int shape = 0;  // tile shape of the range (schedule-5/6 list)
    // full tiles with 16-byte aligned rows (even ghost width, storage
    // extent and block offset): the bulk-copy stage-update kernel applies
    bool full = false;
  };
  std::vector<ExtRange> eranges;
  // FP32 schedule 5: per extent range, tiles of the widest shape whose width
  // divides n_x (two cells per thread) where the pair kernel applies, the
  // range's 16 x 8 tiles (split RHS kernel) elsewhere
  std::vector<Tile> ptiles;
  std::vector<ExtRange> peranges;
  // FP32 y/z pre-pass fed by TMA (every block of the group qualifies: row
  // length, cells per field and block offset multiples of 4 floats): column
  // tiles walking z; tma_pre is cleared if a tensor map cannot be encoded
  std::vector<Tile> ztiles;
  bool tma_pre = false;
  size_t o_tiles = 0, o_wtiles = 0, o_stiles = 0, o_rtiles = 0, o_ptiles = 0, o_ztiles = 0;
  bool empty() const { return tiles.empty(); }
};

// Work groups: one per (differencing order, precision).  Orders 4 and 6
// keep groups 0..3; 2nd order (2 ghosts) takes 4 and 5.
constexpr int NGRP = 6;
inline int group_of(int order, bool f32) { return 2 * (order == 6 ? 1 : order == 2 ? 2 : 0) + (f32 ? 1 : 0); }

}  // namespace z4c

struct z4c_ctx {
  std::vector<z4c::Instance> inst;
  std::vector<z4c_block> blocks;
  std::vector<z4c::DevBlock> dblocks;
  z4c::Group grp[z4c::NGRP];
  std::vector<z4c::CellRef> somm[2];    // Sommerfeld cells, per precision (0 FP64, 1 FP32)
  std::vector<z4c::GhostCopy> gcopy[2];  // same-level ghost copies, per precision
  std::vector<z4c::Tile> ctiles;         // every interior tile (constraints), in block order
  std::vector<int8_t> wide_shape;        // per block: tile shape on the schedule-5/6 list (0: 16 x 8)
  std::vector<int8_t> wide_pair;         // per block: 1 if schedule 6 runs it two cells per thread
  std::vector<int32_t> cfirst;           // first ctile of each block, and the total
  // mesh refinement transfer (FP64 instances with more than one level)
  std::vector<z4c::RestrictRef> rghost;  // coarse ghost cells <- restriction of a finer block
  std::vector<z4c::RestrictRef> rbuf;    // coarse-buffer slots <- restriction of a same-level block
  std::vector<z4c::CbCopy> cbcopy;       // coarse-buffer slots <- a coarser block's active cell
  std::vector<z4c::ProlongRef> prol;     // fine ghost cells <- prolongation from the buffer
  std::vector<int32_t> pidx;             // buffer slots, [125][prolongation entries] once built
  std::vector<z4c::PBox> pbox;           // ghost regions prolonged as boxes
  std::vector<int32_t> pslots, paxtab;   // their coarse-box slots and per-axis stencil tables
  std::vector<double> wtab;              // restriction weight patterns (5 each)
  double pw[100] = {0};                  // prolongation weights [3-point][shift + 2][child][5]
  int ncb = 0;                           // coarse-buffer slots
  // block-structured restriction (every fine block with restriction targets
  // has at most RB_NMAX cells per axis): the fine blocks, the scatter list,
  // wtab rows of the weight pattern keys -4..3 (5 points: krow[key + 4];
  // 3 points at offset off in the window: krow[8 + 3 (key + 4) + off])
  bool rb_mode = false;
  std::vector<int32_t> rblocks;
  std::vector<z4c::RbCopy> rbcopy;
  int32_t krow[32] = {0};
  std::vector<double> dt_host;           // time step per block
  size_t reg_elems = 0;
  int max_S = 0;
  bool has[2] = {false, false};          // precisions present
  // scratch layout (byte offsets)
  size_t o_blocks = 0, o_somm[2] = {0, 0}, o_gcopy[2] = {0, 0}, o_ctiles = 0, o_part = 0, o_res = 0,
         o_dt = 0, o_sh0 = 0, o_sh1 = 0, o_ds64 = 0, o_ds32 = 0, o_rghost = 0, o_rbuf = 0, o_cbcopy = 0,
         o_prol = 0, o_pidx = 0, o_wtab = 0, o_pw = 0, o_cb = 0, o_status = 0, o_kbuf = 0, o_kbuf_somm = 0, o_tmap = 0, o_rblocks = 0,
         o_rbcopy = 0, o_krow = 0, o_rb = 0, o_pbox = 0, o_pslots = 0,
         o_paxtab = 0, o_cfirst = 0, o_diag = 0, scratch_total = 0;
  // bound buffers
  double *reg[4] = {nullptr, nullptr, nullptr, nullptr};
  char *scratch = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  bool shadow_valid = false;
  bool dt_dirty = true;
  // kernel variant per precision: schedule (1 one kernel, 2 pre-pass + fused,
  // 3 FP32 only: pre-pass + shared-memory staged kernel where the block
  // qualifies, 4 FP32 only: pre-pass + RHS kernel storing k + stage-update
  // kernel) and occupancy (resident CTAs per SM the pre-pass-schedule FP32
  // kernel is built for)
  int sched[2] = {2, 2}, occ[2] = {1, 4};
  bool epi_tma = false;  // FP32 split schedules: the bulk-copy stage update where tiles allow
  bool pre_tma = true;   // FP32 y/z pre-pass: the TMA-fed kernel where the group allows
  // graph of one RK4 step
  cudaGraphExec_t graph = nullptr;
  std::string err;

  const z4c::DevBlock *d_blocks() const { return (const z4c::DevBlock *)(scratch + o_blocks); }
  const z4c::Tile *d_tiles(int g) const { return (const z4c::Tile *)(scratch + grp[g].o_tiles); }
  const z4c::Tile *d_wtiles(int g) const { return (const z4c::Tile *)(scratch + grp[g].o_wtiles); }
  const z4c::Tile *d_stiles(int g) const { return (const z4c::Tile *)(scratch + grp[g].o_stiles); }
  const z4c::Tile *d_rtiles(int g) const { return (const z4c::Tile *)(scratch + grp[g].o_rtiles); }
  int32_t *d_status() const { return (int32_t *)(scratch + o_status); }
  float *d_kbuf() const { return (float *)(scratch + o_kbuf); }
  float *d_kbuf_somm() const { return (float *)(scratch + o_kbuf_somm); }
  // tensor maps (128 bytes each) of FP32 shadow q for every block
  const void *d_tmap(int q) const { return scratch + o_tmap + (size_t)q * 128 * dblocks.size(); }
  bool has_staged() const { return !grp[3].stiles.empty(); }
  bool has_wide() const {
    for (const z4c::Group &G : grp)
      for (const z4c::Group::ExtRange &e : G.peranges)
        if (G.f32 && e.shape > 0) return true;
    return false;
  }
  bool has_pair() const {
    for (const z4c::Group &G : grp)
      for (const z4c::Group::ExtRange &e : G.peranges)
        if (G.f32 && e.shape > 0 && e.pair) return true;
    return false;
  }
  const z4c::CellRef *d_somm(int p) const { return (const z4c::CellRef *)(scratch + o_somm[p]); }
  const z4c::GhostCopy *d_gcopy(int p) const { return (const z4c::GhostCopy *)(scratch + o_gcopy[p]); }
  const z4c::Tile *d_ctiles() const { return (const z4c::Tile *)(scratch + o_ctiles); }
  double *d_part() const { return (double *)(scratch + o_part); }
  double *d_res() const { return (double *)(scratch + o_res); }
  double *d_dt() const { return (double *)(scratch + o_dt); }
  // FP32 arrays in the state layout start 16 bytes past a 256-byte boundary:
  // with 4 ghosts and a row length that is a multiple of 8 floats, every
  // row's interior then starts on a 32-byte sector boundary, so a warp's
  // 16-float row slice spans 2 sectors instead of 3 (the FP64 layout is
  // already aligned: 4 ghosts are 32 bytes)
  static constexpr size_t F32_SHIFT = 16;
  float *d_sh(int q) const { return (float *)(scratch + (q == 0 ? o_sh0 : o_sh1) + F32_SHIFT); }
  void *d_dstore(bool f32) const { return f32 ? scratch + o_ds32 + F32_SHIFT : scratch + o_ds64; }
  bool smr() const { return !prol.empty() || !rghost.empty() || !pbox.empty(); }
  template <class T>
  const T *at(size_t o) const { return (const T *)(scratch + o); }
  double *d_cb() const { return (double *)(scratch + o_cb); }
  void drop_graph() {
    if (graph) {
      cudaGraphExecDestroy(graph);
      graph = nullptr;
    }
  }
  // side stream and fork/join events of the captured step: the Sommerfeld
  // cells of a stage run beside its interior kernels (created on first
  // capture, released with the context)
  bool fork_somm = true;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void drop_side() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
    side = nullptr;
    ev_fork = ev_join = nullptr;
  }
};

namespace z4c {

inline int fail(z4c_ctx *c, int code, const char *fmt, ...) {
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

}  // namespace z4c

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return z4c::fail(ctx, Z4C_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                       __FILE__, __LINE__);                                                  \
  } while (0)
