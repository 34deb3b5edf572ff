// Internal definitions shared by the translation units of the CUDA library.
// Not part of the C ABI (include/z4c.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace z4c {

constexpr int NF = 22;
enum Field {
  CHI = 0, GXX, GXY, GXZ, GYY, GYZ, GZZ, KHAT, AXX, AXY, AXZ, AYY, AYZ, AZZ,
  GAMX, GAMY, GAMZ, THETA, ALPHA, BETAX, BETAY, BETAZ
};

// Symmetric 3x3 index -> component 0..5 (xx xy xz yy yz zz).
__host__ __device__ constexpr int S6(int i, int j) {
  return i == j ? (i == 0 ? 0 : (i == 1 ? 3 : 5))
                : ((i + j) == 1 ? 1 : ((i + j) == 2 ? 2 : 4));
}

// Per-block descriptor, resident in device memory (caller scratch).
struct DevBlock {
  int32_t n[3];   // interior cells
  int32_t e[3];   // storage extents n + 2g
  int32_t g;      // ghost width
  int32_t order;  // 4 or 6
  int32_t S;      // cells per field = e0 e1 e2
  int32_t pad;
  int64_t off;    // element offset of the block's field 0 within a register
  double lo[3];   // lower corner of the active region
  double h;       // spacing
  // finite-difference scale factors (1 / (denominator * h^p)); FP64 and FP32
  double s1, s2, smix, slop, sko;
  float s1f, s2f, smixf, slopf, skof;
  float hf;
  // physics parameters of the block's problem instance (Sec. 2, Sec. 4.3)
  double kappa1, kappa2, eta, chi_floor;
  int32_t lapse, shift;  // 0 harmonic / 1 one-plus-log; 0 frozen / 1 Gamma-driver
  int32_t instance;      // independent problem this block belongs to
  int32_t f32;           // 1: FP32-RHS block (FP32 shadow holds its stage states)
};

// One interior tile: TX x TY cells of one z-plane of one block.
struct Tile {
  int32_t block, i0, j0, k0;  // interior-relative origin
};
// The FP32 schedule-5 tile list mixes tile shapes of 128 cells: shape s is
// (TX << s) x (TY >> s), kept in bits 28..29 of Tile::block (0 elsewhere).
constexpr int TILE_SHAPE_SHIFT = 28;
constexpr int32_t TILE_BLOCK_MASK = (1 << TILE_SHAPE_SHIFT) - 1;

// One Sommerfeld cell (a ghost cell outside the domain) of one block: its
// storage index and (i, j, k) storage coordinates, and per axis d the
// difference it takes in bits 2d..2d+1 (SOMM_CENTRED, or one-sided pointing
// into the block: SOMM_FORWARD for a cell below the interior, SOMM_BACKWARD
// above it).
struct CellRef {
  int32_t block, cidx;
  int16_t i, j, k;
  uint16_t code;
};
enum SommKind { SOMM_CENTRED = 0, SOMM_FORWARD = 1, SOMM_BACKWARD = 2 };

// One same-level ghost copy: dst cell <- src cell, all fields.
struct GhostCopy {
  int32_t dst_block, dst_cidx, src_block, src_cidx;
};

// Mesh refinement transfer (paper Sec. 3.1), FP64 registers only.
// Restriction: the value at a coarse cell covered by fine block `src` is
// sum_{a,b,c} w[pz][c] w[py][b] w[px][a] u[src, s + a + b e0 + c e0 e1] over
// the 5^3 fine cells starting at storage cell s (weights by pattern id).
struct RestrictRef {
  int32_t dst;    // ghost mode: destination block; buffer mode: unused
  int32_t didx;   // ghost mode: destination cell index; buffer mode: coarse-buffer slot
  int32_t src;    // fine block
  int32_t s;      // storage index of the stencil's lowest corner in src
  int32_t wp[3];  // weight pattern per axis (x, y, z)
  int32_t cc;     // the coarse cell in src's coarse lattice: c_x | c_y << 8 | c_z << 16
};
// Block-structured restriction (fine blocks of at most RB_NMAX cells per
// axis): every coarse cell of a listed fine block is restricted into the
// block's slab of rb (RB_NC3 values per field), then scattered: to a coarse
// ghost cell (dst >= 0: block, storage index didx) or a coarse-buffer slot
// (dst < 0: slot didx); ci = coarse cell index (c_z nc_y + c_y) nc_x + c_x.
constexpr int RB_NMAX = 16;
constexpr int RB_NC3 = (RB_NMAX / 2) * (RB_NMAX / 2) * (RB_NMAX / 2);
struct RbCopy {
  int32_t dst, didx, rb, ci;
};
// Coarse-buffer slot <- active cell of a coarser block.
struct CbCopy {
  int32_t slot, src, scidx, pad;
};
// Prolongation of one parent coarse cell into its fine ghost children of
// block dst: child (dx, dy, dz) at cidx0 + dx + dy e0 + dz e0 e1 is written
// if bit dx + 2 dy + 4 dz of mask is set (children beyond the storage, with
// an odd ghost width, are not); coarse values from 125 coarse-buffer slots
// (x fastest): slot q of entry e is idx[q * nentries + e] on the device
// (base = 125 e in the host list before the transpose).  Bits 8 + 3d .. 10 + 3d of mask hold
// the stencil shift along axis d plus 2 (0..4): the 5 coarse cells are
// parent + shift - 2 .. parent + shift + 2, shift != 0 only next to a
// non-periodic outer boundary.
struct ProlongRef {
  int32_t dst, cidx0, base, mask;
};
constexpr int PROLONG_SHIFT_BIT = 8;
// set for 2 ghosts: the weights are the 3-point rows pw[50..99]
constexpr int PROLONG_NP3_BIT = 17;
// Box prolongation: one ghost region (face, edge or corner) of fine block
// dst that lies wholly in one coarser block.  Fine cells: storage origin o,
// extents nf; coarse values from the coarse-buffer slots slots[tab + q] of a
// box of nc cells (x fastest).  Per fine index along axis d (entries ax +
// (0 | nf0 | nf0 + nf1) + i): the stencil's first coarse cell in the box
// (low 16 bits) and the pw row (high 16 bits).  Smem bounds per box below.
struct PBox {
  int32_t dst, tab, ax;
  int16_t o[3];
  uint8_t nf[3], nc[3];
};
constexpr int PB_C = 1024, PB_X = 1536, PB_Y = 1536;

// Which update the stage kernel applies after computing k = RHS(x):
//   MODE_RHS:  rhs_out = k
//   MODE_S1:   acc = u0 + cb k;  next = enforce(u0 + ca k)
//   MODE_S23:  acc = acc + cb k; next = enforce(u0 + ca k)
//   MODE_S4:   next = enforce(acc + cb k)
enum StageMode { MODE_RHS = 0, MODE_S1 = 1, MODE_S23 = 2, MODE_S4 = 3 };

struct StageArgs {
  const DevBlock *blocks;
  const double *x64;  // stage state (FP64): stencil source in FP64 mode, chi source in FP32 mode
  const float *x32;   // FP32 shadow of the stage state (FP32 mode)
  const double *u0;
  double *acc;
  double *next;       // next stage state (FP64)
  float *next32;      // FP32 shadow of the next stage state (FP32 mode)
  double *rhs_out;    // MODE_RHS output
  void *dstore;       // stored y/z first derivatives (pre-pass), FP64 or FP32 like the stencils
  const double *dts;  // time step of each block (its instance's dt)
  double fa, fb;      // next = base + fa dt k, acc = acc + fb dt k (classic RK4 weights)
  int32_t mode;
  int32_t next_full;  // FP32 mode: 1 = write every field of next in FP64, 0 = chi only
  int32_t *status;    // device word; a kernel whose bounded wait gave up ORs in 1
  float *kbuf;        // schedule 4: the FP32 RHS per tile, [tile][field][TX * TY]
  const void *tmap32; // FP32 y/z pre-pass fed by TMA: the tensor maps of x32, one per block (or null)
};

// Fields whose FP32 shadow holds the value minus one (their value at
// infinity and in flat space: chi, the gt diagonal, alpha), so that FP32
// keeps the relative precision of their deviation from 1.
__host__ __device__ constexpr bool shadow_shifted(int f) {
  return f == CHI || f == GXX || f == GYY || f == GZZ || f == ALPHA;
}

// fields with stored y/z first derivatives (their mixed second derivatives
// are taken from them): chi, gt_ij, alpha, beta^i
constexpr int NDS = 11;

// Tiles of the FP32 y/z pre-pass fed by TMA: PRE_TMA_PX x PRE_TMA_PY columns
// (one thread each) walking PRE_TMA_NZ planes; the tile's storage x is a
// multiple of PRE_TMA_PX.
constexpr int PRE_TMA_PX = 16;
constexpr int PRE_TMA_PY = 8;
constexpr int PRE_TMA_NZ = 16;
constexpr int PRE_TMA_NQ = 4;   // fields per CTA: a column takes ceil(11 / NQ) = 3 CTAs (field groups)
constexpr int PRE_TMA_LA = 2;   // planes in flight beyond the 2W + 1 of the stencil

// Interior tile shape of the RHS kernels.
constexpr int TX = 16;
constexpr int TY = 8;

// ---- launchers (defined in the kernel translation units) ----
// refinement transfer: restriction into ghost cells (to_buffer = false) or
// into coarse-buffer slots (true); buffer copies; prolongation from the buffer
cudaError_t launch_restrict(double *reg, const DevBlock *blocks, const RestrictRef *list, int n,
                            const double *wtab, bool to_buffer, double *cb, int ncb, cudaStream_t st);
cudaError_t launch_restrict_blocks(const double *reg, const DevBlock *blocks, const int32_t *rblocks, int nrb,
                                   const double *wtab, const int32_t *krow, double *rb, cudaStream_t st);
cudaError_t launch_rb_scatter(double *reg, const DevBlock *blocks, const RbCopy *list, int n, const double *rb,
                              double *cb, int ncb, cudaStream_t st);
cudaError_t launch_prolong_boxes(double *reg, const DevBlock *blocks, const PBox *boxes, int nbox,
                                 const int32_t *slots, const int32_t *axtab, const double *cb, int ncb,
                                 const double *pw, cudaStream_t st);
// diagnostics (z4c_diag.cu): per-block refinement indicators over a tile
// list in block order (first[b] = first tile of block b), puncture tracker
// One puncture for track_kernel: its block, its position wrapped into a
// periodic domain (for the interpolation) and as given (for the update).
struct TrackIn {
  int32_t block, pad;
  double xw[3], x0[3];
};
cudaError_t launch_indicators(const double *u, const DevBlock *blocks, const Tile *tiles, int ntiles,
                              const int32_t *first, int nb, double *part, double *out, cudaStream_t st);
// ds: the FP64 y/z pre-pass arrays of u (required)
cudaError_t launch_psi4(const double *u, const DevBlock *blocks, const Tile *tiles, int ntiles, const double *ds,
                        double *out, cudaStream_t st);
cudaError_t launch_track(const double *u, const DevBlock *blocks, const TrackIn *in, int np, double dt, double *out,
                         cudaStream_t st);
cudaError_t launch_cb_copy(const double *reg, const DevBlock *blocks, const CbCopy *list, int n, double *cb,
                           int ncb, cudaStream_t st);
cudaError_t launch_prolong(double *reg, const DevBlock *blocks, const ProlongRef *list, int n,
                           const int32_t *idx, const double *cb, int ncb, const double *pw, cudaStream_t st);
// FP32 fused kernel with shared-memory staging (schedule 3), for blocks whose
// rows allow 16-byte aligned bulk copies; the tiles of other blocks use the
// pre-pass schedule
cudaError_t launch_staged_f32(int order, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);
// failure-detection probe: a bounded mbarrier wait that runs out (status |= 1)
cudaError_t launch_wait_probe(int32_t *status, int rounds, cudaStream_t st);
// FP32 split schedule (4): the pre-pass-schedule RHS kernel stores k (FP32)
// per tile in a.kbuf, then an epilogue kernel applies the RK stage update and
// the FP64 enforcement at high occupancy
// RHS kernel of one extent range (ext = cubic storage extent the kernel is
// specialised for, 0 = runtime strides; a.kbuf already offset to the range's
// first tile), and the stage-update kernel over the whole tile list
cudaError_t launch_split_rhs_f32(int order, int ext, const StageArgs &a, const Tile *tiles, int ntiles,
                                 cudaStream_t st);
cudaError_t launch_split_epilogue(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);
// the same, persistent, fed by bulk copies into shared memory (full tiles,
// even ghost width and storage extent, 16-byte aligned registers)
cudaError_t launch_split_epilogue_tma(const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);
bool epilogue_tma_ok(const StageArgs &a);
// schedules 5 and 6: the split RHS kernel on wide tiles (shape 1: 32 x 4,
// 2: 64 x 2) for the extents built, one cell per thread or (pair) two cells
// per thread on packed f32x2 arithmetic
bool wide_ext_built(int order, int ext);
cudaError_t launch_wide_rhs_f32(int order, int ext, int shape, bool pair, const StageArgs &a, const Tile *tiles,
                                int ntiles, cudaStream_t st);
// cubic storage extents with a specialised split RHS kernel (per order)
bool split_ext_built(int order, int ext);
// FP64 fused pre-pass-schedule kernel for one extent range (ext as above;
// extents without a specialised kernel use runtime strides)
cudaError_t launch_fused_pre_f64_ext6(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);
cudaError_t launch_fused_pre_f64_ext4(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);
// 2nd order with 2 ghosts (z4c_interior_order2_f64.cu, z4c_interior_order2_f32.cu)
cudaError_t launch_fused_pre_f64_ext2(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);
cudaError_t launch_prepass_f64_order2(const StageArgs &a, const Tile *wtiles, int nwtiles, cudaStream_t st);
cudaError_t launch_fused_f64_order2(const StageArgs &a, const Tile *tiles, int ntiles, bool pre, cudaStream_t st);
cudaError_t launch_prepass_f32_order2(const StageArgs &a, const Tile *wtiles, int nwtiles, cudaStream_t st);
cudaError_t launch_fused_f32_order2(int occ, const StageArgs &a, const Tile *tiles, int ntiles, bool pre,
                                    cudaStream_t st);
bool split_ext_built2(int ext);
cudaError_t launch_split_rhs2(int ext, const StageArgs &a, const Tile *tiles, int ntiles, cudaStream_t st);
// FP32 fused pre-pass-schedule kernel built for 2 or 4 resident CTAs per SM
cudaError_t launch_fused_pre_f32_occ2(int order, const StageArgs &a, const Tile *tiles, int ntiles,
                                      cudaStream_t st);
cudaError_t launch_fused_pre_f32_occ4(int order, const StageArgs &a, const Tile *tiles, int ntiles,
                                      cudaStream_t st);
// y/z first-derivative pre-pass; fused RHS + stage kernel (pre: reads the
// pre-pass output, else the single-kernel schedule)
cudaError_t launch_prepass_f64(int order, const StageArgs &a, const Tile *wtiles, int nwtiles, cudaStream_t st);
cudaError_t launch_prepass_f32(int order, const StageArgs &a, const Tile *wtiles, int nwtiles, cudaStream_t st);
// the same derivatives from the z-walking kernel fed by TMA tensor copies
// (a.tmap32 set; orders with prepass_tma_built): bit-identical results
bool prepass_tma_built(int order);
// (rounds: try_wait attempts per bounded wait; 0 makes every CTA give up at
// its first wait, drain its copies and report, as a failure-path test)
cudaError_t launch_prepass_tma_f32(int order, const StageArgs &a, const Tile *ztiles, int n, cudaStream_t st,
                                   uint32_t rounds = 1u << 22);
cudaError_t launch_fused_f64(int order, const StageArgs &a, const Tile *tiles, int ntiles, bool pre,
                             cudaStream_t st);
cudaError_t launch_fused_f32(int order, const StageArgs &a, const Tile *tiles, int ntiles, bool pre,
                             cudaStream_t st);
// FP64 cells: one kernel (RHS + stage update).  FP32-RHS cells: the FP32
// RHS into k records at a.kbuf (somm_kbuf_floats(ncells) floats), then the
// FP64 stage update.
cudaError_t launch_sommerfeld(bool f32, const StageArgs &a, const CellRef *cells, int ncells,
                              cudaStream_t st);
size_t somm_kbuf_floats(int ncells);
cudaError_t launch_ghosts_f64(double *reg, const DevBlock *blocks, const GhostCopy *list, int n,
                              cudaStream_t st);
cudaError_t launch_ghosts_f32(float *reg, const DevBlock *blocks, const GhostCopy *list, int n,
                              cudaStream_t st);
// instance < 0: every block; otherwise only the blocks of that instance
cudaError_t launch_initial_data(double *u0, const DevBlock *blocks, int nblocks, int max_S, int instance,
                                int kind, const double *par, int npar, cudaStream_t st);
// FP32-RHS blocks only
cudaError_t launch_to_shadow(const double *src, float *dst, const DevBlock *blocks, int nblocks,
                             int max_S, cudaStream_t st);
// per-CTA partial records of the tiles' blocks of this order (and instance,
// if >= 0); records of other blocks are zero
cudaError_t launch_constraint_partials(int order, const double *u0, const DevBlock *blocks,
                                       const Tile *tiles, int ntiles, int instance, double r_mask,
                                       double *per_cell, double *partials, cudaStream_t st);
cudaError_t launch_constraint_finalize(const double *partials, int n, double *result, cudaStream_t st);

cudaError_t peak_fma(bool f64, cudaStream_t st, double *flops_per_s);
cudaError_t peak_convert(int mode, cudaStream_t st, double *conv_per_s);

}  // namespace z4c
