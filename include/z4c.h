/*
 * z4c.h -- C ABI of the GB300 (sm_103a) Z4c right-hand-side + RK4 library.
 *
 * The library evolves the vacuum Z4c system (paper Sec. 2: Z4c with
 * Bona-Masso lapse and Gamma-driver shift) on a pack of MeshBlocks
 * (Sec. 3: a Mesh of rectangular MeshBlocks, each an active region plus a
 * ghost region; blocks batched into one pack to cut kernel launches) with
 * cell-centred 2nd/4th/6th-order finite differences (Sec. 3.2; 2nd order with
 * 2 ghosts is the paper's default with 2 ghost cells, Sec. 3.1), Kreiss-Oliger
 * dissipation and constraint damping (Sec. 4.3), and classic RK4 whose
 * ghost zones are refilled at every stage (Sec. 3).  Throughput is counted
 * in zone-cycles per second (Sec. 5).
 *
 * Conventions shared by every call
 *   - 22 evolved fields in this order:
 *       0 chi, 1..6 gt_xx gt_xy gt_xz gt_yy gt_yz gt_zz, 7 Khat,
 *       8..13 At_xx At_xy At_xz At_yy At_yz At_zz, 14..16 Gam^x Gam^y Gam^z,
 *       17 Theta, 18 alpha, 19..21 beta^x beta^y beta^z.
 *   - A "register" is one full copy of the state in FP64: for each block in
 *     creation order and each field, an (n_z+2g) x (n_y+2g) x (n_x+2g)
 *     array with i fastest; blocks are concatenated.  z4c_state_bytes()
 *     gives its size.
 *   - Every device buffer (registers, scratch, outputs) is allocated and
 *     owned by the caller; the library never allocates device memory.  The
 *     library owns only host-side descriptors and CUDA graphs.
 *   - All GPU work is enqueued on the stream given to z4c_bind().  Calls
 *     return after enqueueing unless stated otherwise.
 *   - Every call returns a z4c_status (0 = success, negative = error);
 *     nothing throws across the ABI.  z4c_last_error() describes the last
 *     failure of a context.
 */
#ifndef Z4C_GB300_H
#define Z4C_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define Z4C_NFIELDS 22

typedef enum z4c_status {
  Z4C_OK = 0,
  Z4C_ERR_BAD_ARG = -1,      /* null pointer, out-of-range index, bad size */
  Z4C_ERR_BAD_MESH = -2,     /* blocks overlap, leave the mesh, or leave gaps */
  Z4C_ERR_UNSUPPORTED = -3,  /* order not 2/4/6, ghosts < order/2 + 1, odd storage extent */
  Z4C_ERR_CUDA = -4,         /* a CUDA runtime call failed */
  Z4C_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
  Z4C_ERR_NAN = -6,          /* a constraint norm came out NaN */
  Z4C_ERR_NOT_BOUND = -7     /* z4c_bind() has not been called */
} z4c_status;

/* Mesh (Sec. 3): the physical domain [lo, hi].  periodic = 1 wraps every
 * direction; periodic = 0 uses the Sommerfeld outer boundary (outer_bc = 1):
 * each ghost cell whose centre lies outside the domain evolves
 * d_t u = -(x^k d_k u + u - u_inf)/r with 2nd-order one-sided differences. */
typedef struct z4c_mesh {
  double lo[3];
  double hi[3];
  int32_t periodic;
  int32_t outer_bc;
} z4c_mesh;

/* One MeshBlock (Sec. 3): n interior cells per direction, lower corner lo of
 * the active region, cubic cell spacing h.  instance: the independent
 * problem the block belongs to (z4c_create_batch; 0 for z4c_create).  level:
 * refinement level, h = h0 / 2^level with one h0 per instance (static mesh
 * refinement, Sec. 3.1).  The blocks of an instance are the leaves of an
 * oct-tree: equal n, aligned to their level's block lattice, tiling the mesh;
 * with more than one level, n is even and >= 8, neighbours (faces, edges,
 * corners) differ by at most one level, every prolongation stencil finds its
 * coarse values one level coarser or on its own level (else
 * Z4C_ERR_BAD_MESH), and the instance is FP64 (rhs_precision 64). */
typedef struct z4c_block {
  int32_t level;
  int32_t n[3];
  double lo[3];
  double h;
  int32_t instance;
  int32_t reserved;
} z4c_block;

/* Physical and numerical parameters (Sec. 2, Sec. 4.3).
 *   ko_sigma      Kreiss-Oliger strength sigma (0.5 or 0.02 in the paper)
 *   kappa1/2      Z4c constraint damping (kappa1 = 0.02, kappa2 = 0)
 *   eta           Gamma-driver damping
 *   chi_floor     floor applied to chi wherever 1/chi appears
 *   cfl           Courant factor, informational (callers pass dt)
 *   lapse         0 harmonic (d_t alpha = -alpha^2 Khat), 1 1+log (-2 alpha Khat)
 *   shift         0 frozen (d_t beta = 0), 1 Gamma-driver (Gam - eta beta)
 *   rhs_precision 64: everything FP64; 32: stencils and RHS algebra in FP32,
 *                 state, RK accumulation, 1/chi, constraint enforcement and
 *                 constraint norms in FP64
 *   schedule      0 default (below), 1 one fused kernel per stage, 2 a pre-pass
 *                 storing the y/z first derivatives of chi, gt, alpha, beta
 *                 (in scratch) followed by the fused kernel, which then forms
 *                 mixed second derivatives as one stencil on the stored
 *                 values (fewer operations, fewer registers); default 2;
 *                 3 (FP32-RHS only) as 2, but the fused kernel stages each
 *                 field's stencil rows in shared memory with bulk
 *                 asynchronous copies (TMA) for blocks that allow 16-byte
 *                 aligned rows (order 6, 4 ghosts, n_x % 16 == 0,
 *                 n_y % 8 == 0), schedule 2 for the others; 4 (FP32-RHS
 *                 only) as 2, but the RHS kernel stores k in FP32 and a
 *                 second kernel applies the RK stage update and the FP64
 *                 enforcement at high occupancy; 5 (FP32-RHS only) as 4,
 *                 but on tiles 64 (or 32) cells wide and 2 (or 4) rows
 *                 high, so that a warp reads along one row, for cubic
 *                 blocks with a compiled kernel (order 6, n = 32, 64, 96,
 *                 128), 16 x 8 tiles for the others; 6 (FP32-RHS only) as
 *                 5, and the RHS kernel computes two neighbouring cells of
 *                 a row per thread with packed two-lane FP32 arithmetic
 *                 where the ghost width and n_x are even.  FP64 instances
 *                 given 3 to 6 use 2.  Default (0): 2 for FP64, 4 for
 *                 FP32-RHS */
typedef struct z4c_params {
  double ko_sigma;
  double kappa1;
  double kappa2;
  double eta;
  double chi_floor;
  double cfl;
  int32_t lapse;
  int32_t shift;
  int32_t rhs_precision;
  int32_t schedule;
} z4c_params;

typedef struct z4c_ctx z4c_ctx;

/* Register indices for z4c_fill_ghosts / z4c_rhs / z4c_get_state. */
#define Z4C_REG_U0 0     /* evolved state */
#define Z4C_REG_STAGE_A 1
#define Z4C_REG_STAGE_B 2
#define Z4C_REG_ACC 3

/* Initial-data kinds for z4c_set_initial_data. */
#define Z4C_ID_FLAT 0
#define Z4C_ID_GAUGE_WAVE 1        /* params {A, d, t}: H = 1 - A sin(2 pi (x - t)/d) */
#define Z4C_ID_LINEAR_WAVE 2       /* params {A, d, t}: gamma_yy,zz = 1 +- A sin(2 pi (x - t)/d) */
#define Z4C_ID_SCHWARZSCHILD 3     /* params {M, lapse_kind}: isotropic; 0 alpha = psi^-2, 1 static */
#define Z4C_ID_BRILL_LINDQUIST 4   /* params {np, m_1, x_1, y_1, z_1, ...}, alpha = psi^-2 */

/* Create a context for one pack of blocks on one mesh (Sec. 3).
 * blocks: nblocks entries (host memory, copied).  ghosts >= fd_order/2 + 1,
 * fd_order 2, 4 or 6, every storage extent n+2*ghosts even.  Blocks must tile
 * the mesh exactly with equal n along shared faces.  Makes no CUDA call.
 * On success *out owns the context (release with z4c_destroy). */
int z4c_create(const z4c_mesh *mesh, const z4c_block *blocks, int nblocks, int ghosts,
               int fd_order, const z4c_params *params, z4c_ctx **out);

/* One independent problem of a batch: its Mesh, parameters, ghost width and
 * differencing order (the arguments of z4c_create). */
typedef struct z4c_instance {
  z4c_mesh mesh;
  z4c_params params;
  int32_t ghosts;
  int32_t fd_order;
} z4c_instance;

/* A pack of independent problems evolved together (the paper's
 * MeshBlockPack, Sec. 3, across problems): instances may differ in mesh,
 * block size, order, precision and parameters.  blocks: the blocks of every
 * instance, grouped by instance in increasing order (block.instance), each
 * instance's blocks tiling its mesh as in z4c_create.  One RK4 step of the
 * whole batch is one CUDA graph (z4c_rk4_step_batch), each instance with its
 * own dt.  Registers hold the blocks in the order given.  Makes no CUDA call. */
int z4c_create_batch(const z4c_instance *instances, int ninstances, const z4c_block *blocks, int nblocks,
                     z4c_ctx **out);

/* Bytes of one FP64 register (see conventions). */
int z4c_state_bytes(const z4c_ctx *ctx, size_t *bytes_per_register);

/* Bytes of device scratch the context needs: descriptor tables, work lists,
 * FP32 shadow copies (rhs_precision 32) and reduction partials. */
int z4c_scratch_bytes(const z4c_ctx *ctx, size_t *bytes);

/* Attach caller-owned device buffers and the CUDA stream (cudaStream_t
 * passed as void*; a non-default stream enables CUDA-graph replay in
 * z4c_rk4_step).  u0, stage_a, stage_b, acc: z4c_state_bytes() each, 256-byte
 * aligned.  scratch: z4c_scratch_bytes(), 256-byte aligned.  Uploads the
 * descriptor tables into scratch, with the TMA tensor maps of the FP32
 * shadows that the y/z pre-pass of qualifying blocks reads through (encoded
 * here, as they hold the buffers' addresses), and waits for the copies. */
int z4c_bind(z4c_ctx *ctx, void *u0, void *stage_a, void *stage_b, void *acc, void *scratch,
             void *cuda_stream);

/* Analytic initial data of the given kind into every storage cell of U0. */
int z4c_set_initial_data(z4c_ctx *ctx, int kind, const double *params, int nparams);

/* The same for the blocks of one instance only (instance = -1: all). */
int z4c_set_initial_data_instance(z4c_ctx *ctx, int instance, int kind, const double *params, int nparams);

/* Fill the ghost cells of register reg from neighbouring blocks' active
 * cells (same level) or by periodic wrap (Sec. 3); at refinement boundaries
 * (Sec. 3.1) a ghost cell facing a finer block gets the restriction of its
 * active data (5-point Lagrange per axis inside the fine active region) and
 * a ghost cell facing a coarser block the 5^3-point Lagrange prolongation
 * of coarse values (coarser active cells, or restrictions of same-level
 * data).  Sommerfeld cells are evolved, never overwritten. */
int z4c_fill_ghosts(z4c_ctx *ctx, int reg);

/* Raw right-hand side of register reg (ghosts must be filled) into rhs_out
 * (device, z4c_state_bytes(), FP64, same layout).  Interior and Sommerfeld
 * cells are written, other ghost cells set to 0. */
int z4c_rhs(z4c_ctx *ctx, int reg, void *rhs_out);

/* nsteps classic RK4 steps of size dt on U0 (Sec. 3, Sec. 4.3): per stage,
 * ghost fill, then one fused kernel computing the RHS and the stage update
 * with det gt = 1 / tr At = 0 enforcement.  On a non-default stream the
 * step is captured once into a CUDA graph and replayed. */
int z4c_rk4_step(z4c_ctx *ctx, double dt, int nsteps);

/* nsteps RK4 steps of every instance of a batch, instance i with time step
 * dt_per_instance[i] (host array of ninstances doubles).  The steps read dt
 * from a device table, so one captured graph serves every choice of dt. */
int z4c_rk4_step_batch(z4c_ctx *ctx, const double *dt_per_instance, int nsteps);

/* Hamiltonian and momentum constraints of U0 (ghosts are filled first).
 * norms (host, 6 doubles): ||H||_2, ||M||_2, max|H|, ||H||_2 and ||M||_2
 * over cells with r > r_mask, max|M|; ||X||_2 = sqrt(sum X^2 h^3 / sum h^3)
 * over interior cells.  per_cell_out (device, nullable): 4 values per
 * storage cell (H, M^x, M^y, M^z) laid out like a 4-field register.
 * Synchronises the stream.  Returns Z4C_ERR_NAN if a norm is NaN. */
int z4c_constraints(z4c_ctx *ctx, double r_mask, double *norms, void *per_cell_out);

/* The constraint norms over the blocks of one instance (instance = -1: all);
 * per_cell_out as in z4c_constraints (cells of other instances are 0). */
int z4c_constraints_instance(z4c_ctx *ctx, int instance, double r_mask, double *norms, void *per_cell_out);

/* Copy register reg to / from host memory (bytes = z4c_state_bytes()).
 * Synchronous.  Pinned host memory makes the copy faster.  The evolved
 * state is the interior and Sommerfeld cells; ghost cells hold the values of
 * the last fill of that register (call z4c_fill_ghosts first for current
 * ones; for FP32-RHS blocks the RK4 step fills only the FP32 copy's ghosts). */
int z4c_get_state(z4c_ctx *ctx, int reg, void *host, size_t bytes);
int z4c_set_state(z4c_ctx *ctx, int reg, const void *host, size_t bytes);

/* End-to-end call on host buffers: copy host_in into U0, run nsteps RK4
 * steps, copy U0 into host_out; synchronous. */
int z4c_evolve_host(z4c_ctx *ctx, const void *host_in, void *host_out, size_t bytes, double dt,
                    int nsteps);

/* Wait for the stream; reports any CUDA error, and Z4C_ERR_TIMEOUT if a
 * kernel's bounded wait on its own bulk copies gave up since the last
 * report (that launch's results are then invalid).  z4c_get_state,
 * z4c_evolve_host, z4c_profile_steps and z4c_autotune report it too. */
int z4c_sync(z4c_ctx *ctx);

/* Failure-detection test aid (no counterpart in the paper): enqueue on the
 * context's stream one kernel whose bounded mbarrier wait must run out (it
 * waits for 16 bytes of bulk copies and issues none), after at most
 * `rounds` try_wait attempts (1..65536), then z4c_sync().  Returns
 * Z4C_ERR_TIMEOUT with its z4c_last_error text, exactly as after a staged
 * kernel whose copies never landed; the context stays usable and the status
 * word is cleared.  Touches no register. */
int z4c_test_wait_timeout(z4c_ctx *ctx, int rounds);

/* Failure-detection test aid for the TMA-fed y/z pre-pass (z4c_set_prepass):
 * run it once on U0's FP32 shadow with a wait limit of zero try_wait
 * attempts, so that every CTA gives up at its first wait on copies it has
 * issued, waits a bounded time for those copies to land, sets the status
 * word and returns; then z4c_sync().  Returns Z4C_ERR_TIMEOUT with its
 * z4c_last_error text, the status word cleared and the context usable; it
 * writes only the pre-pass derivative arrays, which every stage recomputes.
 * Z4C_ERR_UNSUPPORTED when no block runs that kernel. */
int z4c_test_prepass_timeout(z4c_ctx *ctx);

/* Measurement aid: run nsteps RK4 steps with plain (not graph) launches,
 * each bracketed by CUDA events on the context's stream, and return the
 * average milliseconds per step spent in each kernel kind (4 doubles):
 * ms[0] ghost fill, ms[1] fused interior RHS + stage update, ms[2]
 * Sommerfeld cells, ms[3] y/z first-derivative pre-pass (schedule 2).
 * Advances U0 exactly like z4c_rk4_step.  Synchronous. */
int z4c_profile_steps(z4c_ctx *ctx, double dt, int nsteps, double *ms);

/* Select a kernel variant explicitly: schedule 1 to 6 (see z4c_params;
 * 3 to 6 apply to FP32-RHS blocks, FP64 blocks then use 2) and occupancy,
 * the resident CTAs per SM the pre-pass-schedule fused kernel's registers
 * are budgeted for: 1 always; 2 or 4 for the FP32-RHS kernel (with schedule
 * 3: for the blocks that do not qualify for staging); schedules 4 to 6 are
 * built for 4 only.  Other combinations return Z4C_ERR_UNSUPPORTED.  Makes
 * no CUDA call. */
int z4c_set_variant(z4c_ctx *ctx, int schedule, int occupancy);

/* FP32-RHS split schedules (4 to 6): which kernel applies the RK stage
 * update and the enforcement.  kind 0 (the default): the plain kernel, one
 * thread per cell at high occupancy; kind 1: a persistent kernel fed by
 * bulk asynchronous copies (TMA) of each tile's k record and FP64 rows into
 * shared memory, for the tiles that allow it (full tiles, even ghost width
 * and storage extent, 16-byte aligned registers), the plain kernel for the
 * others.  The same arithmetic either way (bit-identical results).
 * Z4C_ERR_BAD_ARG for another kind.  Makes no CUDA call. */
int z4c_set_epilogue(z4c_ctx *ctx, int kind);

/* FP32-RHS blocks: which kernel computes the y/z first derivatives of the
 * eleven fields with mixed second derivatives (the pre-pass of schedules 2
 * to 6; paper Sec. 2, the second derivatives of the Z4c RHS).  kind 1 (the
 * default): a kernel whose CTAs each walk a column of 16 planes, fed by TMA
 * tensor copies of every plane's rows (with the y halo) into a shared-memory
 * ring, for order-4 and order-6 groups whose blocks have rows, fields and
 * block offsets that are multiples of 4 floats; the plane-tiled kernel for
 * the others.  kind 0: the plane-tiled kernel everywhere.  Identical results
 * either way (bit for bit).  Z4C_ERR_BAD_ARG for another kind.  Makes no
 * CUDA call. */
int z4c_set_prepass(z4c_ctx *ctx, int kind);

/* How many blocks have their y/z pre-pass computed by the TMA-fed kernel
 * under the current z4c_set_prepass kind (0 with kind 0, for FP64 blocks, or
 * where the blocks do not qualify; a group whose tensor maps could not be
 * encoded at z4c_bind drops out).  Z4C_ERR_BAD_ARG for a null context.
 * Makes no CUDA call. */
int z4c_prepass_tma_blocks(const z4c_ctx *ctx);

/* Pick the fastest kernel variant for this context on this GPU: the
 * schedule (1 or 2; for FP32-RHS blocks also 4, and 3, 5 and 6 where
 * blocks qualify; see z4c_params)
 * and, for the FP32-RHS fused kernel, the number of resident CTAs per SM its
 * registers are budgeted for (1, 2, 4), for the split schedules the
 * stage-update kernel (z4c_set_epilogue), and the y/z pre-pass kind
 * (z4c_set_prepass) where blocks qualify for the TMA-fed one.
 * Each candidate runs reps + 1 times the ghost fill and stage 1 of RK4 (which
 * reads U0 and overwrites only the accumulator and stage A, so U0 keeps its
 * value), with the Sommerfeld cells on a second stream beside the interior
 * kernels as in the captured step; the fastest is kept, FP64 and FP32-RHS
 * kernels tuned separately.
 * Reported (either pointer may be NULL): the FP32-RHS choice if the context
 * has FP32-RHS blocks, else the FP64 one.
 * Synchronous.  Call before z4c_rk4_step, or it re-captures its graph. */
int z4c_autotune(z4c_ctx *ctx, int reps, int *schedule_out, int *occupancy_out);

/* Refinement indicators of every block (paper Sec. 3.2, the chi-min and
 * d-chi criteria): over the block's interior cells, chi_min[b] = min chi and
 * dchi_max[b] = max |grad chi|, the gradient by the block's centred
 * first-derivative stencil (order 2, 4 or 6), in FP64.  Fills the ghost cells
 * of register reg first.  chi_min, dchi_max: host arrays of nblocks
 * doubles, in block order.  Synchronous. */
int z4c_block_indicators(z4c_ctx *ctx, int reg, double *chi_min, double *dchi_max);

/* Puncture tracker (paper Sec. 3.3): one step x <- x - dt beta(x) for each
 * of np <= Z4C_MAX_PUNCTURES punctures (forward Euler; call once per RK4
 * step with that step's dt).  beta is interpolated from register reg by
 * 4-point Lagrange interpolation per axis over the cell centres around x,
 * in the first block (in block order) whose closed box [lo, lo + n h]
 * contains x (after wrapping into a periodic domain).  Fills the ghost
 * cells of reg first.  xyz: host, 3 doubles per puncture, updated in place;
 * beta_out (host, nullable): 3 doubles per puncture, beta at the old
 * position.  Single-instance contexts only (Z4C_ERR_UNSUPPORTED
 * otherwise); Z4C_ERR_BAD_ARG if a puncture lies in no block.
 * Synchronous. */
#define Z4C_MAX_PUNCTURES 64
int z4c_track_punctures(z4c_ctx *ctx, int reg, int np, double *xyz, double dt, double *beta_out);

/* Weyl scalar Psi4 on the grid (paper Sec. 3.3: the outgoing Weyl scalar in
 * a coordinate tetrad; no interpolation onto spheres), in FP64, at every
 * interior cell of every block:
 *   Psi4 = (E_ij - i B_ij) mb^i mb^j,
 *   E_ij = R_ij + K K_ij - K_ik gamma^kl K_lj,
 *   B_ij = symmetric part of gamma_im eps^mkl D_k K_lj,
 * from gamma_ij = gt_ij / chi, K_ij = (At_ij + gt_ij K / 3) / chi,
 * K = Khat + 2 Theta, with the block's centred stencils; the tetrad
 * mb = (e_theta - i e_phi) / sqrt(2) comes from Gram-Schmidt in gamma_ij on
 * the coordinate vectors x^i, (-y, x, 0) and (x z, y z, -(x^2 + y^2)) about
 * the origin.  Cells on the z axis (tetrad undefined) and all non-interior
 * cells get 0.  Fills the ghost cells of register reg first.  A context
 * with FP32-RHS blocks only keeps its y/z derivative store for this call in
 * the accumulator register (stage register A when reg is the accumulator),
 * whose content is undefined between steps anyway.
 * out_device: device, caller-owned, 2 * (register elements / 22) doubles:
 * for each block in order, the real part over its storage cells
 * ((n_z+2g) x (n_y+2g) x (n_x+2g), x fastest), then the imaginary part.
 * Synchronous. */
int z4c_psi4(z4c_ctx *ctx, int reg, void *out_device);

/* Measurement aid: FP64 (fp64 = 1) or FP32 (fp64 = 0) fused multiply-add
 * throughput of the current device in FLOP/s, from independent FMA chains
 * with no memory traffic (the ALU roofline of the RHS kernels).  Enqueued on
 * cuda_stream and synchronised.  Allocates nothing. */
int z4c_peak_fma(int fp64, void *cuda_stream, double *flops_per_s);

/* Measurement aid: float <-> double conversions per second of the current
 * device (the FP32-RHS path's conversion cost).  mode 0: float -> double by
 * the hardware conversion; 1: the same by the integer-pipe bit manipulation
 * the FP32-RHS kernels use; 2: double -> float by the hardware (round to
 * nearest even); 3: the same on the integer pipe.  Independent chains with
 * no memory traffic; enqueued on cuda_stream and synchronised.  Allocates
 * nothing.  Z4C_ERR_BAD_ARG for another mode. */
int z4c_peak_convert(int mode, void *cuda_stream, double *conv_per_s);

/* Constraint norms of one MeshBlock without any device allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory themselves, for example a diagnostic hook
 * inside a host code that owns the whole device memory pool, or a monitor
 * that must not allocate while an evolution is in flight.  It computes the
 * same six norms as z4c_constraints() for a single block, using no context
 * and no caller scratch: its reduction records live in a fixed, file-scope
 * device array of Z4C_STATIC_MAX_TILES records of 8 doubles (about 1 MiB),
 * which every GPU that loads this library holds until the process exits.
 *
 *   u_device   the block's state in device memory, one register of a
 *              single block: 22 fields of (n_z+2g) x (n_y+2g) x (n_x+2g)
 *              FP64, i fastest, ghost cells already filled
 *   n, ghosts, fd_order, lo, h, chi_floor, r_mask  as in z4c_create /
 *              z4c_constraints
 *   norms      host, 6 doubles (same order as z4c_constraints)
 *   cuda_stream  stream to run on (void * cudaStream_t); the call waits for it
 *
 * One record is used per 16 x 8 tile of one z-plane; a block needing more
 * than Z4C_STATIC_MAX_TILES tiles (e.g. larger than 128^3) is rejected with
 * Z4C_ERR_UNSUPPORTED.  Calls no cudaMalloc/cudaFree and no allocating
 * library routine.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device, which must be the device
 * that holds u_device, and synchronises cuda_stream before it returns.
 * Every call shares the array and overwrites the records it reads; calls
 * that overlap on the GPU (other streams or threads without ordering) race
 * on it.  Returns Z4C_ERR_NAN if a norm is NaN. */
#define Z4C_STATIC_MAX_TILES 16384
int z4c_constraints_static(const void *u_device, const int32_t n[3], int ghosts, int fd_order,
                           const double lo[3], double h, double chi_floor, double r_mask,
                           double *norms, void *cuda_stream);

/* The interior tile of block `block` under the context's current kernel
 * variant (after z4c_autotune: the one it kept): tx x ty cells of one
 * z-plane per CTA, and the cells each thread computes (2 for the FP32-RHS
 * schedule 6 on qualifying blocks, else 1).  Z4C_ERR_BAD_ARG for a bad
 * block index or a NULL output.  Makes no CUDA call. */
int z4c_tile_shape(const z4c_ctx *ctx, int block, int *tx, int *ty, int *cells_per_thread);

/* Number of kernel launches one RK4 step enqueues. */
int z4c_launches_per_step(const z4c_ctx *ctx);

/* Text of the last error of ctx (never NULL; "" when none). */
const char *z4c_last_error(const z4c_ctx *ctx);

/* Release the context (not the caller's buffers). */
void z4c_destroy(z4c_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* Z4C_GB300_H */
