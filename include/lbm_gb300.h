/*
 * lbm_gb300.h -- C-ABI of the GB300-native refined-grid D3Q19 lattice Boltzmann library.
 *
 * The method is the volume-based grid refinement of Schornbaum & Ruede,
 * "Massively parallel algorithms for the lattice Boltzmann method on non-uniform
 * grids" (arXiv:1508.07982): D3Q19 SRT/TRT collision (Sec. 2), a 2:1-balanced
 * forest of octrees of equal-sized blocks (Sec. 3.2-3.3), and the recursive level
 * schedule of Alg. 1 / Alg. 2 (Sec. 4.1) with homogeneous explosion (Eq. ctof) and
 * averaging coalescence (Eq. ftoc).  Every step of a time step runs in the library's
 * own sm_103a CUDA kernels; there is no CPU fallback.
 *
 * Conventions used by every call:
 *  - Coordinates are in level-0 cell units.  Cell (i, j, k) of level L has its centre
 *    at ((i + 0.5) / 2^L, (j + 0.5) / 2^L, (k + 0.5) / 2^L).
 *  - PDF directions follow this fixed D3Q19 order (an interface convention, like a file
 *    format):  0 (0,0,0); 1 (+1,0,0) 2 (-1,0,0) 3 (0,+1,0) 4 (0,-1,0) 5 (0,0,+1)
 *    6 (0,0,-1); 7 (+1,+1,0) 8 (-1,-1,0) 9 (+1,-1,0) 10 (-1,+1,0) 11 (+1,0,+1)
 *    12 (-1,0,-1) 13 (+1,0,-1) 14 (-1,0,+1) 15 (0,+1,+1) 16 (0,-1,-1) 17 (0,+1,-1)
 *    18 (0,-1,+1).  Weights 1/3, 1/18 (faces), 1/36 (edges).
 *  - Per-level cell arrays are "block-major": the level's leaf blocks in the order of
 *    lbm_get_block_table, each block's B^3 cells in x-fastest, then y, then z order.
 *  - Every call returns an lbm_status; no exception crosses the ABI.  On failure,
 *    lbm_last_error() returns a thread-local description.
 *  - Device memory is owned by the forest (batch, net) handle and released by lbm_destroy
 *    (lbm_batch_destroy, lbm_net_destroy); it comes from the lbm_allocator given at creation,
 *    or from cudaMalloc without one.  Caller buffers are owned by the caller.  `on_device` = 1 means a pointer is a CUDA
 *    device pointer on the forest's device; 0 means host memory (pinned or pageable).
 *  - `stream` is a cudaStream_t (0 = the legacy default stream).  Calls that launch work
 *    are asynchronous on that stream unless stated otherwise; calls that return host
 *    data synchronise the stream.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,       /* invalid argument or description */
    LBM_EUNBALANCED = 2,  /* a forest check found a 2:1 balance violation (internal error) */
    LBM_ENOMEM = 3,       /* device or host allocation failed */
    LBM_ECUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    LBM_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
    LBM_ENONFINITE = 6    /* a reduction met a NaN or Inf */
} lbm_status;

/* Device-memory hook.  A forest, batch or net created with one takes every device buffer it
 * holds from `alloc` and gives it back through `release`; created with NULL (or alloc = NULL) it
 * uses cudaMalloc and cudaFree.  The hook lets a host framework own the memory, for example a
 * caching allocator that already holds the GPU's memory.
 *   alloc(bytes, stream, user)    returns a device pointer to `bytes` bytes on the current device,
 *                                 aligned to 256 bytes, or NULL on failure (the call that needed
 *                                 it then returns LBM_ENOMEM).  `stream` is the object's stream
 *                                 (cudaStream_t), on which the library orders all use of the
 *                                 memory; after each allocation the library synchronises it, so
 *                                 memory still in use by work queued there is never written.
 *   release(ptr, bytes, stream, user)  takes back a pointer that alloc returned, with its size.
 *                                 The library first synchronises `stream`, so nothing still
 *                                 reads or writes the memory.
 *   user                          passed through unchanged.
 * Both are called on the thread that makes the creating, reconfiguring or destroying call, never
 * from a stream callback.  The library copies the struct; the functions and `user` must stay
 * valid until the object is destroyed.  Pinned host buffers (a few bytes per object) and the
 * fixed array of lbm_mass_momentum_noalloc do not go through the hook. */
typedef struct lbm_allocator {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*release)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} lbm_allocator;

typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_NOSLIP = 1, LBM_BC_VELOCITY = 2, LBM_BC_FREESLIP = 3 } lbm_bc;
typedef enum { LBM_SRT = 0, LBM_TRT = 1 } lbm_collision;

/* PDF storage.  FP64 stores f_a; FP32S and FP16S store the shifted value f_a - w_a rho0 and
 * collide in FP32; coalescence means and the mass/momentum totals accumulate in FP64. */
typedef enum { LBM_FP64 = 0, LBM_FP32S = 1, LBM_FP16S = 2 } lbm_precision;

#define LBM_MAX_LEVELS 8
#define LBM_MAX_SPHERES 64
#define LBM_MAX_REGIONS 64

/* Domain and refinement description (Sec. 3.3: a uniform root grid whose blocks are split
 * into 8 while marked by the application; the library adds the splits 2:1 balance needs).
 *   root_blocks   number of root blocks per axis (>= 1)
 *   block_cells   B, cells per block edge on every level: 8, 16 or 32
 *   max_level     deepest level a split may create (0 .. LBM_MAX_LEVELS-1)
 *   bc[6]         faces x-, x+, y-, y+, z-, z+; periodic faces come in pairs.  Free-slip
 *                 (named only, Sec. 4.1) is read as specular reflection: the value entering a
 *                 cell across the face is the one its tangential neighbour sent towards the
 *                 face, with the normal component of the direction reversed; beyond several
 *                 faces, the first non-free-slip face in the order z+, z-, y+, y-, x+, x-
 *                 applies, or, if all are free-slip, the reflection in each (an obstacle at
 *                 the mirrored cell bounces the value back instead).  Level interfaces may meet
 *                 free-slip faces: the reflection also serves the streamed ghost layers 1-2, whose
 *                 mirrored neighbours hold exploded or streamed values like any other source
 *                 (Sec. 4.1 extends the boundary treatment to the innermost ghost layers).
 *   bc_velocity   wall velocity of LBM_BC_VELOCITY faces (Sec. 5.2: velocity bounce-back)
 *   rho0          reference density of the incompressible equilibrium (Eq. fequ)
 *   spheres       no-slip obstacles (cx, cy, cz, r): a cell whose centre lies inside
 *   regions       refinement regions: {kind, target level, p0..p5} with kind 0 = box
 *                 (lo xyz, hi xyz) and kind 1 = ball (centre xyz, radius); a block of level
 *                 L < target that overlaps the region (with positive volume, or closer than
 *                 the radius) is split.
 *   u_shift       FP32S / FP16S storage: the stored value of direction a is f_a - f_a^eq(rho0,
 *                 u_shift) (the precision extension's shift by w_a rho0, generalised to a
 *                 reference velocity; zero gives f_a - w_a rho0).  Set it to the prevailing flow
 *                 velocity (a channel's inlet plug): the stored deviations, and so the storage
 *                 rounding, shrink with |u - u_shift|.  |u_shift| < 0.3; ignored for FP64. */
typedef struct {
    int32_t root_blocks[3];
    int32_t block_cells;
    int32_t max_level;
    int32_t precision;    /* lbm_precision */
    int32_t collision;    /* lbm_collision */
    int32_t bc[6];        /* lbm_bc */
    double bc_velocity[6][3];
    double rho0;
    int32_t n_spheres;
    double spheres[LBM_MAX_SPHERES][4];
    int32_t n_regions;
    double regions[LBM_MAX_REGIONS][8];
    double u_shift[3];
} lbm_forest_desc;

/* Application callbacks (Sec. 3.3).  refine: return nonzero to split block (bx, by, bz) of
 * `level` (block coordinates of that level).  flag: return nonzero if the cell centred at
 * (x, y, z) of `level` is a no-slip obstacle.  Both may be NULL and are only called during
 * lbm_create_forest / lbm_plan_create, on the calling thread. */
typedef int (*lbm_refine_fn)(int level, int bx, int by, int bz, void* user);
typedef int (*lbm_flag_fn)(int level, double x, double y, double z, void* user);

typedef struct lbm_forest lbm_forest;
typedef struct lbm_plan lbm_plan;

/* Thread-local text of the last failure on this thread ("" if none).  Never NULL. */
const char* lbm_last_error(void);

/* The D3Q19 tables in the order above: e[19][3], w[19], opposite index opp[19].  Host only. */
lbm_status lbm_lattice(int32_t* e, double* w, int32_t* opp);

/* ---- host-only forest planning (no CUDA call) -------------------------------------------
 * Builds the leaf set (refinement by regions and callback, then 2:1 balance across faces,
 * edges and corners, Sec. 3.2-3.3), the per-level block tables and the cell classes, without
 * touching a GPU.  lbm_plan_leaves writes the level's leaf blocks as (bx, by, bz) triples in
 * block-table order (pass NULL to query the count into *n).  lbm_plan_counts writes
 * {leaf blocks, owned fluid cells, ghost-layer-1/2 fluid cells, ghost blocks}.
 * lbm_plan_ghost_work writes the ghost stream work of the level's two sub-steps,
 * {cells 1, values 1, cells 2, values 2}: the ghost-layer cells and (cell, direction) values
 * that the stream computes because a later pull reads them (owned pulls of sub-step 2 read
 * layer 1; the coalescence of Eq. ftoc reads the coalescing directions of the children), the
 * rest of ghost layers 1-2 being never read (Sec. 4.3-4.4). */
lbm_status lbm_plan_create(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag,
                           void* user, lbm_plan** out);
lbm_status lbm_plan_num_levels(const lbm_plan* p, int32_t* n_levels);
lbm_status lbm_plan_leaves(const lbm_plan* p, int32_t level, int32_t* n, int32_t* blocks);
lbm_status lbm_plan_counts(const lbm_plan* p, int32_t level, int64_t counts[4]);
lbm_status lbm_plan_ghost_work(const lbm_plan* p, int32_t level, int64_t work[4]);
lbm_status lbm_plan_destroy(lbm_plan* p);

/* ---- forest lifetime --------------------------------------------------------------------
 * lbm_create_forest plans the forest (as lbm_plan_create), allocates both PDF grids of every
 * level on the current CUDA device (two-grid storage, Sec. 4.1), uploads the block tables and
 * binds `stream`.  `alloc` (NULL: cudaMalloc) supplies that memory and every later buffer of the
 * forest (residual history, autotuning snapshots, work counters).  The state starts undefined;
 * call lbm_set_level_params and lbm_init_equilibrium before stepping.  lbm_destroy frees
 * everything (NULL is a no-op). */
lbm_status lbm_create_forest(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag,
                             void* user, void* stream, const lbm_allocator* alloc, lbm_forest** out);
lbm_status lbm_destroy(lbm_forest* f);
lbm_status lbm_num_levels(const lbm_forest* f, int32_t* n_levels);

/* Leaf blocks of `level` as (bx, by, bz) triples: the block-major order of every per-level
 * array: the traversal of the forest of octrees, root blocks in x-fastest order and, within each
 * root, the Morton (z-order) curve (Sec. 3.3, 4.5); level 0 is the root grid, x fastest.  Pass
 * blocks = NULL to query the count into *n. */
lbm_status lbm_get_block_table(const lbm_forest* f, int32_t level, int32_t* n, int32_t* blocks);

/* Cell updates of one coarse step: sum over levels of owned fluid cells x 2^L (every level
 * L takes 2^L steps per coarse step, Sec. 2.3). */
lbm_status lbm_cell_updates_per_coarse_step(const lbm_forest* f, int64_t* n);

/* ---- parameters (Sec. 2.3) ----------------------------------------------------------------
 * From the level-0 rate: lambda_e,L (or omega_L) by Eq. (omega_scaling_0), lambda_o,L by
 * Eq. (lambda_oL) at fixed magic parameter Lambda_eo (ignored for SRT, where lambda_o =
 * lambda_e), body acceleration a_L = a_0 / 2^L by Eq. (force_scaling).  accel0 may be NULL.
 * The explicit variant takes per-level arrays lambda_e[n_levels], lambda_o[n_levels],
 * accel[n_levels][3].  Both copy the values to the device on the forest's stream. */
lbm_status lbm_set_level_params(lbm_forest* f, double lambda_e0, double magic_lambda,
                                const double accel0[3]);
lbm_status lbm_set_level_params_explicit(lbm_forest* f, const double* lambda_e,
                                         const double* lambda_o, const double* accel);

/* ---- state --------------------------------------------------------------------------------
 * Equilibrium start (Eq. fequ) on one level: f = f^eq(rho, u) on owned fluid cells, taken
 * as the post-streaming state of Fig. 5 (1).  rho[n_cells] and u[3][n_cells] are block-major
 * FP64 arrays (n_cells = leaf blocks x B^3; values of obstacle cells are ignored); either may
 * be NULL for rho0 / rest.  level = -1 applies rho = rho0, u = u_const to every level, with
 * u_const given in `u` as 3 doubles (NULL = rest). */
lbm_status lbm_init_equilibrium(lbm_forest* f, int32_t level, const double* rho, const double* u,
                                int32_t on_device);

/* Advances n_steps coarse time steps: Alg. 1 with same-level exchange, boundary treatment and
 * coalescence fused into each level's stream-collide kernel (Alg. 2), and one explosion kernel
 * per visit of a finer level (Eq. ctof; it writes the ghost values that owned cells pull in the
 * first sub-step, the stream reads the others from the coarse parents).  The whole coarse step
 * is one CUDA graph, replayed per step on the forest's stream; asynchronous. */
lbm_status lbm_step_coarse(lbm_forest* f, int32_t n_steps);

/* Macroscopic fields (Eq. fvelocity; the velocity adds a_L/2 as in Sec. 2.1) of the current
 * state of one level, block-major FP64: rho[n_cells], u[3][n_cells]; NaN on obstacle cells.
 * level = -1 returns every level in one array, level 0 first, each level block-major:
 * rho[N], u[3][N] with N the sum of the levels' n_cells (lbm_get_block_table gives each level's
 * blocks in the same order).  Either output may be NULL.  Synchronises the stream when
 * on_device = 0. */
lbm_status lbm_get_macroscopic(lbm_forest* f, int32_t level, double* rho, double* u,
                               int32_t on_device);

/* PDFs of one level's owned cells, pdfs[19][n_cells] FP64 (unshifted f_a), block-major.  The
 * stored state is the post-collision state of the next step (the kernels store f-tilde).
 * lbm_set_pdfs writes the same layout back (checkpoint / resume, bit-exact for FP64 and FP16S;
 * with FP32S and u_shift != 0 the FP64 f = v + f^eq(rho0, u_shift) of a stored value v below
 * about 2e-9 can round, so a resumed run may differ in the last FP32 bits). */
lbm_status lbm_get_pdfs(lbm_forest* f, int32_t level, double* pdfs, int32_t on_device);
lbm_status lbm_set_pdfs(lbm_forest* f, int32_t level, const double* pdfs, int32_t on_device);

/* Volume-weighted totals over owned fluid cells of all levels: out[0] = sum 8^-L rho, out[1..3] =
 * sum 8^-L j with j = sum_a e_a f_a of the post-streaming state (the moments the last collision
 * of each cell started from).  After lbm_step_coarse the step kernels have recorded them: each
 * level's last sub-step of the coarse step sums its cells' moments per warp in the compute type,
 * and this call adds the warp sums in FP64 (no PDF is read).  After lbm_init_equilibrium,
 * lbm_set_pdfs, a batched step or an autotune they are summed from the stored PDFs instead, with
 * j = sum_a e_a f~_a - rho0 a (the collision adds rho0 a): FP32 per-cell sums of the shifted values
 * with FP32/FP16 storage, FP64 with FP64 storage.  The two agree up to the rounding of the stored
 * values.  out is host memory; synchronises the stream.  Returns LBM_ENONFINITE if a total is not
 * finite. */
lbm_status lbm_reduce_mass_momentum(lbm_forest* f, double out[4]);

/* ---- measurement -------------------------------------------------------------------------
 * lbm_timing_begin(f, max_steps) makes the next lbm_step_coarse calls (at most max_steps
 * coarse steps in total) enqueue the step's kernels directly, one after another on the forest's
 * stream, with a CUDA event recorded before and after every kernel (the launches the captured
 * graph holds; the side launches that the graph runs on a branch beside the column walk run here
 * in series, so that every kernel is timed alone).  lbm_timing_end synchronises and returns, per
 * level, the summed time in ms and the number of launches of the column-walk (stream-collide)
 * kernels, of the explosion kernels and of the side kernels (coupled cells and ghost work of the
 * FP32/FP16 layouts) (arrays of length n_levels; any may be NULL), then stops timing. */
lbm_status lbm_timing_begin(lbm_forest* f, int32_t max_steps);
lbm_status lbm_timing_end(lbm_forest* f, double* ms_per_level, int64_t* launches_per_level,
                          double* ms_explode_per_level, int64_t* launches_explode_per_level,
                          double* ms_side_per_level, int64_t* launches_side_per_level);

/* Thread mapping of the stream-collide kernel (results do not depend on it).  ctas_per_sm (1 to 4)
 * selects the kernel variant compiled for that many resident 256-thread CTAs per SM (its shared
 * memory may allow fewer; fewer CTAs stage more planes ahead).  LBM_FP64: each thread walks
 * 2^cells_per_thread_log2 cells (<= B) of one z-column of a block.  LBM_FP32S / LBM_FP16S: the
 * column walk is persistent (one grid of resident CTAs that take chunks of planes from a counter)
 * and each thread updates two x-adjacent cells, so cells_per_thread_log2 is only checked.  The
 * default is (log2 B - 3, 3) for LBM_FP64 and (log2 B - 3, 2) otherwise.  Synchronises the stream
 * and drops the captured graphs; the next lbm_step_coarse captures them again. */
lbm_status lbm_set_kernel_config(lbm_forest* f, int32_t cells_per_thread_log2, int32_t ctas_per_sm);
lbm_status lbm_get_kernel_config(const lbm_forest* f, int32_t* cells_per_thread_log2, int32_t* ctas_per_sm);

/* Number of kernel launches one coarse step issues (the nodes of the captured graph). */
lbm_status lbm_launches_per_coarse_step(const lbm_forest* f, int32_t* n);

/* Picks the fastest thread mapping for this forest: times n_steps coarse steps (Alg. 1) for every
 * (cells_per_thread_log2 <= log2 B, ctas_per_sm in 1..4) pair, applies the fastest as
 * lbm_set_kernel_config would, and writes it and its ms per coarse step (outputs may be NULL).
 * The state of the forest (every level's two PDF grids and parities) is copied on the device first
 * and restored afterwards, so the call leaves the simulation where it was; the copy needs as much
 * device memory again as the PDF grids.  The results of later steps do not depend on the mapping.
 * Synchronises the stream.  LBM_EINVAL if the forest is not initialised or is being timed. */
lbm_status lbm_autotune(lbm_forest* f, int32_t n_steps, int32_t* cells_per_thread_log2, int32_t* ctas_per_sm,
                        double* ms_per_step);

/* Picks the block size for a description: for every B in {8, 16, 32} that divides the domain
 * (root_blocks x block_cells level-0 cells per axis, kept fixed: root_blocks becomes N / B) it
 * creates the forest with block size B (through `alloc`, on `stream`), sets the level parameters as
 * lbm_set_level_params(lambda_e0, magic_lambda, accel0) does, starts it from rest, tunes its thread
 * mapping as lbm_autotune(n_steps) does, and destroys it; it writes the B with the fewest ms per
 * coarse step to *block_cells and each candidate's ms to ms_per_step[0..2] (B = 8, 16, 32; -1 where
 * B does not divide the domain or the forest cannot be built).  The regions and obstacles are the
 * same for every B, but refinement splits whole blocks, so a larger B covers the requested regions
 * with more cells: the time per coarse step of the same problem, not GLUPS, decides.  Refinement
 * by callback is not supported (the callback takes block coordinates, which depend on B): refine
 * must be NULL.  LBM_EINVAL for invalid arguments or when no candidate can be built.  The paper
 * fixes its block size per run (Sec. 3.2); this is a tuning aid. */
lbm_status lbm_autotune_block_size(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag, void* user,
                                   double lambda_e0, double magic_lambda, const double accel0[3], void* stream,
                                   const lbm_allocator* alloc, int32_t n_steps, int32_t* block_cells,
                                   double ms_per_step[3]);

/* ---- batches of forests --------------------------------------------------------------------
 * Many independent forests (for example a parameter study of small cases) stepped together:
 * one coarse step of every member is Alg. 1 over the deepest member, and each phase of it (the
 * stream-collide sub-step F_L(s) or the explosion E_L of one level, Sec. 4) is a single
 * persistent launch over the work of all members, so that a phase of small forests fills the
 * GPU with one launch instead of one per member.  Members without level L have no work in the
 * phases of level L.  Each member computes exactly what lbm_step_coarse computes for it.
 *
 * lbm_batch_create(forests, n, alloc, out): the members must share precision, collision model,
 * block size and stream; the batch's own launch tables come from `alloc` (NULL: cudaMalloc); they stay owned by the caller, stay usable through every lbm_* call, and must
 * outlive the batch.  The batch reads each member's buffers through pointers taken when it builds
 * its graphs, so it must be destroyed and re-created after a member is re-created.
 * lbm_batch_step(b, n): n coarse steps of every member on the members' stream (graph replay,
 * asynchronous); every member must be initialised, with parameters set, and at the same two-grid
 * parity (members stepped only together are).  lbm_batch_set_kernel_config / lbm_batch_autotune
 * set or tune the thread mapping of the batch's launches as the single-forest calls do (autotune
 * restores every member's state).  lbm_batch_cell_updates_per_coarse_step sums the members' cell
 * updates; lbm_batch_launches_per_coarse_step counts the launches of one coarse step. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(lbm_forest* const* forests, int32_t n, const lbm_allocator* alloc,
                            lbm_batch** out);
lbm_status lbm_batch_step(lbm_batch* b, int32_t n_steps);
lbm_status lbm_batch_set_kernel_config(lbm_batch* b, int32_t cells_per_thread_log2, int32_t ctas_per_sm);
lbm_status lbm_batch_autotune(lbm_batch* b, int32_t n_steps, int32_t* cells_per_thread_log2, int32_t* ctas_per_sm,
                              double* ms_per_step);
lbm_status lbm_batch_cell_updates_per_coarse_step(const lbm_batch* b, int64_t* n);
lbm_status lbm_batch_launches_per_coarse_step(const lbm_batch* b, int32_t* n);
lbm_status lbm_batch_destroy(lbm_batch* b);

/* Steady-state residual: r = ||u(t) - u(t')||_2 / ||u(t)||_2 over the owned fluid cells of all
 * levels, each cell weighted by its volume 8^-L, where u is the velocity of lbm_get_macroscopic,
 * t the state now and t' the state at the previous call (call it every 10 coarse steps; the flow
 * counts as steady when r < 1e-6).  The paper defines no residual; this is the reading used for
 * the warm-start comparison.  The first call on a forest only records u and returns r = HUGE_VAL.
 * Keeps one velocity copy per level on the device.  Synchronises the stream; LBM_ENONFINITE if a
 * fluid cell's velocity is not finite (a diverged run). */
lbm_status lbm_velocity_residual(lbm_forest* f, double* r);

/* FP64 arithmetic peak of the current device, measured: a kernel of independent FP64 fused
 * multiply-add chains on every SM, timed with CUDA events on `stream` over `reps` launches after
 * a warm-up.  *gfma = FP64 FMA instructions (thread level) per second / 1e9 (a GFLOP/s figure is
 * twice that).  This is the roofline denominator of the FP64 column walk, whose update is bound by
 * the FP64 pipe on this GPU (the paper has no counterpart: it is a measurement of the hardware).
 * Synchronises the stream. */
lbm_status lbm_probe_fp64_fma(int32_t reps, double* gfma, void* stream);

/* ---- learned warm start: a 3-D convolutional net -------------------------------------------
 * The paper has no learned component; this net serves the warm start of the refined levels.  It
 * maps the coarse-only solution, upsampled onto a refined block plus a halo, to the refined
 * solution there; lbm_init_equilibrium then starts the refined levels from f^eq of its output
 * (Eq. fequ), and the LBM itself runs unmodified.
 *
 * Net: `layers` 3x3x3 convolutions, zero padding, width 16, ReLU between layers and none after
 * the last.  Layer 0 reads the first `in_channels` channels, the last layer writes the first
 * `out_channels`.  Activations are device tensors of `nvol` volumes of D x H x W voxels, x fastest,
 * channels last with 16 BF16 channels per voxel (unused channels zero): [nvol][D][H][W][16].  The
 * products run on the tensor cores with BF16 operands and FP32 accumulation; each layer's output
 * is rounded to BF16.  Parameters are FP32, per layer W[27][16 out][16 in] (tap o = (dz+1)*9 +
 * (dy+1)*3 + (dx+1)) then b[16]; lbm_net_num_params counts them, get/set copy them to/from host
 * memory.  Weights start He-uniform from a SplitMix64 stream seeded by `seed`.
 *
 * lbm_net_forward writes the last layer's BF16 output z.  lbm_net_predict writes the FP32
 * prediction pred[N][out_channels] = skip + z (skip FP32 [N][out_channels], may be NULL).
 * lbm_net_gradient (after a forward or predict call on the same input) computes the mean squared
 * error of that prediction against target[N][out_channels] over the voxels weight[N] marks (NULL:
 * all; the mean divides by sum(weight) x out_channels) and the gradients of every parameter
 * (lbm_net_get_grads); lbm_net_train_step does forward, gradient and one Adam step (beta 0.9 /
 * 0.999, eps 1e-8) with learning rate lr.  All pointers except the host parameter buffers are
 * device pointers; calls run on `stream` and synchronise it where they return a loss.  The
 * parameters, optimiser moments and the activations of the largest volume set seen so far come
 * from `alloc` (NULL: cudaMalloc); a call on more voxels than before grows the activations. */
typedef struct lbm_net lbm_net;

/* Data movement of the warm start (device pointers, asynchronous on `stream`).
 * lbm_warmstart_features: inputs of the net for the blocks[nblocks][3] (block coordinates) of a
 * refined level `level` of block size B: one volume of (B + 2 halo)^3 voxels per block.  Each
 * voxel takes the coarse-only solution sampled trilinearly at its cell centre.  The coarse-only
 * solution is coarse_rho[n0] and coarse_u[3][n0], a level-0-only forest of coarse_blocks[3] blocks
 * of the same B, in that forest's block-major order.  Axes in periodic_mask (bit a) wrap, walled
 * axes clamp; coarse obstacle cells are skipped.  Channels:
 *   0      (rho - 1) rho_scale
 *   1..3   u u_scale
 *   4      1 inside an obstacle sphere (spheres[nspheres][4] = cx, cy, cz, r in level-0 units) or
 *          outside the domain
 *   5      level / 2
 * x is BF16 [nblocks][D][D][D][16]; skip (FP32 [..][4], may be NULL) receives channels 0..3.
 * lbm_warmstart_targets: a refined level's solution (block-major rho[n], u[3][n], n = nblocks B^3,
 * as lbm_get_macroscopic returns it) scaled the same way into target FP32 [..][4] on each volume's
 * interior, with weight 1 on fluid interior voxels and 0 elsewhere.
 * lbm_warmstart_fields: the inverse map of a prediction FP32 [..][4] to block-major rho[n],
 * u[3][n] of the interior voxels, ready for lbm_init_equilibrium(on_device = 1). */
lbm_status lbm_warmstart_features(const double* coarse_rho, const double* coarse_u, const int32_t coarse_blocks[3],
                                  int32_t B, int32_t periodic_mask, int32_t level, int32_t halo, const int32_t* blocks,
                                  int32_t nblocks, const double* spheres, int32_t nspheres, double rho_scale,
                                  double u_scale, void* x, float* skip, void* stream);
lbm_status lbm_warmstart_targets(const double* rho, const double* u, int32_t B, int32_t halo, int32_t nblocks,
                                 double rho_scale, double u_scale, float* target, float* weight, void* stream);
lbm_status lbm_warmstart_fields(const float* pred, int32_t B, int32_t halo, int32_t nblocks, double rho_scale,
                                double u_scale, double* rho, double* u, void* stream);
lbm_status lbm_net_create(int32_t layers, int32_t in_channels, int32_t out_channels, uint64_t seed, void* stream,
                          const lbm_allocator* alloc, lbm_net** out);
lbm_status lbm_net_destroy(lbm_net* n);
lbm_status lbm_net_num_params(const lbm_net* n, int64_t* count);
lbm_status lbm_net_get_params(const lbm_net* n, float* host);
lbm_status lbm_net_set_params(lbm_net* n, const float* host);
lbm_status lbm_net_forward(lbm_net* n, const void* x, int32_t D, int32_t H, int32_t W, int32_t nvol, void* z);
lbm_status lbm_net_predict(lbm_net* n, const void* x, const float* skip, int32_t D, int32_t H, int32_t W, int32_t nvol,
                           float* pred);
lbm_status lbm_net_gradient(lbm_net* n, const float* skip, const float* target, const float* weight, double* loss);
lbm_status lbm_net_get_grads(const lbm_net* n, float* host);
lbm_status lbm_net_train_step(lbm_net* n, const void* x, const float* skip, const float* target, const float* weight,
                              int32_t D, int32_t H, int32_t W, int32_t nvol, float lr, double* loss);
/* Tensor-core path of the convolutions: 1 (default) runs them with tcgen05.mma into TMEM where
 * a volume's zero-padded planes fit in shared memory (W, H up to about 40), 0 with warp-level
 * mma.sync everywhere.  Both compute the same products in BF16 x BF16 -> FP32; the sums are
 * ordered differently.  Calls that wait on the tcgen05 kernel return LBM_ETIMEOUT if one of its
 * bounded waits ran out. */
lbm_status lbm_net_set_backend(lbm_net* n, int32_t backend);
/* Test of the timeout path: with on = 1 the tcgen05 convolution issues no tensor-core products and
 * polls its mbarrier at most 1,024 times, so the wait runs out with nothing asynchronous in flight;
 * the kernel flags it, releases its tensor memory and returns, and the call that waits on it
 * (lbm_net_forward, lbm_net_predict, lbm_net_train_step) returns LBM_ETIMEOUT with incomplete
 * outputs.  on = 0 (the default) restores normal operation.  No GPU fault is involved. */
lbm_status lbm_net_set_wait_test(lbm_net* n, int32_t on);

/* ---- totals without allocation ------------------------------------------------------------
 * The paper has no counterpart: this entry point serves callers that cannot allocate device
 * memory when they need mass and momentum totals (runtimes that own all device memory through
 * their own pool; hosts that forbid dynamic allocation after start-up).  It calls no cudaMalloc, cudaFree or
 * other allocating routine.  Its per-CTA partial sums live in one fixed device array of
 * (LBM_NOALLOC_MAX_CELLS / LBM_NOALLOC_CELLS_PER_CTA) x 5 doubles = 640 KiB, which every GPU that
 * loads the library holds until the process exits.
 *
 *   pdfs      device pointer, [19][n_cells] in the storage layout of `precision`: LBM_FP64 holds f
 *             (for example the output of lbm_get_pdfs, which is always FP64 f); LBM_FP32S and
 *             LBM_FP16S hold f - f^eq(rho0, u_shift), the forests' own storage of those precisions
 *   n_cells   0 .. LBM_NOALLOC_MAX_CELLS; larger counts return LBM_EINVAL without launching
 *   rho0      reference density; with the shifted layouts each finite cell adds rho0 to rho
 *   u_shift   host pointer to 3 doubles, the storage shift of the shifted layouts (NULL = 0); each
 *             finite cell adds rho0 u_shift to j.  Ignored for LBM_FP64
 *   out       device pointer to 5 doubles: {sum rho, sum j_x, sum j_y, sum j_z, skipped}, with
 *             j = sum_a e_a f_a of the values given.  Cells whose 19 values do not sum to a finite
 *             number are left out and counted in `skipped`: obstacle cells (NaN by design) and any
 *             diverged fluid cell, so a count above the caller's obstacle count flags divergence
 *   stream    cudaStream_t; the call is asynchronous
 * Body force: a forest's stored state is post-collision, whose momentum includes rho0 a per fluid
 * cell (Sec. 2.1).  lbm_reduce_mass_momentum subtracts it; this entry point returns j of the values
 * as given, so callers with a body force subtract rho0 a per fluid cell themselves.
 * A CUDA error already pending when the call starts is returned as LBM_ECUDA without launching.
 * The first call on each device looks up the device address of the fixed array
 * (cudaGetSymbolAddress, which allocates nothing).
 * All calls share the array and it keeps the last call's partial sums; every call writes each
 * slot it reads, so nothing has to be cleared, but calls that overlap on the GPU (other streams
 * or threads without ordering between them) race on it and return wrong totals. */
#define LBM_NOALLOC_CELLS_PER_CTA 4096
#define LBM_NOALLOC_MAX_CELLS (16384 * 4096)
lbm_status lbm_mass_momentum_noalloc(const void* pdfs, int32_t precision, int64_t n_cells, double rho0,
                                     const double* u_shift, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
