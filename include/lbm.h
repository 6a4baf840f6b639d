/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the lattice Boltzmann
 * shape-optimisation loop of Wang, Fan & Luo, "Lattice Boltzmann method for
 * shape optimization of fluid distributor" (arXiv:1303.0107).
 *
 * The library owns every device buffer it allocates.  Caller buffers are
 * borrowed for the duration of a call only.  Nothing is thrown across the
 * ABI: every entry point returns an lbm_status.  A failed call leaves its
 * handle usable unless the status is LBM_ERR_CUDA; lbm_last_error() gives a
 * one-line description of the last failure on the calling thread.
 *
 * Lattice units throughout: dx = dt = 1.  x runs along the flow (0..nx-1),
 * y across (0..ny-1); a cell is addressed as idx = y*nx + x.  Directions:
 * 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.
 *
 * Geometry rules (checked by lbm_create_geometry, LBM_ERR_GEOMETRY otherwise):
 *   - rows 0 and ny-1 are solid (the frame; row 0 may be fluid when
 *     lbm_params.mirror puts a symmetry plane below it);
 *   - inlet cells are the fluid cells of column 0, outlet cells those of
 *     column nx-1; each fluid cell (0,y) has a fluid (1,y) and each fluid
 *     (nx-1,y) a fluid (nx-2,y);
 *   - at least one inlet and one outlet cell, at most LBM_MAX_OUTLETS outlet
 *     runs; 4 <= nx <= 131072, 3 <= ny < 524288, and 9 * ny * pitch < 2^31
 *     with pitch = nx rounded up to 64; with the zero-gradient outlet
 *     (LBM_OUT_NEUMANN) nx mod 32 != 1, because the outlet cell takes the
 *     streamed populations of cell nx-2 from the neighbouring lane of its
 *     32-cell row segment (LBM_ERR_ARG).
 * The optimiser never changes columns 0, 1, nx-2, nx-1 nor rows 0, ny-1.
 *
 * Threading: a handle is used by one host thread at a time.  All device work
 * of a handle runs on the stream given at creation (or a stream the library
 * creates when none is given); every entry point returns after that work is
 * complete unless stated otherwise.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAX_OUTLETS 64

typedef struct lbm_handle_s* lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, odd step count, ...) */
  LBM_ERR_GEOMETRY = 2,  /* cell map violates the geometry rules above */
  LBM_ERR_OOM = 3,       /* device or pinned host allocation failed */
  LBM_ERR_CUDA = 4,      /* a CUDA call failed; the handle must be destroyed */
  LBM_ERR_DIVERGED = 5,  /* a reduction or a score is not finite */
  LBM_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
  LBM_ERR_BUSY = 7,      /* resource temporarily unavailable (admission refused) */
  LBM_ERR_CANCELLED = 8  /* a served request withdrawn with lbm_server_cancel */
} lbm_status;

typedef enum {
  LBM_F32 = 0,          /* populations stored as FP32, shifted: g_i = f_i - w_i rho0 */
  LBM_BF16_SHIFTED = 1, /* stored as BF16, shifted; FP32 collision arithmetic */
  LBM_F16_SHIFTED = 2   /* stored as FP16, shifted; FP32 collision arithmetic */
} lbm_precision;

typedef enum {
  LBM_OUT_CONST_RHO = 0, /* outlet density fixed at rho0 (see lbm_port_scheme) */
  LBM_OUT_NEUMANN = 1    /* zero-gradient outlet (Sec. 3.3): unknown f3,f6,f7 copied
                            from the streamed populations of cell (nx-2, y) */
} lbm_outlet_rule;

typedef enum {
  LBM_PORTS_REGULARIZED = 0, /* velocity inlet / constant-density outlet: the Zou-He
                                density and velocity, non-equilibrium bounce-back for
                                the unknown populations, then the port cell is
                                regularised (f^eq + projected non-equilibrium stress);
                                stable for tau close to 1/2 */
  LBM_PORTS_ZOU_HE = 1       /* plain Zou-He reconstruction of the unknown populations */
} lbm_port_scheme;

typedef enum {
  LBM_REINIT_WARM = 0, /* after an exchange only new fluid cells restart at f^eq(rho0, 0) */
  LBM_REINIT_COLD = 1  /* after an exchange every fluid cell restarts at f^eq(rho0, 0) */
} lbm_reinit;

typedef enum {
  LBM_COLLIDE_BGK = 0,         /* single relaxation time, Eq. 1 */
  LBM_COLLIDE_REGULARIZED = 1, /* BGK applied to the regularised populations: the
                                  non-equilibrium part is projected on its second
                                  moment before relaxing (more stable as tau -> 1/2) */
  LBM_COLLIDE_SMAGORINSKY = 2  /* BGK with a local relaxation time from the
                                  Smagorinsky eddy viscosity (constant c_smag) */
} lbm_collision;

typedef struct {
  int32_t nx, ny;         /* lattice size */
  double tau;             /* BGK relaxation time of Eq. 1 (> 1/2); nu = (tau - 1/2)/3 */
  double rho0;            /* reference density: initial state, outlet density */
  double u_max;           /* centre-line speed of the parabolic inlet profile */
  int32_t outlet;         /* lbm_outlet_rule */
  int32_t precision;      /* lbm_precision */
  int32_t reinit;         /* lbm_reinit */
  int32_t residual_every; /* K: the residual compares u at the last step with u
                             K steps earlier; even, >= 2 (0 disables it) */
  int32_t ports;          /* lbm_port_scheme */
  int32_t guard;          /* 1: connectivity guard -- a fluid cell may turn solid
                             only if it is simple: its fluid 4-neighbours stay
                             connected within its 3 x 3 block without it and it
                             joins exactly one solid part (4-connectivity number 1) */
  int32_t collision;      /* lbm_collision */
  int32_t mirror;         /* 1: a symmetry plane lies half a cell below row 0 (Sec. 3.3
                             computes half of the domain): row 0 may be fluid, and
                             what streams in across the plane is the mirror image of
                             what row 0 sends out; an inlet run touching the plane is
                             half of a run twice as wide centred on it */
  double c_smag;          /* Smagorinsky constant (LBM_COLLIDE_SMAGORINSKY; >= 0) */
} lbm_params;

typedef struct {
  double dp;        /* pressure drop: mean p = rho/3 (Eq. 4) over inlet cells minus
                       the mean over all outlet cells (Sec. 2.3 step 5) */
  double m_in;      /* sum of rho u_x over the inlet cells (per unit depth) */
  double residual;  /* sum |u(T) - u(T-K)|_1 / sum |u(T)|_1 over fluid cells; -1 if not computed */
  int32_t n_outlets;
  int32_t reserved;
  double m_out[LBM_MAX_OUTLETS]; /* sum of rho u_x over the cells of each outlet, runs
                                    numbered from y = 0 upward */
  double theta;     /* Eq. 9: max m_out / min m_out */
  double dg;        /* Eq. 10-11: maldistribution factor of m_out */
  int64_t steps_done;  /* total time steps taken by this handle */
  int64_t fluid_cells; /* current number of fluid cells */
} lbm_solve_result;

typedef struct {
  int32_t n_swapped;   /* number of fluid->solid (= solid->fluid) exchanges made */
  int32_t reserved;
  int64_t fluid_count; /* fluid cells after the exchange (always equal to before) */
  lbm_solve_result solve;
} lbm_opt_result;

/* field selectors for lbm_read_fields / lbm_load_state (one per call) */
#define LBM_FIELD_RHO 1u  /* float[ny][nx]: rho of the last step (0 on solid cells) */
#define LBM_FIELD_UX 2u   /* float[ny][nx]: u_x of the last step (0 on solid cells) */
#define LBM_FIELD_UY 4u   /* float[ny][nx]: u_y of the last step (0 on solid cells) */
#define LBM_FIELD_MASK 8u /* uint8[ny][nx]: current cell types, 1 = solid, 0 = fluid */
#define LBM_FIELD_POPS 16u /* storage type [9][ny][nx]: post-collision populations in
                              stored (shifted) form g_i = f_i - w_i rho0; FP32 for
                              LBM_F32, BF16 / FP16 bit patterns otherwise */
#define LBM_FIELD_DRHO 32u /* float[ny][nx]: rho - rho0 of the last step */

/* Sec. 2.3 step 1 and Sec. 3.3: create a lattice from a cell map.
 * params      host pointer, copied.
 * cell_types  host uint8[ny][nx] row-major, 1 = solid, 0 = fluid; copied.
 * cuda_stream cudaStream_t to run on, or NULL for a library-owned stream.
 * out         receives the handle (NULL on failure).
 * The state starts at the equilibrium of rho0 at rest (Sec. 3.3).        */
lbm_status lbm_create_geometry(const lbm_params* params, const uint8_t* cell_types, void* cuda_stream,
                               lbm_handle* out);

/* Sec. 2.3 step 2, Eq. 1-2: advance n_steps time steps of the fused
 * stream-collide update (bounce-back walls, inlet and outlet rules of Sec. 3.3),
 * then reduce the pressure drop, flow rates and residual in FP64.
 * n_steps must be even and >= 2 (steps run as pairs of the single-lattice
 * scheme).  out: host pointer, caller-owned.                             */
lbm_status lbm_solve(lbm_handle h, int64_t n_steps, lbm_solve_result* out);

/* Sec. 2.2 (Eq. 5, Eq. 6) and Sec. 2.3 steps 3-4: from the field of the last
 * solve, exchange n = min(n_swap, interface fluid cells, interface solid
 * cells) fluid cells of lowest dynamic pressure with the n solid cells of
 * largest viscous stress, re-initialise (params.reinit), then solve n_steps.
 * Requires a previous lbm_solve on this handle.  out: host, caller-owned.  */
lbm_status lbm_optimize_step(lbm_handle h, int32_t n_swap, int64_t n_steps, lbm_opt_result* out);

/* Copy one field (a single LBM_FIELD_* bit) into dst.
 * dst_bytes must be at least the field's size; dst_is_device != 0 means dst
 * is device memory of the handle's device (written on the handle's stream).  */
lbm_status lbm_read_fields(lbm_handle h, uint32_t which, void* dst, size_t dst_bytes, int dst_is_device);

/* Restore the populations (LBM_FIELD_POPS layout) saved by lbm_read_fields,
 * for checkpoint/resume on a handle with the same cell map.             */
lbm_status lbm_load_state(lbm_handle h, const void* pops, size_t bytes, int src_is_device);

/* Put the handle back to its creation state: initial cell map, equilibrium
 * populations, steps_done = 0.  No allocation.                          */
lbm_status lbm_reset(lbm_handle h);

/* Test hook for the selection of Sec. 2.3 step 3 on a supplied field: scores
 * (Eq. 5, Eq. 6, FP64, no fused multiply-add) and the deterministic choice,
 * fluid cells by (q ascending, idx ascending), solid cells by (sigma
 * descending, idx ascending), on the handle's current cell map.
 * drho, ux, uy: host float[ny][nx], rho = rho0 + drho.  fluid_idx_out and
 * solid_idx_out: host int32[n_swap], receive the chosen cell indices sorted
 * ascending; n_out receives n.  The handle's state is not changed.       */
lbm_status lbm_select_swaps(lbm_handle h, const float* drho, const float* ux, const float* uy,
                            int32_t n_swap, int32_t* fluid_idx_out, int32_t* solid_idx_out,
                            int32_t* n_out);

/* ---- the whole optimisation loop ------------------------------------------
 * Sec. 2.3 run end to end on one handle: a first solve, then up to max_iter
 * iterations of {exchange, re-solve} (lbm_optimize_step).  The paper stops
 * when the pressure drop "tends to extremum" without a tolerance; the reading
 * here: stop after an iteration once |dp_k - dp_(k-1)| <= tol |dp_k| has held
 * for `patience` consecutive iterations (tol <= 0: run all max_iter).  The
 * paper fixes neither the number of cells per exchange nor what to keep: with
 * adapt = 1, n_swap is halved (down to 1) after every iteration that raised
 * dp; with keep_best = 1, the handle ends in the state (cell map,
 * populations and fields) of the lowest dp seen.                           */
typedef struct {
  int64_t n_steps;   /* time steps of every solve (even, >= 2) */
  int32_t max_iter;  /* exchange iterations at most (>= 0) */
  int32_t n_swap;    /* exchanges per iteration at the start (>= 1) */
  double tol;        /* extremum test tolerance (relative); <= 0 disables it */
  int32_t patience;  /* consecutive calm iterations that stop the loop (>= 1) */
  int32_t adapt;     /* 0 or 1 */
  int32_t keep_best; /* 0 or 1 */
  int32_t reserved;  /* must be 0 */
} lbm_opt_plan;

typedef struct {
  int32_t iterations;   /* exchange iterations run */
  int32_t best_iter;    /* iteration with the lowest dp (0: the first solve) */
  int32_t stopped;      /* 1 if the extremum test ended the loop */
  int32_t n_swap_final; /* n_swap in force at the end */
  int64_t swapped;      /* cells exchanged over all iterations (each way) */
  double dp_first;      /* dp of the first solve */
  double dp_best;       /* lowest dp */
  double dp_last;       /* dp of the last solve run */
} lbm_opt_summary;

/* dp_history: host double[max_iter + 1] or NULL; receives dp of the first
 * solve and of every iteration run (summary.iterations + 1 values).
 * out: host, caller-owned.  On an error the history up to the failure has
 * been written and the handle holds the state of the failing call.        */
lbm_status lbm_optimize(lbm_handle h, const lbm_opt_plan* plan, double* dp_history, lbm_opt_summary* out);

/* Largest lattice (nx * ny cells) accepted by lbm_select_swaps_noalloc;
 * nx and ny are also limited to 4096 each.                              */
#define LBM_NOALLOC_MAX_CELLS 262144

/* The selection of lbm_select_swaps without any device allocation.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- for example code running inside a host application whose
 * memory pool owns the whole device and forbids raw allocations, or a loop
 * that must not risk the implicit device synchronisation of cudaMalloc and
 * cudaFree.  The caller passes device buffers only and no handle is needed:
 *   nx, ny       lattice size, nx * ny <= LBM_NOALLOC_MAX_CELLS, nx, ny <= 4096
 *                (LBM_ERR_ARG beyond that, before any device work);
 *   tau, rho0    as in lbm_params (mu = rho0 (tau - 1/2) / 3);
 *   cell_types   device uint8[ny][nx], 1 = solid, 0 = fluid;
 *   drho, ux, uy device float[ny][nx] (rho = rho0 + drho);
 *   fluid_idx_out, solid_idx_out  device int32[n_swap]: the chosen cells,
 *                ascending; n_out: device int32, receives n, or -1 if a score
 *                is not a number;
 *   cuda_stream  stream to enqueue on (NULL: the legacy default stream).
 * The selection is that of lbm_select_swaps on a handle created with
 * guard = 0: the connectivity guard of lbm_params.guard is not applied.
 * The call only enqueues kernels and a memset on the stream (it copies
 * nothing from host memory) and returns; results are valid once that work
 * has completed on the stream.  All intermediate storage is one static
 * device array of about 7.4 MB that every GPU loading the library keeps
 * until the process exits; every call looks up its device address with
 * cudaGetSymbolAddress.  The first call on each device is also where CUDA
 * loads the library's device code for that device (module loading is lazy
 * by default), which commits the array and the selection kernels in device
 * memory: make that first call before any stream capture, and before the
 * application reserves the device's memory for its own pool.
 * All calls share the array and it keeps the previous call's contents, so
 * calls whose work overlaps on the GPU (different streams, no ordering)
 * corrupt each other; calls on one stream are ordered and safe.  Errors
 * are reported as for every entry point, through lbm_last_error().        */
lbm_status lbm_select_swaps_noalloc(int32_t nx, int32_t ny, double tau, double rho0,
                                    const uint8_t* cell_types, const float* drho,
                                    const float* ux, const float* uy, int32_t n_swap,
                                    int32_t* fluid_idx_out, int32_t* solid_idx_out,
                                    int32_t* n_out, void* cuda_stream);

/* Release every resource of the handle.  NULL is accepted.              */
void lbm_destroy(lbm_handle h);

/* Static description of a status code.                                  */
const char* lbm_status_str(lbm_status s);

/* Description of the last failure on the calling thread ("" if none).   */
const char* lbm_last_error(void);

/* Test hook for the failure paths: the device allocation made after `after`
 * further successful ones fails as if the device were full (LBM_ERR_OOM from
 * the call that needed it); after < 0 switches the hook off.  One-shot.   */
void lbm_debug_fail_alloc(int64_t after);

/* Test hook for the bounded device-side waits (process-wide; on != 0 until
 * called again with 0): the persistent step kernel's grid barriers then wait
 * for one arrival more than the grid makes, and the resident kernel's halo
 * polls for a step tag that nobody writes, so every wait gives up after its
 * poll limit (2^22 loads, a few seconds), the launch ends early and the
 * solve returns LBM_ERR_TIMEOUT; the handle stays usable (lbm_reset or
 * lbm_load_state restores a state).  No device fault is involved.         */
void lbm_debug_barrier_timeout(int32_t on);

/* Test hook of the bounds-checked build (built with -DLBM_CHECK_BOUNDS, loaded
 * with LBM_CHECKED=1 by the Python binding): that build surrounds every
 * lattice's population planes with canary blocks and checks them after each
 * solve and optimiser step (LBM_ERR_CUDA, naming the lattice, if one was
 * overwritten).  This call overwrites a few bytes of the handle's upper canary
 * with a host-side memset inside the allocation, so that the next solve
 * reports it.  LBM_ERR_ARG in the normal build, which has no canaries.    */
lbm_status lbm_debug_damage_canary(lbm_handle h);

/* Sizes of the handle's task lists (builds them if needed; synchronises the
 * handle's stream): *segments = row segments holding a fluid cell (the work
 * of launch mode 0), *windows = interior windows of 64 cells among them
 * (row y, cells 64p .. 64p+63, p >= 0, with rows y-1..y+1 fluid over cells
 * 64p-1 .. 64p+64; the columns beyond the lattice count as solid), which
 * launch mode 4 takes two cells a lane.  0 windows on lattices with a
 * symmetry plane.  Either pointer may be NULL.                            */
lbm_status lbm_debug_task_counts(lbm_handle h, int32_t* segments, int32_t* windows);

/* Number of device kernels this process has launched through the library
 * (graph launches count every kernel node).                             */
uint64_t lbm_kernel_launches(void);

/* Bytes the library has copied from host to device memory (*h2d) and from
 * device to host memory (*d2h) in this process through the lbm_* and
 * lbm_batch_* entry points (uploads of cell maps and tables, result blocks,
 * exchange counters, field reads): the transfer cost of a run, for its
 * end-to-end accounting.  Either pointer may be NULL.                     */
void lbm_transfer_bytes(uint64_t* h2d, uint64_t* d2h);

/* Device time of the stream-collide kernels of this handle, measured with CUDA
 * events on the handle's stream around each solve's sequence of time steps
 * (the FP64 reductions and the exchange are outside it).  ms, launches and
 * fluid_updates (fluid cells x steps) are accumulated since creation or since
 * the last call with reset != 0; any output pointer may be NULL.          */
lbm_status lbm_kernel_time(lbm_handle h, int reset, double* ms, int64_t* launches,
                           int64_t* fluid_updates);

/* Launch shape the handle's time steps use: warps per block, blocks, the
 * launch mode `persistent` -- 0: one launch per phase over the row segments;
 * 1: every run of time steps in one cooperative launch with grid-wide
 * barriers between phases; 2: on-chip resident solves (each solve one
 * cooperative launch, the populations in shared memory, neighbouring blocks
 * exchanging tagged halo words; plain BGK lattices whose cells fit on the
 * device); 3: one launch per phase over compacted fluid-cell tasks (32
 * consecutive fluid cells per warp; plain BGK lattices without a
 * zero-gradient outlet); 4: one launch per phase over paired tasks (a warp
 * takes each interior window of 64 cells -- cells and neighbours all fluid
 * -- two cells a lane with paired loads and stores, and every other row
 * segment as in mode 0; plain BGK lattices) -- cells_per_thread = row segments each warp
 * updates at once (1 or 2), and stages = 0 (populations loaded straight into
 * registers) or 2 / 3 (copied into shared memory that many segments ahead of
 * their update).  Tuned on the handle's own lattice at its first solve of
 * 256 steps or more, unless set with lbm_set_step_config.  Any output
 * pointer may be NULL.                                                    */
lbm_status lbm_step_config(lbm_handle h, int32_t* warps_per_block, int32_t* grid, int32_t* persistent,
                           int32_t* cells_per_thread, int32_t* stages);
/* Fix the launch shape (and skip tuning): warps_per_block 4, 8, 12, 16 or
 * 32 with one cell per thread, 4, 8, 12 or 24 with two (32 and 24: one
 * block per SM); 8 or 16 when persistent = 1 (8 with two cells per thread);
 * 4, 8 or 16 with stages.  cells_per_thread 1 or 2, stages 0, 2 or 3
 * (staged loads: one cell per thread, persistent = 0); persistent = 2:
 * resident solves, the shape follows from the lattice (the other arguments
 * are ignored); persistent = 3: cell tasks, warps_per_block 4, 8, 12, 16 or
 * 32, one cell per thread, stages 0; persistent = 4: paired tasks,
 * warps_per_block 4, 8, 12 or 24, cells_per_thread 2, stages 0 (windows
 * loaded into registers) or 2, 3, 4 (copied into shared memory that many
 * tasks ahead).  The grid is
 * sized for the device.  LBM_ERR_ARG for any other shape, or for modes 2 - 4
 * on lattices they do not serve.  Every shape computes the same values, so this changes timings
 * only.                                                                   */
lbm_status lbm_set_step_config(lbm_handle h, int32_t warps_per_block, int32_t persistent,
                               int32_t cells_per_thread, int32_t stages);

/* ---- batches -------------------------------------------------------------
 * Many candidate geometries (Sec. 2.3 applied to each) stepped together: one
 * work-list over all members, one launch per time step, per optimiser
 * iteration and per reduction for the whole batch.  Members may differ in
 * size, tau, u_max, outlet rule, port scheme and re-initialisation; they
 * share precision and residual_every.  Each member evolves exactly as it
 * would in a handle of its own (same results, bit for bit).                */
typedef struct lbm_batch_s* lbm_batch;

/* params: host lbm_params[n]; cell_types: host array of n host pointers to
 * uint8[ny_i][nx_i]; both copied.  Same geometry rules as a handle.        */
lbm_status lbm_batch_create(int32_t n, const lbm_params* params, const uint8_t* const* cell_types,
                            void* cuda_stream, lbm_batch* out);
/* As lbm_solve for every member; out: host lbm_solve_result[n].          */
lbm_status lbm_batch_solve(lbm_batch b, int64_t n_steps, lbm_solve_result* out);
/* As lbm_optimize_step for every member; n_swap: host int32[n] (per member);
 * out: host lbm_opt_result[n].                                            */
lbm_status lbm_batch_optimize_step(lbm_batch b, const int32_t* n_swap, int64_t n_steps,
                                   lbm_opt_result* out);
/* As lbm_read_fields for member `member` (0 <= member < n).               */
lbm_status lbm_batch_read_fields(lbm_batch b, int32_t member, uint32_t which, void* dst,
                                 size_t dst_bytes, int dst_is_device);
/* Every member back to its creation state.                                */
lbm_status lbm_batch_reset(lbm_batch b);
/* As lbm_kernel_time, for the batch's time steps (fluid_updates over all members). */
lbm_status lbm_batch_kernel_time(lbm_batch b, int reset, double* ms, int64_t* launches,
                                 int64_t* fluid_updates);
/* As lbm_step_config / lbm_set_step_config.  A batch whose populations
 * exceed the L2 cache runs its time steps in member groups of about a third
 * of the L2 each (members in order, each group with its own work-list and
 * tuned shape), so that a group stays L2-resident through a solve;
 * reductions and exchanges run over the whole batch, and every member
 * evolves exactly as alone.  lbm_batch_step_config then reports the first
 * group's shape; lbm_batch_set_step_config fixes one shape for the whole
 * batch and ends the grouping.  LBM_GROUPS=0 in the environment turns it
 * off.                                                                    */
lbm_status lbm_batch_step_config(lbm_batch b, int32_t* warps_per_block, int32_t* grid, int32_t* persistent,
                                 int32_t* cells_per_thread, int32_t* stages);
/* Number of member groups the batch's time steps run in (1: not grouped;
 * decided at the first solve of 256 steps or more).  n_groups: host.      */
lbm_status lbm_batch_step_groups(lbm_batch b, int32_t* n_groups);
lbm_status lbm_batch_set_step_config(lbm_batch b, int32_t warps_per_block, int32_t persistent,
                                     int32_t cells_per_thread, int32_t stages);
void lbm_batch_destroy(lbm_batch b);

/* ---- serving ---------------------------------------------------------------
 * A request loop with continuous batching.  The paper has no counterpart: it
 * runs one design problem at a time.  Requests -- a solve of a geometry, or
 * the optimisation loop of Sec. 2.3 on it -- arrive at any time from any
 * host thread.  A scheduler thread inside the library admits them in arrival
 * order while their device footprint fits the budget and a slot is free,
 * keeps their populations, masks and fields resident on the device, and
 * advances every resident request in the same launches (one work-list over
 * all of them, as a batch).  Between ticks -- runs of at most max_tick_steps
 * time steps, cut where a resident request finishes a solve -- it retires
 * finished requests, runs the exchanges of the requests that start a new
 * optimiser iteration, and admits new ones.  Each request evolves exactly as
 * it would alone in a handle of its own (same results, bit for bit), whatever
 * else is resident.                                                        */
typedef struct lbm_server_s* lbm_server;

typedef struct {
  int32_t precision;        /* lbm_precision of every request's populations */
  int32_t max_active;       /* most requests resident at once (>= 1) */
  int64_t hbm_budget_bytes; /* admission limit on the summed footprints of the
                               resident requests; 0 = 80 % of the device memory
                               free at creation */
  int32_t max_tick_steps;   /* longest run of time steps between two admissions
                               (even, >= 2) */
  int32_t reserved;         /* must be 0 */
} lbm_server_config;

typedef struct {
  lbm_params params;         /* precision must be the server's; residual_every 0 */
  const uint8_t* cell_types; /* host uint8[ny][nx], 1 = solid; copied at submit */
  int64_t n_steps;           /* time steps of every solve (even, >= 2) */
  int32_t n_iter;            /* optimiser iterations after the first solve (0: solve only) */
  int32_t n_swap;            /* exchanges per iteration (>= 0) */
  int64_t tag;               /* caller's identifier, returned with the result */
  uint8_t* out_mask;         /* optional host uint8[ny][nx]: final cell map */
  float* out_drho;           /* optional host float[ny][nx] each: rho - rho0, u_x, u_y */
  float* out_ux;             /*   of the last step; the out_* buffers must stay valid */
  float* out_uy;             /*   until the request's result has been polled        */
} lbm_request;

typedef struct {
  int64_t tag;
  int32_t status;           /* lbm_status of the request */
  int32_t n_swapped;        /* exchanges made over all iterations */
  double t_submit;          /* server clock (lbm_server_now), seconds */
  double t_admit;
  double t_done;
  int64_t fluid_updates;    /* fluid cells x time steps of the request */
  int64_t footprint_bytes;  /* device bytes charged against the budget */
  double dp_first;          /* pressure drop after the first solve */
  lbm_solve_result last;    /* reductions after the last solve */
} lbm_served;

typedef struct {
  int64_t submitted, admitted, completed, failed;
  int64_t ticks, exchanges;          /* scheduler ticks; ticks that ran an exchange */
  int64_t fluid_updates;             /* over all requests */
  int64_t resident_bytes, peak_resident_bytes; /* charged footprints */
  int64_t device_bytes, peak_device_bytes;     /* device memory the server holds */
  int32_t active, peak_active, queued, reserved;
  double busy_s;                     /* wall time spent in ticks */
  double step_ms;                    /* CUDA-event time of the time steps */
  int64_t budget_bytes;              /* the admission limit in force */
} lbm_server_stats;

/* Start a server (and its scheduler thread) on the current device.
 * cfg: host, copied.  cuda_stream: stream for all device work, or NULL.   */
lbm_status lbm_server_create(const lbm_server_config* cfg, void* cuda_stream, lbm_server* out);
/* Queue a request (thread-safe; returns at once).  LBM_ERR_ARG or
 * LBM_ERR_GEOMETRY for a request that can never run (also when its
 * footprint alone exceeds the budget); the request is then not queued.    */
lbm_status lbm_server_submit(lbm_server s, const lbm_request* r);
/* Move up to max_out finished requests into out (host lbm_served[max_out]),
 * waiting up to wait_ms milliseconds for the first; returns how many.     */
int32_t lbm_server_poll(lbm_server s, lbm_served* out, int32_t max_out, int32_t wait_ms);
/* Withdraw request `tag`: a queued one leaves the queue at once, a resident
 * one is retired at the next tick boundary; either way its result carries
 * LBM_ERR_CANCELLED.  LBM_ERR_ARG if no queued or resident request has the tag. */
lbm_status lbm_server_cancel(lbm_server s, int64_t tag);
/* Wait until nothing is queued or resident; LBM_ERR_TIMEOUT after timeout_ms. */
lbm_status lbm_server_wait_idle(lbm_server s, int32_t timeout_ms);
lbm_status lbm_server_get_stats(lbm_server s, lbm_server_stats* out);
/* Seconds since the server was created (the clock of lbm_served).         */
double lbm_server_now(lbm_server s);
/* Device bytes a request of these parameters is charged at admission.     */
int64_t lbm_server_footprint(const lbm_params* params, int32_t n_iter);
/* Stop the scheduler (resident and queued requests are dropped) and free
 * everything.  NULL is accepted.                                          */
void lbm_server_destroy(lbm_server s);

/* Algorithmic memory traffic of one fluid-cell update of the stream-collide
 * kernel for a storage precision: 9 populations read and 9 written
 * (2 * 9 * sizeof(stored population)) plus the cell's mask bit (1/8 byte).  */
double lbm_bytes_per_fluid_update(int32_t precision);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
