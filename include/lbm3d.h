/*
 * lbm3d.h -- C ABI of the three-dimensional (D3Q19) form of the loop of
 * Sec. 2.3: a lattice BGK solve on a 3D cell map, the FP64 pressure drop and
 * outlet flow rates, and the optimality-criterion exchange of fluid and solid
 * cells at fixed volume.  The paper computes in 2D and names 3D distributors
 * as the next step; the 3D rules below carry its 2D rules over one axis at a
 * time (stated per entry point).
 *
 * Status codes, error reporting (lbm_last_error), ownership and threading are
 * those of lbm.h: the library owns its device buffers, caller buffers are
 * borrowed for the call, every call returns after its device work is done.
 *
 * Lattice units, dx = dt = 1.  x runs along the flow (0..nx-1), y and z
 * across; a cell is addressed as idx = (z*ny + y)*nx + x.  Directions:
 *   0 rest; 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z;
 *   7 (+x,+y), 8 (-x,-y), 9 (+x,-y), 10 (-x,+y), 11 (+x,+z), 12 (-x,-z),
 *   13 (+x,-z), 14 (-x,+z), 15 (+y,+z), 16 (-y,-z), 17 (+y,-z), 18 (-y,+z);
 * weights 1/3, 1/18 (faces), 1/36 (edges); c_s^2 = 1/3.
 *
 * Geometry rules (lbm3d_create; LBM_ERR_GEOMETRY otherwise):
 *   - the faces y = 0, y = ny-1, z = 0, z = nz-1 are solid (but a face next
 *     to a symmetry plane, see mirror);
 *   - inlet cells are the fluid cells of x = 0, outlet cells those of
 *     x = nx-1; a fluid (0,y,z) has a fluid (1,y,z), a fluid (nx-1,y,z) a
 *     fluid (nx-2,y,z); at least one inlet and one outlet cell;
 *   - the outlet cells form at most LBM_MAX_OUTLETS regions (4-connected in
 *     y, z), numbered in the order of their first cell (z-major, then y);
 *   - 4 <= nx, 3 <= ny, 3 <= nz, nx*ny*nz < 2^31 (LBM_ERR_ARG otherwise).
 * The optimiser never changes the cells with x < 2, x > nx-3, y = 0,
 * y = ny-1, z = 0 or z = nz-1 (a plane's layer stays as given).
 */
#ifndef LBM3D_GB300_H
#define LBM3D_GB300_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3d_handle_s* lbm3d_handle;

typedef struct {
  int32_t nx, ny, nz;  /* lattice size */
  int32_t precision;   /* lbm_precision: populations stored shifted, g_i = f_i - w_i rho0,
                          as FP32, BF16 or FP16; FP32 arithmetic in every case */
  double tau;          /* BGK relaxation time (> 1/2); nu = (tau - 1/2)/3 */
  double rho0;         /* reference density: initial state, outlet density */
  double u_max;        /* inlet speed scale: u_x = u_max a_y a_z with a = 4 s (1 - s) across
                          the inlet cell's fluid run along y and along z, s the cell
                          centre's position in its run (Sec. 3.3's parabola per axis) */
  int32_t reinit;      /* lbm_reinit, as in 2D */
  int32_t collision;   /* lbm_collision, as in 2D: BGK, regularised BGK (the non-equilibrium
                          part relaxed on its second-order Hermite projection) or Smagorinsky
                          (BGK at the local tau_eff of the closure nu_t = C^2 |S|) */
  double c_smag;       /* Smagorinsky constant C (>= 0) */
  int32_t mirror;      /* symmetry planes (Sec. 3.3's half domain, per plane): bit 0 a plane
                          half a cell below y = 0, bit 1 one below z = 0 (both: a quarter
                          domain).  The layer next to a plane may be fluid; what crosses a
                          plane comes back with that component of c negated (both past the
                          corner), a solid image reflects as a wall, and an inlet run
                          against a plane is half of a run twice as wide */
  int32_t reserved;    /* zero */
} lbm3d_params;

typedef struct {
  double dp;       /* mean p = rho/3 over the inlet cells minus the mean over the outlet cells */
  double m_in;     /* sum of rho u_x over the inlet cells */
  int32_t n_outlets;
  int32_t reserved;
  double m_out[LBM_MAX_OUTLETS]; /* sum of rho u_x over the cells of each outlet region */
  int64_t steps_done;            /* total time steps taken by this handle */
  int64_t fluid_cells;           /* current number of fluid cells */
} lbm3d_solve_result;

typedef struct {
  int32_t n_swapped;   /* fluid->solid (= solid->fluid) exchanges made */
  int32_t reserved;
  int64_t fluid_count; /* fluid cells after the exchange (equal to before) */
  lbm3d_solve_result solve;
} lbm3d_opt_result;

/* field selectors for lbm3d_read_fields (one per call); dense [nz][ny][nx] */
#define LBM3D_FIELD_DRHO 1u /* float: rho - rho0 of the last step (0 on solid cells) */
#define LBM3D_FIELD_UX 2u   /* float: u_x of the last step (0 on solid cells) */
#define LBM3D_FIELD_UY 4u   /* float: u_y */
#define LBM3D_FIELD_UZ 8u   /* float: u_z */
#define LBM3D_FIELD_MASK 16u /* uint8: current cell types, 1 = solid */
#define LBM3D_FIELD_POPS 32u /* storage type [19][nz][ny][nx]: post-collision populations in
                                shifted form g_i = f_i - w_i rho0 (garbage on solid cells) */

/* Create a lattice from a cell map; the state starts at rest at rho0.
 * params      host pointer, copied.
 * cell_types  host uint8[nz][ny][nx], 1 = solid, 0 = fluid; copied.
 * cuda_stream cudaStream_t to run on, or NULL for a library-owned stream.
 * out         receives the handle (NULL on failure).                     */
lbm_status lbm3d_create(const lbm3d_params* params, const uint8_t* cell_types, void* cuda_stream,
                        lbm3d_handle* out);
void lbm3d_destroy(lbm3d_handle h);

/* Advance n_steps (even, >= 2) time steps of the fused stream-collide update
 * (halfway bounce-back on solid cells; ports: the inlet imposes
 * u = (u_in, 0, 0), the outlet rho = rho0, each unknown population taking
 * the equilibrium plus the non-equilibrium part of its opposite, then the
 * port cell regularised), then reduce dp, m_in and m_out in FP64.
 * out: host, caller-owned.  LBM_ERR_DIVERGED if a density or speed of the
 * last step is not finite.                                              */
lbm_status lbm3d_solve(lbm3d_handle h, int64_t n_steps, lbm3d_solve_result* out);

/* Sec. 2.2-2.3 steps 3-4 on the 6-neighbourhood: from the field of the last
 * solve, exchange n = min(n_swap, interface fluid cells, interface solid
 * cells) fluid cells of lowest q = 1/2 rho |u|^2 with the n solid cells of
 * largest sigma = sum over fluid face neighbours (order +x, +y, -x, -y, +z,
 * -z) of mu |u_t| / 0.5, |u_t| the magnitude of the neighbour's two velocity
 * components along the shared face (FP64, no fused multiply-add; ties to the
 * smaller idx); re-initialise (params.reinit), then solve n_steps.       */
lbm_status lbm3d_optimize_step(lbm3d_handle h, int32_t n_swap, int64_t n_steps, lbm3d_opt_result* out);

/* The whole loop of Sec. 2.3 on a 3D lattice, with the plan and summary of
 * lbm_optimize (lbm.h): a first solve, then up to max_iter iterations of
 * lbm3d_optimize_step, the same stopping test, n_swap halving and keeping
 * of the best state (populations, mask and fields) as in 2D.  dp_history:
 * host double[max_iter + 1] or NULL.  out: host, caller-owned.           */
lbm_status lbm3d_optimize(lbm3d_handle h, const lbm_opt_plan* plan, double* dp_history, lbm_opt_summary* out);

/* Copy one field (a single LBM3D_FIELD_* bit) into dst; dst_is_device != 0:
 * dst is device memory, written on the handle's stream.                   */
lbm_status lbm3d_read_fields(lbm3d_handle h, uint32_t which, void* dst, size_t dst_bytes, int dst_is_device);

/* Replace the populations (LBM3D_FIELD_POPS layout); values on solid cells
 * are ignored.  For checkpoint/resume and for tests from a given state.   */
lbm_status lbm3d_load_state(lbm3d_handle h, const void* pops, size_t bytes, int src_is_device);

/* Test hook of the selection on a supplied field (host float [nz][ny][nx]
 * each, rho = rho0 + drho) and the handle's current cell map; the chosen
 * indices go to host int32[n_swap] arrays sorted ascending, n to n_out.   */
lbm_status lbm3d_select_swaps(lbm3d_handle h, const float* drho, const float* ux, const float* uy,
                              const float* uz, int32_t n_swap, int32_t* fluid_idx_out,
                              int32_t* solid_idx_out, int32_t* n_out);

/* Time of the stream-collide kernels since creation (or the last reset),
 * from CUDA events around them on the handle's stream; launches and fluid
 * cell updates in the same span.                                          */
lbm_status lbm3d_kernel_time(lbm3d_handle h, int reset, double* ms, int64_t* launches, int64_t* fluid_updates);

/* Block shape of the stream-collide kernels: warps per block (4, 8 or 16). */
lbm_status lbm3d_set_block(lbm3d_handle h, int32_t warps_per_block);

/* Test hook: the stream-collide tasks of the current work-list.  A row
 * segment (32 cells of one mask word) holding at least P fluid cells is one
 * warp task; the fluid cells of the sparser segments (but for the first and
 * last word of a row and the layers next to a symmetry plane) are packed 32
 * to a warp task.  P is 16 with FP32 storage and 24 with 16-bit storage,
 * or LBM3D_PACK_BELOW (environment at lbm3d_create, 0 .. 32; 0: every
 * segment holding fluid is a task).  Both give the same bits per cell
 * (Eq. 1-2 with the rules of Sec. 3.3).  Host int32 outputs.              */
lbm_status lbm3d_debug_task_counts(lbm3d_handle h, int32_t* segment_tasks, int32_t* packed_tasks);

#ifdef __cplusplus
}
#endif

#endif /* LBM3D_GB300_H */
