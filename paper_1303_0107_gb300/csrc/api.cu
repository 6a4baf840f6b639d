// C ABI of the library (include/lbm.h): argument checks and dispatch to the
// engine (engine.cu).  A handle (lbm_create_geometry) is an engine of one
// member, a batch (lbm_batch_create) an engine of many; the server
// (server.cu) drives an engine whose member list changes between solves.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

using namespace lbm;

struct lbm_handle_s {
  Engine* e;
};
struct lbm_batch_s {
  Engine* e;
};

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

extern "C" {

const char* lbm_status_str(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_GEOMETRY: return "invalid geometry";
    case LBM_ERR_OOM: return "out of memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_DIVERGED: return "diverged (non-finite value)";
    case LBM_ERR_TIMEOUT: return "timeout";
    case LBM_ERR_BUSY: return "busy";
    case LBM_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char* lbm_last_error(void) { return t_last_error.c_str(); }

uint64_t lbm_kernel_launches(void) { return launches_total(); }

void lbm_transfer_bytes(uint64_t* h2d, uint64_t* d2h) { transfer_bytes(h2d, d2h); }

void lbm_debug_fail_alloc(int64_t after) { set_alloc_failure(after); }

void lbm_debug_barrier_timeout(int32_t on) { set_barrier_timeout_test(on); }

lbm_status lbm_debug_damage_canary(lbm_handle h) {
  if (!h) return fail(LBM_ERR_ARG, "NULL handle");
  return debug_damage_canary(h->e);
}

lbm_status lbm_debug_task_counts(lbm_handle h, int32_t* segments, int32_t* windows) {
  if (!h) return fail(LBM_ERR_ARG, "NULL handle");
  return debug_task_counts(h->e, segments, windows);
}

double lbm_bytes_per_fluid_update(int32_t precision) {
  return 2.0 * 9.0 * (double)storage_bytes(precision) + 1.0 / 8.0;
}

// ---- single lattice ----------------------------------------------------------

void lbm_destroy(lbm_handle h) {
  if (!h) return;
  delete h->e;
  delete h;
}

lbm_status lbm_create_geometry(const lbm_params* params, const uint8_t* cell_types, void* cuda_stream,
                               lbm_handle* out) {
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || !cell_types) return fail(LBM_ERR_ARG, "params or cell_types is NULL");
  Engine* E = nullptr;
  lbm_status st = engine_create(1, params, &cell_types, cuda_stream, &E);
  if (st != LBM_OK) return st;
  *out = new lbm_handle_s{E};
  return LBM_OK;
}

lbm_status lbm_reset(lbm_handle h) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  return engine_reset(h->e);
}

lbm_status lbm_solve(lbm_handle h, int64_t n_steps, lbm_solve_result* out) {
  if (!h || !out) return fail(LBM_ERR_ARG, "handle or out is NULL");
  return engine_solve(h->e, n_steps, out);
}

lbm_status lbm_optimize_step(lbm_handle h, int32_t n_swap, int64_t n_steps, lbm_opt_result* out) {
  if (!h || !out) return fail(LBM_ERR_ARG, "handle or out is NULL");
  if (!h->e->solved) return fail(LBM_ERR_ARG, "lbm_optimize_step needs a field: call lbm_solve first");
  return engine_optimize(h->e, &n_swap, n_steps, out);
}

lbm_status lbm_optimize(lbm_handle h, const lbm_opt_plan* plan, double* dp_history, lbm_opt_summary* out) {
  if (!h || !plan || !out) return fail(LBM_ERR_ARG, "handle, plan or out is NULL");
  return engine_optimize_loop(h->e, *plan, dp_history, out);
}

lbm_status lbm_read_fields(lbm_handle h, uint32_t which, void* dst, size_t dst_bytes, int dst_is_device) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  (void)dst_is_device;  // unified addressing: cudaMemcpyDefault handles both
  return engine_read(h->e, 0, which, dst, dst_bytes);
}

lbm_status lbm_load_state(lbm_handle h, const void* pops, size_t bytes, int src_is_device) {
  if (!h || !pops) return fail(LBM_ERR_ARG, "handle or pops is NULL");
  (void)src_is_device;
  Engine* E = h->e;
  Member* m = E->m[0];
  const size_t nx = m->nx, ny = m->ny, ncell = nx * ny;
  const size_t sb = storage_bytes(E->precision);
  if (bytes < 9 * ncell * sb) return fail(LBM_ERR_ARG, "pops too small");
  for (int i = 0; i < 9; ++i)
    CU(xfer2d(static_cast<char*>(m->f) + i * m->plane * sb, (size_t)m->pitch * sb,
                         static_cast<const char*>(pops) + i * ncell * sb, nx * sb, nx * sb, ny,
                         cudaMemcpyDefault, E->stream));
  CU(cudaStreamSynchronize(E->stream));
  return LBM_OK;
}

lbm_status lbm_kernel_time(lbm_handle h, int reset, double* ms, int64_t* launches, int64_t* fluid_updates) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  return engine_kernel_time(h->e, reset, ms, launches, fluid_updates);
}

lbm_status lbm_step_config(lbm_handle h, int32_t* warps_per_block, int32_t* grid, int32_t* persistent,
                           int32_t* cells_per_thread, int32_t* stages) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  return engine_step_config(h->e, warps_per_block, grid, persistent, cells_per_thread, stages);
}

lbm_status lbm_set_step_config(lbm_handle h, int32_t warps_per_block, int32_t persistent, int32_t cells_per_thread,
                               int32_t stages) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  return engine_set_step_config(h->e, warps_per_block, persistent, cells_per_thread, stages);
}

lbm_status lbm_select_swaps(lbm_handle h, const float* drho, const float* ux, const float* uy,
                            int32_t n_swap, int32_t* fluid_idx_out, int32_t* solid_idx_out,
                            int32_t* n_out) {
  if (!h || !drho || !ux || !uy || !n_out || (n_swap > 0 && (!fluid_idx_out || !solid_idx_out)))
    return fail(LBM_ERR_ARG, "NULL argument");
  if (n_swap < 0) return fail(LBM_ERR_ARG, "n_swap must be >= 0");
  Engine* E = h->e;
  Member* m = E->m[0];
  const size_t nx = m->nx, ny = m->ny;
  // the member's view with its fields replaced by copies of the given ones
  float* tmp = nullptr;
  LatticeView* vdev = nullptr;
  CU(dev_malloc(reinterpret_cast<void**>(&tmp), 3 * m->plane * sizeof(float)));
  if (dev_malloc(reinterpret_cast<void**>(&vdev), sizeof(LatticeView)) != cudaSuccess) {
    cudaFree(tmp);
    return fail(LBM_ERR_OOM, "cudaMalloc(view)");
  }
  LatticeView v = m->view;
  v.drho = tmp;
  v.ux = tmp + m->plane;
  v.uy = tmp + 2 * m->plane;
  v.sel_off = 0;
  v.word_off = 0;
  lbm_status st = LBM_OK;
  auto step = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == LBM_OK) st = fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  step(cudaMemsetAsync(tmp, 0, 3 * m->plane * sizeof(float), E->stream), "memset");
  const float* srcs[3] = {drho, ux, uy};
  for (int k = 0; k < 3; ++k)
    step(xfer2d(tmp + k * m->plane, (size_t)m->pitch * 4, srcs[k], nx * 4, nx * 4, ny,
                           cudaMemcpyDefault, E->stream), "copy field");
  step(xfer(vdev, &v, sizeof(v), cudaMemcpyHostToDevice, E->stream), "view");
  E->h_nswap[0] = n_swap;
  step(xfer(E->n_swap_dev.p, E->h_nswap, sizeof(int), cudaMemcpyHostToDevice, E->stream), "n_swap");
  // one lattice: E->word_off is {0, words}
  step(launch_oc_select(vdev, static_cast<const int*>(E->L.word_off.p), 1, E->L.total_words,
                                static_cast<const int*>(E->n_swap_dev.p), E->oc, E->stream), "select");
  step(xfer(E->h_info, E->oc.info, 8 * sizeof(int), cudaMemcpyDeviceToHost, E->stream), "info");
  step(cudaStreamSynchronize(E->stream), "sync");
  const int n = st == LBM_OK ? E->h_info[0] : 0;
  if (st == LBM_OK && n > 0) {
    step(xfer(fluid_idx_out, E->oc.sel_f, n * sizeof(int), cudaMemcpyDefault, E->stream), "out");
    step(xfer(solid_idx_out, E->oc.sel_s, n * sizeof(int), cudaMemcpyDefault, E->stream), "out");
    step(cudaStreamSynchronize(E->stream), "sync");
  }
  cudaFree(tmp);
  cudaFree(vdev);
  if (st != LBM_OK) return st;
  *n_out = n;
  if (E->h_info[3] != 0) return fail(LBM_ERR_DIVERGED, "a score is NaN");
  return LBM_OK;
}

// ---- batches -------------------------------------------------------------------

lbm_status lbm_batch_create(int32_t n, const lbm_params* params, const uint8_t* const* cell_types,
                            void* cuda_stream, lbm_batch* out) {
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !params || !cell_types) return fail(LBM_ERR_ARG, "need n >= 1, params and cell_types");
  Engine* E = nullptr;
  lbm_status st = engine_create(n, params, cell_types, cuda_stream, &E);
  if (st != LBM_OK) return st;
  *out = new lbm_batch_s{E};
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch b) {
  if (!b) return;
  delete b->e;
  delete b;
}

lbm_status lbm_batch_reset(lbm_batch b) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  return engine_reset(b->e);
}

lbm_status lbm_batch_solve(lbm_batch b, int64_t n_steps, lbm_solve_result* out) {
  if (!b || !out) return fail(LBM_ERR_ARG, "batch or out is NULL");
  return engine_solve(b->e, n_steps, out);
}

lbm_status lbm_batch_optimize_step(lbm_batch b, const int32_t* n_swap, int64_t n_steps, lbm_opt_result* out) {
  if (!b || !n_swap || !out) return fail(LBM_ERR_ARG, "batch, n_swap or out is NULL");
  return engine_optimize(b->e, n_swap, n_steps, out);
}

lbm_status lbm_batch_read_fields(lbm_batch b, int32_t member, uint32_t which, void* dst, size_t dst_bytes,
                                 int dst_is_device) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  (void)dst_is_device;
  return engine_read(b->e, member, which, dst, dst_bytes);
}

lbm_status lbm_batch_kernel_time(lbm_batch b, int reset, double* ms, int64_t* launches, int64_t* fluid_updates) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  return engine_kernel_time(b->e, reset, ms, launches, fluid_updates);
}

lbm_status lbm_batch_step_groups(lbm_batch b, int32_t* n_groups) {
  if (!b || !n_groups) return fail(LBM_ERR_ARG, "batch or output is NULL");
  *n_groups = engine_step_groups(b->e);
  return LBM_OK;
}

lbm_status lbm_batch_step_config(lbm_batch b, int32_t* warps_per_block, int32_t* grid, int32_t* persistent,
                                 int32_t* cells_per_thread, int32_t* stages) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  return engine_step_config(b->e, warps_per_block, grid, persistent, cells_per_thread, stages);
}

lbm_status lbm_batch_set_step_config(lbm_batch b, int32_t warps_per_block, int32_t persistent,
                                     int32_t cells_per_thread, int32_t stages) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  return engine_set_step_config(b->e, warps_per_block, persistent, cells_per_thread, stages);
}

}  // extern "C"
