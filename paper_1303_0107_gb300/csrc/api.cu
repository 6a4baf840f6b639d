// C ABI of the library (include/lbm.h): lattice handles, the solve loop of
// Sec. 2.3 (steps 2-5) and field access.  Host code only: it validates
// arguments, owns device memory, and enqueues the kernels of step.cu,
// worklist.cu, reduce.cu and oc.cu on the handle's stream.  The repeated
// stream-collide pairs are replayed from CUDA graphs captured once per handle.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbm {

static std::atomic<uint64_t> g_launches{0};
static thread_local bool t_capturing = false;
static thread_local std::string t_last_error;

void count_launches(uint64_t n) {
  if (!t_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

void set_last_error(const std::string& msg) { t_last_error = msg; }

bool debug_sync() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_DEBUG_SYNC");
    return e && e[0] == '1';
  }();
  return on;
}

}  // namespace lbm

using namespace lbm;

namespace {

constexpr int kGraphPairs[3] = {64, 8, 1};
// views[0]: the lattice; views[1]: same, moments into the *_prev fields;
// views[2]: scratch fields of the selection test hook
constexpr int kViews = 3;

lbm_status fail(lbm_status s, const std::string& msg) {
  t_last_error = msg;
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

size_t storage_bytes(int precision) { return precision == LBM_F32 ? 4 : 2; }

}  // namespace

struct lbm_handle_s {
  lbm_params p{};
  int nx = 0, ny = 0, pitch = 0, wpr = 0;
  int n_outlets = 0;
  std::vector<int> outlet_start, outlet_len;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  int grid = 1;
  size_t plane = 0;

  void* f = nullptr;
  uint32_t* mask = nullptr;   // word (0, 0) of the padded mask
  uint32_t* mask0 = nullptr;  // initial cell map, same layout
  uint32_t* mask_base = nullptr;
  uint32_t* mask0_base = nullptr;
  size_t mask_bytes = 0;      // whole padded allocation
  float *drho = nullptr, *ux = nullptr, *uy = nullptr, *ux_prev = nullptr, *uy_prev = nullptr;
  float* u_in = nullptr;
  int *d_outlet_start = nullptr, *d_outlet_len = nullptr;
  LatticeView* views = nullptr;
  LatticeView host_view{};
  SegRef* segs = nullptr;   // row segments holding fluid cells
  int* n_segs = nullptr;
  int* seg_scratch = nullptr;
  double* partials = nullptr;
  double* result = nullptr;
  unsigned long long* fluid_dev = nullptr;
  uint8_t* cells_dev = nullptr;
  float* dense_f = nullptr;
  OcScratch oc{};

  double* h_result = nullptr;  // pinned
  int* h_info = nullptr;       // pinned
  unsigned long long* h_count = nullptr;

  cudaGraphExec_t graphs[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // around the time steps of a solve
  double step_ms = 0.0;
  int64_t step_launches = 0, fluid_updates = 0;

  int64_t steps_done = 0;
  int64_t fluid_cells = 0;
  bool solved = false;
  std::vector<void*> allocations;
};

namespace {

template <class T>
cudaError_t dalloc(lbm_handle h, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) {
    h->allocations.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

// Geometry rules of include/lbm.h; also finds the inlet runs (parabolic
// profile of Sec. 3.3 per run) and the outlet runs.
lbm_status check_and_describe(lbm_handle h, const uint8_t* cells, std::vector<float>& u_in) {
  const int nx = h->nx, ny = h->ny;
  for (int x = 0; x < nx; ++x)
    if (!cells[x] || !cells[(size_t)(ny - 1) * nx + x])
      return fail(LBM_ERR_GEOMETRY, "rows 0 and ny-1 must be solid");
  int n_in = 0;
  for (int y = 0; y < ny; ++y) {
    const uint8_t* r = cells + (size_t)y * nx;
    if (!r[0] && r[1]) return fail(LBM_ERR_GEOMETRY, "inlet cell without a fluid cell behind it");
    if (!r[nx - 1] && r[nx - 2]) return fail(LBM_ERR_GEOMETRY, "outlet cell without a fluid cell before it");
    n_in += r[0] ? 0 : 1;
  }
  if (n_in == 0) return fail(LBM_ERR_GEOMETRY, "no inlet cell in column 0");
  u_in.assign(ny, 0.0f);
  for (int y = 0; y < ny;) {
    if (cells[(size_t)y * nx]) { ++y; continue; }
    const int y_lo = y;
    while (y < ny && !cells[(size_t)y * nx]) ++y;
    const int width = y - y_lo;
    for (int yy = y_lo; yy < y; ++yy) {
      const double s = ((double)(yy - y_lo) + 0.5) / (double)width;
      u_in[yy] = (float)(4.0 * h->p.u_max * s * (1.0 - s));
    }
  }
  h->outlet_start.clear();
  h->outlet_len.clear();
  for (int y = 0; y < ny;) {
    if (cells[(size_t)y * nx + nx - 1]) { ++y; continue; }
    const int y_lo = y;
    while (y < ny && !cells[(size_t)y * nx + nx - 1]) ++y;
    h->outlet_start.push_back(y_lo);
    h->outlet_len.push_back(y - y_lo);
  }
  h->n_outlets = (int)h->outlet_start.size();
  if (h->n_outlets == 0) return fail(LBM_ERR_GEOMETRY, "no outlet cell in column nx-1");
  if (h->n_outlets > LBM_MAX_OUTLETS) return fail(LBM_ERR_GEOMETRY, "more than LBM_MAX_OUTLETS outlets");
  return LBM_OK;
}

lbm_status run_plain_pairs(lbm_handle h, int64_t pairs);

// With LBM_DEBUG_SYNC=1: wait for the work just enqueued and name it on failure.
#define DEBUG_SYNC(h, what)                                                              \
  do {                                                                                   \
    if (debug_sync() && !t_capturing) {                                                  \
      cudaError_t e_ = cudaStreamSynchronize((h)->stream);                               \
      if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    }                                                                                    \
  } while (0)

lbm_status launch_pair(lbm_handle h, int moments_view) {
  // moments_view: -1 none, 0 into the lattice fields, 1 into the *_prev fields
  const int prec = h->p.precision;
  CU(launch_stream_collide(prec, 0, 0, h->views, h->segs, h->n_segs, h->grid, h->stream));
  DEBUG_SYNC(h, "stream-collide phase A");
  const LatticeView* v = moments_view == 1 ? h->views + 1 : h->views;
  CU(launch_stream_collide(prec, 1, moments_view >= 0 ? 1 : 0, v, h->segs, h->n_segs, h->grid,
                           h->stream));
  DEBUG_SYNC(h, moments_view >= 0 ? "stream-collide phase B with moments" : "stream-collide phase B");
  return LBM_OK;
}

lbm_status ensure_graph(lbm_handle h, int which) {
  if (h->graphs[which]) return LBM_OK;
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  t_capturing = true;
  lbm_status st = LBM_OK;
  for (int k = 0; k < kGraphPairs[which] && st == LBM_OK; ++k) st = launch_pair(h, -1);
  t_capturing = false;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graphs[which], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status run_plain_pairs(lbm_handle h, int64_t pairs) {
  if (debug_sync()) {
    for (int64_t k = 0; k < pairs; ++k) {
      lbm_status st = launch_pair(h, -1);
      if (st != LBM_OK) return st;
    }
    return LBM_OK;
  }
  for (int which = 0; which < 3 && pairs > 0; ++which) {
    const int64_t chunk = kGraphPairs[which];
    const int64_t reps = pairs / chunk;
    if (reps == 0) continue;
    lbm_status st = ensure_graph(h, which);
    if (st != LBM_OK) return st;
    for (int64_t r = 0; r < reps; ++r) {
      CU(cudaGraphLaunch(h->graphs[which], h->stream));
      count_launches(2 * chunk);
    }
    pairs -= reps * chunk;
  }
  return LBM_OK;
}

lbm_status rebuild_worklist(lbm_handle h) {
  CU(launch_build_segments(h->mask, h->ny, h->wpr, 0, h->seg_scratch, h->segs, h->n_segs, h->stream));
  CU(launch_count_fluid(h->mask, h->nx, h->ny, h->wpr, h->fluid_dev, h->stream));
  return LBM_OK;
}

lbm_status initial_state(lbm_handle h) {
  const size_t fb = 9 * h->plane * storage_bytes(h->p.precision);
  CU(cudaMemcpyAsync(h->mask_base, h->mask0_base, h->mask_bytes, cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemsetAsync(h->f, 0, fb, h->stream));  // shifted equilibrium at rest: g = 0
  const size_t fl = h->plane * sizeof(float);
  for (float* a : {h->drho, h->ux, h->uy, h->ux_prev, h->uy_prev}) CU(cudaMemsetAsync(a, 0, fl, h->stream));
  lbm_status st = rebuild_worklist(h);
  if (st != LBM_OK) return st;
  CU(cudaMemcpyAsync(h->h_count, h->fluid_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->fluid_cells = (int64_t)*h->h_count;
  h->steps_done = 0;
  h->solved = false;
  return LBM_OK;
}

// after the stream has been synchronised: add the steps' device time
void account_steps(lbm_handle h, int64_t n_steps) {
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, h->ev_begin, h->ev_end) == cudaSuccess) h->step_ms += ms;
  h->step_launches += n_steps;
  h->fluid_updates += n_steps * h->fluid_cells;
}

void fill_result(lbm_handle h, lbm_solve_result* out) {
  const double* r = h->h_result;
  std::memset(out, 0, sizeof(*out));
  out->dp = r[0];
  out->m_in = r[1];
  out->residual = r[2];
  out->n_outlets = h->n_outlets;
  out->theta = r[8];
  out->dg = r[9];
  for (int j = 0; j < h->n_outlets; ++j) out->m_out[j] = r[10 + j];
  out->steps_done = h->steps_done;
  out->fluid_cells = h->fluid_cells;
}

// Enqueue n_steps (even) and the reductions; copy the results to pinned host
// memory.  The caller synchronises.
lbm_status enqueue_solve(lbm_handle h, int64_t n_steps) {
  const int K = h->p.residual_every;
  const bool with_res = K >= 2 && (K % 2) == 0 && n_steps >= (int64_t)K + 2;
  lbm_status st;
  CU(cudaEventRecord(h->ev_begin, h->stream));
  if (with_res) {
    if ((st = run_plain_pairs(h, (n_steps - K) / 2 - 1)) != LBM_OK) return st;
    if ((st = launch_pair(h, 1)) != LBM_OK) return st;
    if ((st = run_plain_pairs(h, K / 2 - 1)) != LBM_OK) return st;
  } else {
    if ((st = run_plain_pairs(h, n_steps / 2 - 1)) != LBM_OK) return st;
  }
  if ((st = launch_pair(h, 0)) != LBM_OK) return st;
  CU(cudaEventRecord(h->ev_end, h->stream));
  if (with_res) {
    CU(launch_residual_partials(h->views, h->ux_prev, h->uy_prev, 0, h->partials, h->stream));
    DEBUG_SYNC(h, "residual partials");
  }
  CU(launch_finalize(h->views, 0, h->d_outlet_start, h->d_outlet_len, h->n_outlets, h->partials,
                     with_res ? 1 : 0, h->result, h->stream));
  DEBUG_SYNC(h, "finalize");
  CU(cudaMemcpyAsync(h->h_result, h->result, kResultDoubles * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  return LBM_OK;
}

}  // namespace

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
  }
  return "unknown status";
}

const char* lbm_last_error(void) { return t_last_error.c_str(); }

uint64_t lbm_kernel_launches(void) { return g_launches.load(); }

double lbm_bytes_per_fluid_update(int32_t precision) {
  return 2.0 * 9.0 * (double)storage_bytes(precision) + 1.0 / 8.0;
}

void lbm_destroy(lbm_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs)
    if (g) cudaGraphExecDestroy(g);
  for (void* p : h->allocations) cudaFree(p);
  if (h->h_result) cudaFreeHost(h->h_result);
  if (h->h_info) cudaFreeHost(h->h_info);
  if (h->h_count) cudaFreeHost(h->h_count);
  if (h->ev_begin) cudaEventDestroy(h->ev_begin);
  if (h->ev_end) cudaEventDestroy(h->ev_end);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

lbm_status lbm_create_geometry(const lbm_params* params, const uint8_t* cell_types, void* cuda_stream,
                               lbm_handle* out) {
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || !cell_types) return fail(LBM_ERR_ARG, "params or cell_types is NULL");
  const lbm_params& p = *params;
  if (p.nx < 4 || p.ny < 3 || (p.nx % 2) != 0 || (int64_t)p.nx * p.ny >= (int64_t)1 << 31 ||
      p.nx > (32 << kSegWordBits) || p.ny >= (1 << (31 - kSegWordBits)))
    return fail(LBM_ERR_ARG, "nx must be even, 4 <= nx <= 131072, 3 <= ny < 524288, nx*ny < 2^31");
  if (!(p.tau > 0.5) || !std::isfinite(p.tau) || !std::isfinite(p.rho0) || !(p.rho0 > 0) ||
      !std::isfinite(p.u_max))
    return fail(LBM_ERR_ARG, "tau must be > 1/2, rho0 > 0, u_max finite");
  if (p.outlet != LBM_OUT_CONST_RHO && p.outlet != LBM_OUT_NEUMANN) return fail(LBM_ERR_ARG, "outlet rule");
  if (p.precision < LBM_F32 || p.precision > LBM_F16_SHIFTED) return fail(LBM_ERR_ARG, "precision");
  if (p.reinit != LBM_REINIT_WARM && p.reinit != LBM_REINIT_COLD) return fail(LBM_ERR_ARG, "reinit");
  if (p.residual_every < 0 || (p.residual_every % 2) != 0) return fail(LBM_ERR_ARG, "residual_every must be even");
  if (p.ports != LBM_PORTS_REGULARIZED && p.ports != LBM_PORTS_ZOU_HE) return fail(LBM_ERR_ARG, "ports");

  lbm_handle h = new lbm_handle_s();
  h->p = p;
  h->nx = p.nx;
  h->ny = p.ny;
  h->pitch = (p.nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
  h->wpr = (p.nx + 31) / 32;
  h->plane = (size_t)h->ny * h->pitch;
  if (9 * h->plane >= ((size_t)1 << 31)) {
    delete h;
    return fail(LBM_ERR_ARG, "lattice too large: 9 * ny * pitch must stay below 2^31 elements");
  }
  std::vector<float> u_in;
  lbm_status st = check_and_describe(h, cell_types, u_in);
  if (st != LBM_OK) {
    delete h;
    return st;
  }
#define CUH(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      lbm_destroy(h);                                                                    \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                    \
  } while (0)
  int dev = 0;
  CUH(cudaGetDevice(&dev));
  CUH(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
  if (cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    CUH(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  const size_t nx = h->nx, ny = h->ny, ncell = nx * ny, nwords = ny * h->wpr;
  const size_t sb = storage_bytes(p.precision);
  CUH(dalloc(h, &h->f, 9 * h->plane * sb));
  h->mask_bytes = (size_t)mask_alloc_words(h->wpr, h->ny) * 4;
  CUH(dalloc(h, &h->mask_base, h->mask_bytes));
  CUH(dalloc(h, &h->mask0_base, h->mask_bytes));
  CUH(cudaMemsetAsync(h->mask_base, 0xff, h->mask_bytes, h->stream));   // padding = wall
  CUH(cudaMemsetAsync(h->mask0_base, 0xff, h->mask_bytes, h->stream));
  h->mask = h->mask_base + mask_origin(h->wpr);
  h->mask0 = h->mask0_base + mask_origin(h->wpr);
  for (float** a : {&h->drho, &h->ux, &h->uy, &h->ux_prev, &h->uy_prev}) CUH(dalloc(h, a, h->plane * 4));
  CUH(dalloc(h, &h->u_in, ny * 4));
  CUH(dalloc(h, &h->d_outlet_start, LBM_MAX_OUTLETS * 4));
  CUH(dalloc(h, &h->d_outlet_len, LBM_MAX_OUTLETS * 4));
  CUH(dalloc(h, &h->views, kViews * sizeof(LatticeView)));
  const size_t nseg_cap = segment_capacity(h->ny, h->wpr);
  CUH(dalloc(h, &h->segs, nseg_cap * sizeof(SegRef)));
  CUH(dalloc(h, &h->n_segs, sizeof(int)));
  CUH(dalloc(h, &h->seg_scratch, segment_scratch_ints(h->ny, h->wpr) * sizeof(int)));
  CUH(dalloc(h, &h->partials, 2 * kResidualBlocks * sizeof(double)));
  CUH(dalloc(h, &h->result, kResultDoubles * sizeof(double)));
  CUH(dalloc(h, &h->fluid_dev, sizeof(unsigned long long)));
  CUH(dalloc(h, &h->cells_dev, ncell));
  CUH(dalloc(h, &h->dense_f, ncell * 4));
  OcScratch& oc = h->oc;
  CUH(dalloc(h, &oc.cnt_f, nwords * 4));
  CUH(dalloc(h, &oc.cnt_s, nwords * 4));
  CUH(dalloc(h, &oc.off_f, (nwords + 1) * 4));
  CUH(dalloc(h, &oc.off_s, (nwords + 1) * 4));
  CUH(dalloc(h, &oc.key_f, ncell * 8));
  CUH(dalloc(h, &oc.key_s, ncell * 8));
  CUH(dalloc(h, &oc.idx_f, ncell * 4));
  CUH(dalloc(h, &oc.idx_s, ncell * 4));
  oc.cap = (int)(ncell / 2 + 1);
  CUH(dalloc(h, &oc.sel_f, (size_t)oc.cap * 4));
  CUH(dalloc(h, &oc.sel_s, (size_t)oc.cap * 4));
  CUH(dalloc(h, &oc.info, 8 * 4));
  CUH(dalloc(h, &oc.scan_tmp, scan_tmp_ints((int)nwords) * 4));
  CUH(cudaMallocHost((void**)&h->h_result, kResultDoubles * sizeof(double)));
  CUH(cudaMallocHost((void**)&h->h_info, 8 * sizeof(int)));
  CUH(cudaMallocHost((void**)&h->h_count, sizeof(unsigned long long)));
  CUH(cudaEventCreate(&h->ev_begin));
  CUH(cudaEventCreate(&h->ev_end));

  // views: [0] lattice, [1] moments into *_prev, [2] hook scratch (filled on use)
  LatticeView v{};
  v.f = h->f;
  v.mask = h->mask;
  v.drho = h->drho;
  v.ux = h->ux;
  v.uy = h->uy;
  v.u_in = h->u_in;
  v.plane = (long long)h->plane;
  v.nx = h->nx;
  v.ny = h->ny;
  v.pitch = h->pitch;
  v.wpr = h->wpr;
  v.omega = (float)(1.0 / p.tau);
  v.rho0 = (float)p.rho0;
  v.outlet_rule = p.outlet;
  v.port_scheme = p.ports;
  v.f_elems = 9 * (long long)h->plane;
  h->host_view = v;
  LatticeView vs[kViews] = {v, v, v};
  vs[1].ux = h->ux_prev;
  vs[1].uy = h->uy_prev;
  CUH(cudaMemcpyAsync(h->views, vs, sizeof(vs), cudaMemcpyHostToDevice, h->stream));
  CUH(cudaMemcpyAsync(h->u_in, u_in.data(), ny * 4, cudaMemcpyHostToDevice, h->stream));
  CUH(cudaMemcpyAsync(h->d_outlet_start, h->outlet_start.data(), h->n_outlets * 4, cudaMemcpyHostToDevice,
                      h->stream));
  CUH(cudaMemcpyAsync(h->d_outlet_len, h->outlet_len.data(), h->n_outlets * 4, cudaMemcpyHostToDevice,
                      h->stream));
  CUH(cudaMemcpyAsync(h->cells_dev, cell_types, ncell, cudaMemcpyHostToDevice, h->stream));
  CUH(launch_pack_mask(h->cells_dev, h->nx, h->ny, h->wpr, h->mask0, h->stream));
#undef CUH
  // enough warps for one segment each where the lattice allows, never more
  // blocks than fit on the device at once (the kernel strides over the list)
  const int bps = stream_collide_blocks_per_sm(p.precision, 0, 0);
  const long long cap = (long long)h->sm_count * bps;
  const long long need = ((long long)nseg_cap + kStepWarps - 1) / kStepWarps;
  h->grid = (int)(need < cap ? need : cap);
  if (h->grid < 1) h->grid = 1;
  st = initial_state(h);
  if (st != LBM_OK) {
    lbm_destroy(h);
    return st;
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_kernel_time(lbm_handle h, int reset, double* ms, int64_t* launches,
                           int64_t* fluid_updates) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  if (ms) *ms = h->step_ms;
  if (launches) *launches = h->step_launches;
  if (fluid_updates) *fluid_updates = h->fluid_updates;
  if (reset) {
    h->step_ms = 0.0;
    h->step_launches = 0;
    h->fluid_updates = 0;
  }
  return LBM_OK;
}

lbm_status lbm_reset(lbm_handle h) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  return initial_state(h);
}

lbm_status lbm_solve(lbm_handle h, int64_t n_steps, lbm_solve_result* out) {
  if (!h || !out) return fail(LBM_ERR_ARG, "handle or out is NULL");
  if (n_steps < 2 || (n_steps % 2) != 0) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  lbm_status st = enqueue_solve(h, n_steps);
  if (st != LBM_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  h->steps_done += n_steps;
  h->solved = true;
  account_steps(h, n_steps);
  fill_result(h, out);
  if (h->h_result[7] != 0.0) return fail(LBM_ERR_DIVERGED, "non-finite pressure drop, flow rate or residual");
  return LBM_OK;
}

lbm_status lbm_optimize_step(lbm_handle h, int32_t n_swap, int64_t n_steps, lbm_opt_result* out) {
  if (!h || !out) return fail(LBM_ERR_ARG, "handle or out is NULL");
  if (n_steps < 2 || (n_steps % 2) != 0) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  if (n_swap < 0) return fail(LBM_ERR_ARG, "n_swap must be >= 0");
  if (!h->solved) return fail(LBM_ERR_ARG, "lbm_optimize_step needs a field: call lbm_solve first");
  const double mu = h->p.rho0 * ((h->p.tau - 0.5) / 3.0);
  CU(launch_oc_select(&h->host_view, h->views, h->p.rho0, mu, n_swap, h->oc, h->stream));
  CU(launch_oc_apply(h->p.precision, h->views, h->mask, h->oc, h->stream));
  if (h->p.reinit == LBM_REINIT_COLD)
    CU(cudaMemsetAsync(h->f, 0, 9 * h->plane * storage_bytes(h->p.precision), h->stream));
  lbm_status st = rebuild_worklist(h);
  if (st != LBM_OK) return st;
  CU(cudaMemcpyAsync(h->h_info, h->oc.info, 8 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaMemcpyAsync(h->h_count, h->fluid_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     h->stream));
  st = enqueue_solve(h, n_steps);
  if (st != LBM_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  h->steps_done += n_steps;
  const int64_t before = h->fluid_cells;
  h->fluid_cells = (int64_t)*h->h_count;
  account_steps(h, n_steps);
  std::memset(out, 0, sizeof(*out));
  out->n_swapped = h->h_info[0];
  out->fluid_count = h->fluid_cells;
  fill_result(h, &out->solve);
  if (h->h_info[3] != 0) return fail(LBM_ERR_DIVERGED, "a dynamic-pressure or stress score is NaN");
  if (h->fluid_cells != before) return fail(LBM_ERR_CUDA, "fluid cell count changed by the exchange");
  if (h->h_result[7] != 0.0) return fail(LBM_ERR_DIVERGED, "non-finite pressure drop, flow rate or residual");
  return LBM_OK;
}

lbm_status lbm_read_fields(lbm_handle h, uint32_t which, void* dst, size_t dst_bytes, int dst_is_device) {
  if (!h || !dst) return fail(LBM_ERR_ARG, "handle or dst is NULL");
  (void)dst_is_device;  // unified addressing: cudaMemcpyDefault handles both
  const size_t nx = h->nx, ny = h->ny, ncell = nx * ny;
  const size_t sb = storage_bytes(h->p.precision);
  switch (which) {
    case LBM_FIELD_MASK:
      if (dst_bytes < ncell) return fail(LBM_ERR_ARG, "dst too small");
      CU(launch_unpack_mask(h->mask, h->nx, h->ny, h->wpr, h->cells_dev, h->stream));
      CU(cudaMemcpyAsync(dst, h->cells_dev, ncell, cudaMemcpyDefault, h->stream));
      break;
    case LBM_FIELD_RHO:
      if (dst_bytes < ncell * 4) return fail(LBM_ERR_ARG, "dst too small");
      CU(launch_rho_from_drho(h->drho, (float)h->p.rho0, h->mask, h->nx, h->ny, h->pitch, h->wpr,
                              h->dense_f, h->stream));
      CU(cudaMemcpyAsync(dst, h->dense_f, ncell * 4, cudaMemcpyDefault, h->stream));
      break;
    case LBM_FIELD_DRHO:
    case LBM_FIELD_UX:
    case LBM_FIELD_UY: {
      if (dst_bytes < ncell * 4) return fail(LBM_ERR_ARG, "dst too small");
      const float* src = which == LBM_FIELD_DRHO ? h->drho : which == LBM_FIELD_UX ? h->ux : h->uy;
      CU(cudaMemcpy2DAsync(dst, nx * 4, src, (size_t)h->pitch * 4, nx * 4, ny, cudaMemcpyDefault, h->stream));
      break;
    }
    case LBM_FIELD_POPS:
      if (dst_bytes < 9 * ncell * sb) return fail(LBM_ERR_ARG, "dst too small");
      for (int i = 0; i < 9; ++i)
        CU(cudaMemcpy2DAsync(static_cast<char*>(dst) + i * ncell * sb, nx * sb,
                             static_cast<const char*>(h->f) + i * h->plane * sb, (size_t)h->pitch * sb,
                             nx * sb, ny, cudaMemcpyDefault, h->stream));
      break;
    default:
      return fail(LBM_ERR_ARG, "which must be exactly one LBM_FIELD_* value");
  }
  CU(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_load_state(lbm_handle h, const void* pops, size_t bytes, int src_is_device) {
  if (!h || !pops) return fail(LBM_ERR_ARG, "handle or pops is NULL");
  (void)src_is_device;
  const size_t nx = h->nx, ny = h->ny, ncell = nx * ny;
  const size_t sb = storage_bytes(h->p.precision);
  if (bytes < 9 * ncell * sb) return fail(LBM_ERR_ARG, "pops too small");
  for (int i = 0; i < 9; ++i)
    CU(cudaMemcpy2DAsync(static_cast<char*>(h->f) + i * h->plane * sb, (size_t)h->pitch * sb,
                         static_cast<const char*>(pops) + i * ncell * sb, nx * sb, nx * sb, ny,
                         cudaMemcpyDefault, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_select_swaps(lbm_handle h, const float* drho, const float* ux, const float* uy,
                            int32_t n_swap, int32_t* fluid_idx_out, int32_t* solid_idx_out,
                            int32_t* n_out) {
  if (!h || !drho || !ux || !uy || !n_out || (n_swap > 0 && (!fluid_idx_out || !solid_idx_out)))
    return fail(LBM_ERR_ARG, "NULL argument");
  if (n_swap < 0) return fail(LBM_ERR_ARG, "n_swap must be >= 0");
  const size_t nx = h->nx, ny = h->ny;
  float* tmp = nullptr;
  CU(cudaMalloc(&tmp, 3 * h->plane * sizeof(float)));
  LatticeView v = h->host_view;
  v.drho = tmp;
  v.ux = tmp + h->plane;
  v.uy = tmp + 2 * h->plane;
  lbm_status st = LBM_OK;
  auto step = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == LBM_OK) st = fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  step(cudaMemsetAsync(tmp, 0, 3 * h->plane * sizeof(float), h->stream), "memset");
  const float* srcs[3] = {drho, ux, uy};
  for (int k = 0; k < 3; ++k)
    step(cudaMemcpy2DAsync(tmp + k * h->plane, (size_t)h->pitch * 4, srcs[k], nx * 4, nx * 4, ny,
                           cudaMemcpyDefault, h->stream), "copy field");
  step(cudaMemcpyAsync(h->views + 2, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream), "view");
  const double mu = h->p.rho0 * ((h->p.tau - 0.5) / 3.0);
  step(launch_oc_select(&v, h->views + 2, h->p.rho0, mu, n_swap, h->oc, h->stream), "select");
  step(cudaMemcpyAsync(h->h_info, h->oc.info, 8 * sizeof(int), cudaMemcpyDeviceToHost, h->stream), "info");
  step(cudaStreamSynchronize(h->stream), "sync");
  int n = st == LBM_OK ? h->h_info[0] : 0;
  if (st == LBM_OK && n > 0) {
    step(cudaMemcpyAsync(fluid_idx_out, h->oc.sel_f, n * sizeof(int), cudaMemcpyDefault, h->stream), "out");
    step(cudaMemcpyAsync(solid_idx_out, h->oc.sel_s, n * sizeof(int), cudaMemcpyDefault, h->stream), "out");
    step(cudaStreamSynchronize(h->stream), "sync");
  }
  cudaFree(tmp);
  if (st != LBM_OK) return st;
  *n_out = n;
  if (h->h_info[3] != 0) return fail(LBM_ERR_DIVERGED, "a score is NaN");
  return LBM_OK;
}

}  // extern "C"
