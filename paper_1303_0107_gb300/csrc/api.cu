// C ABI of the library (include/lbm.h) and the engine behind it.
//
// An engine steps a set of lattices together: each member owns its
// populations, mask and fields; the engine owns one descriptor table, one
// row-segment work-list, one reduction block and one exchange scratch for the
// whole set, so every stage of the loop of Sec. 2.3 (steps 2-5) is one launch
// over all members.  A handle (lbm_create_geometry) is an engine of one
// member, a batch (lbm_batch_create) an engine of many.  Host code only: it
// validates arguments, owns device memory and enqueues the kernels of
// step.cu, worklist.cu, reduce.cu and oc.cu on the engine's stream.  Repeated
// stream-collide pairs are replayed from CUDA graphs captured once per
// engine, after the launch shape has been tuned on the engine's own lattices.
#include <algorithm>
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

static bool autotune_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  return on;
}

}  // namespace lbm

using namespace lbm;

namespace {

constexpr int kGraphPairs[3] = {64, 8, 1};

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

template <class T>
cudaError_t dalloc(std::vector<void*>& allocs, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) {
    allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

// One lattice: its device storage and host description.
struct Member {
  lbm_params p{};
  int nx = 0, ny = 0, pitch = 0, wpr = 0;
  size_t plane = 0;
  std::vector<int> out_start, out_len;
  void* f = nullptr;
  uint32_t *mask_base = nullptr, *mask0_base = nullptr, *mask = nullptr, *mask0 = nullptr;
  size_t mask_bytes = 0;
  float *drho = nullptr, *ux = nullptr, *uy = nullptr, *ux_prev = nullptr, *uy_prev = nullptr;
  float* u_in = nullptr;
  int* d_out = nullptr;  // [LBM_MAX_OUTLETS] starts, then [LBM_MAX_OUTLETS] lengths
  int64_t fluid_cells = 0;
  int64_t steps_done = 0;
  LatticeView view{};
  std::vector<void*> allocs;
  ~Member() {
    for (void* q : allocs) cudaFree(q);
  }
};

// Geometry rules of include/lbm.h; also finds the inlet runs (parabolic
// profile of Sec. 3.3 per run) and the outlet runs.
lbm_status check_and_describe(Member& m, const uint8_t* cells, std::vector<float>& u_in) {
  const int nx = m.nx, ny = m.ny;
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
      u_in[yy] = (float)(4.0 * m.p.u_max * s * (1.0 - s));
    }
  }
  m.out_start.clear();
  m.out_len.clear();
  for (int y = 0; y < ny;) {
    if (cells[(size_t)y * nx + nx - 1]) { ++y; continue; }
    const int y_lo = y;
    while (y < ny && !cells[(size_t)y * nx + nx - 1]) ++y;
    m.out_start.push_back(y_lo);
    m.out_len.push_back(y - y_lo);
  }
  if (m.out_start.empty()) return fail(LBM_ERR_GEOMETRY, "no outlet cell in column nx-1");
  if ((int)m.out_start.size() > LBM_MAX_OUTLETS) return fail(LBM_ERR_GEOMETRY, "more than LBM_MAX_OUTLETS outlets");
  return LBM_OK;
}

lbm_status check_params(const lbm_params& p) {
  if (p.nx < 4 || p.ny < 3 || (p.nx % 2) != 0 || (int64_t)p.nx * p.ny >= (int64_t)1 << 31 ||
      p.nx > (32 << kSegWordBits) || p.ny >= (1 << (31 - kSegWordBits)))
    return fail(LBM_ERR_ARG, "nx must be even, 4 <= nx <= 131072, 3 <= ny < 524288, nx*ny < 2^31");
  const size_t pitch = (size_t)(p.nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
  if (9 * pitch * (size_t)p.ny >= ((size_t)1 << 31))
    return fail(LBM_ERR_ARG, "lattice too large: 9 * ny * pitch must stay below 2^31 elements");
  if (!(p.tau > 0.5) || !std::isfinite(p.tau) || !std::isfinite(p.rho0) || !(p.rho0 > 0) ||
      !std::isfinite(p.u_max))
    return fail(LBM_ERR_ARG, "tau must be > 1/2, rho0 > 0, u_max finite");
  if (p.outlet != LBM_OUT_CONST_RHO && p.outlet != LBM_OUT_NEUMANN) return fail(LBM_ERR_ARG, "outlet rule");
  if (p.precision < LBM_F32 || p.precision > LBM_F16_SHIFTED) return fail(LBM_ERR_ARG, "precision");
  if (p.reinit != LBM_REINIT_WARM && p.reinit != LBM_REINIT_COLD) return fail(LBM_ERR_ARG, "reinit");
  if (p.residual_every < 0 || (p.residual_every % 2) != 0) return fail(LBM_ERR_ARG, "residual_every must be even");
  if (p.ports != LBM_PORTS_REGULARIZED && p.ports != LBM_PORTS_ZOU_HE) return fail(LBM_ERR_ARG, "ports");
  return LBM_OK;
}

// Allocate one member's storage and upload its cell map (packed on the device).
lbm_status member_create(const lbm_params& p, const uint8_t* cells, uint8_t* cells_dev, cudaStream_t stream,
                         Member** out) {
  *out = nullptr;
  lbm_status st = check_params(p);
  if (st != LBM_OK) return st;
  Member* m = new Member();
  m->p = p;
  m->nx = p.nx;
  m->ny = p.ny;
  m->pitch = (p.nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
  m->wpr = (p.nx + 31) / 32;
  m->plane = (size_t)m->ny * m->pitch;
  std::vector<float> u_in;
  st = check_and_describe(*m, cells, u_in);
  if (st != LBM_OK) {
    delete m;
    return st;
  }
#define CUM(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      delete m;                                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                    \
  } while (0)
  const size_t sb = storage_bytes(p.precision);
  CUM(dalloc(m->allocs, &m->f, 9 * m->plane * sb));
  m->mask_bytes = (size_t)mask_alloc_words(m->wpr, m->ny) * 4;
  CUM(dalloc(m->allocs, &m->mask_base, m->mask_bytes));
  CUM(dalloc(m->allocs, &m->mask0_base, m->mask_bytes));
  for (float** a : {&m->drho, &m->ux, &m->uy, &m->ux_prev, &m->uy_prev})
    CUM(dalloc(m->allocs, a, m->plane * 4));
  CUM(dalloc(m->allocs, &m->u_in, (size_t)m->ny * 4));
  CUM(dalloc(m->allocs, &m->d_out, 2 * LBM_MAX_OUTLETS * 4));
  m->mask = m->mask_base + mask_origin(m->wpr);
  m->mask0 = m->mask0_base + mask_origin(m->wpr);
  CUM(cudaMemsetAsync(m->mask_base, 0xff, m->mask_bytes, stream));  // padding = wall
  CUM(cudaMemsetAsync(m->mask0_base, 0xff, m->mask_bytes, stream));
  std::vector<int> outs(2 * LBM_MAX_OUTLETS, 0);
  std::copy(m->out_start.begin(), m->out_start.end(), outs.begin());
  std::copy(m->out_len.begin(), m->out_len.end(), outs.begin() + LBM_MAX_OUTLETS);
  // pageable sources: each call returns once its source has been staged
  CUM(cudaMemcpyAsync(m->u_in, u_in.data(), (size_t)m->ny * 4, cudaMemcpyHostToDevice, stream));
  CUM(cudaMemcpyAsync(m->d_out, outs.data(), outs.size() * 4, cudaMemcpyHostToDevice, stream));
  CUM(cudaMemcpyAsync(cells_dev, cells, (size_t)m->nx * m->ny, cudaMemcpyHostToDevice, stream));
  CUM(launch_pack_mask(cells_dev, m->nx, m->ny, m->wpr, m->mask0, stream));
  CUM(cudaStreamSynchronize(stream));  // cells_dev is reused by the next member
#undef CUM
  LatticeView& v = m->view;
  std::memset(&v, 0, sizeof(v));
  v.f = m->f;
  v.mask = m->mask;
  v.drho = m->drho;
  v.ux = m->ux;
  v.uy = m->uy;
  v.ux_prev = m->ux_prev;
  v.uy_prev = m->uy_prev;
  v.u_in = m->u_in;
  v.out_start = m->d_out;
  v.out_len = m->d_out + LBM_MAX_OUTLETS;
  v.plane = (long long)m->plane;
  v.f_elems = 9 * (long long)m->plane;
  v.rho0d = p.rho0;
  v.mu = p.rho0 * ((p.tau - 0.5) / 3.0);
  v.nx = m->nx;
  v.ny = m->ny;
  v.pitch = m->pitch;
  v.wpr = m->wpr;
  v.omega = (float)(1.0 / p.tau);
  v.rho0 = (float)p.rho0;
  v.outlet_rule = p.outlet;
  v.port_scheme = p.ports;
  v.n_outlets = (int)m->out_start.size();
  *out = m;
  return LBM_OK;
}

}  // namespace

// A set of lattices stepped together.
struct Engine {
  int precision = LBM_F32;
  int residual_every = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  std::vector<Member*> m;
  int n = 0;

  LatticeView* views = nullptr;  // [n]
  int* word_off = nullptr;       // [n + 1] all words (rows 0..ny-1)
  int* seg_word_off = nullptr;   // [n + 1] interior-row words
  int total_words = 0, total_seg_words = 0;
  long long total_cells = 0;
  SegRef* segs = nullptr;
  int* n_segs = nullptr;
  int* seg_scratch = nullptr;
  double* partials = nullptr;
  double* result = nullptr;
  unsigned long long* fluid_dev = nullptr;
  int* n_swap_dev = nullptr;
  OcScratch oc{};
  uint8_t* cells_dev = nullptr;  // largest member's cells
  float* dense_f = nullptr;

  double* h_result = nullptr;  // pinned [n * kResultDoubles]
  int* h_info = nullptr;       // pinned [8 n]
  unsigned long long* h_count = nullptr;  // pinned [n]
  int* h_nswap = nullptr;      // pinned [n]

  cudaGraphExec_t graphs[3] = {nullptr, nullptr, nullptr};
  StepConfig step{kStepWarps, 1};
  bool tuned = false;
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  double step_ms = 0.0;
  int64_t step_launches = 0, fluid_updates = 0;
  bool solved = false;
  std::vector<void*> allocs;

  ~Engine() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& g : graphs)
      if (g) cudaGraphExecDestroy(g);
    for (Member* x : m) delete x;
    for (void* q : allocs) cudaFree(q);
    if (h_result) cudaFreeHost(h_result);
    if (h_info) cudaFreeHost(h_info);
    if (h_count) cudaFreeHost(h_count);
    if (h_nswap) cudaFreeHost(h_nswap);
    if (ev_begin) cudaEventDestroy(ev_begin);
    if (ev_end) cudaEventDestroy(ev_end);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

struct lbm_handle_s {
  Engine* e;
};
struct lbm_batch_s {
  Engine* e;
};

namespace {

// With LBM_DEBUG_SYNC=1: wait for the work just enqueued and name it on failure.
#define DEBUG_SYNC(E, what)                                                              \
  do {                                                                                   \
    if (debug_sync() && !t_capturing) {                                                  \
      cudaError_t e_ = cudaStreamSynchronize((E)->stream);                               \
      if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    }                                                                                    \
  } while (0)

lbm_status launch_pair(Engine* E, int moments) {
  // moments: 0 none, 1 into drho/ux/uy, 2 into drho/ux_prev/uy_prev
  CU(launch_stream_collide(E->precision, 0, 0, E->views, E->segs, E->n_segs, E->step, E->stream));
  DEBUG_SYNC(E, "stream-collide phase A");
  CU(launch_stream_collide(E->precision, 1, moments, E->views, E->segs, E->n_segs, E->step, E->stream));
  DEBUG_SYNC(E, "stream-collide phase B");
  return LBM_OK;
}

lbm_status ensure_graph(Engine* E, int which) {
  if (E->graphs[which]) return LBM_OK;
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(E->stream, cudaStreamCaptureModeThreadLocal));
  t_capturing = true;
  lbm_status st = LBM_OK;
  for (int k = 0; k < kGraphPairs[which] && st == LBM_OK; ++k) st = launch_pair(E, 0);
  t_capturing = false;
  cudaError_t e = cudaStreamEndCapture(E->stream, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&E->graphs[which], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status run_plain_pairs(Engine* E, int64_t pairs) {
  if (debug_sync()) {
    for (int64_t k = 0; k < pairs; ++k) {
      lbm_status st = launch_pair(E, 0);
      if (st != LBM_OK) return st;
    }
    return LBM_OK;
  }
  for (int which = 0; which < 3 && pairs > 0; ++which) {
    const int64_t chunk = kGraphPairs[which];
    const int64_t reps = pairs / chunk;
    if (reps == 0) continue;
    lbm_status st = ensure_graph(E, which);
    if (st != LBM_OK) return st;
    for (int64_t r = 0; r < reps; ++r) {
      CU(cudaGraphLaunch(E->graphs[which], E->stream));
      count_launches(2 * chunk);
    }
    pairs -= reps * chunk;
  }
  return LBM_OK;
}

// Work-list and fluid counts after any change of a cell map.
lbm_status rebuild_worklist(Engine* E) {
  CU(launch_build_segments(E->views, E->seg_word_off, E->n, E->total_seg_words, E->seg_scratch, E->segs,
                           E->n_segs, E->stream));
  CU(launch_count_fluid(E->views, E->word_off, E->n, E->total_words, E->fluid_dev, E->stream));
  DEBUG_SYNC(E, "work-list");
  return LBM_OK;
}

// Largest grid for one block shape: every segment its own warp, but never
// more blocks than fit on the device at once.
StepConfig shape(Engine* E, int wpb, int blocks_per_sm_scale) {
  const int bps = stream_collide_blocks_per_sm(E->precision, 0, 0, wpb);
  const long long cap = (long long)E->sm_count * bps * blocks_per_sm_scale;
  const long long need = ((long long)E->total_seg_words + wpb - 1) / wpb;
  StepConfig c;
  c.warps_per_block = wpb;
  c.grid = (int)std::max<long long>(1, std::min(need, cap));
  return c;
}

// Pick the step launch shape by timing candidate shapes on the engine's own
// lattices.  The populations are saved and restored around the trials, and
// every shape computes the same values per cell, so tuning changes no result.
lbm_status autotune(Engine* E) {
  E->tuned = true;
  E->step = shape(E, kStepWarps, 1);
  if (!autotune_enabled() || debug_sync()) return LBM_OK;
  const size_t sb = storage_bytes(E->precision);
  std::vector<void*> backups(E->n, nullptr);
  for (int i = 0; i < E->n; ++i) {
    const size_t bytes = 9 * E->m[i]->plane * sb;
    if (cudaMalloc(&backups[i], bytes) != cudaSuccess) {  // no room: keep the default shape
      for (void* b : backups) cudaFree(b);
      cudaGetLastError();
      return LBM_OK;
    }
    CU(cudaMemcpyAsync(backups[i], E->m[i]->f, bytes, cudaMemcpyDeviceToDevice, E->stream));
  }
  std::vector<StepConfig> cand;
  for (int wpb : {4, 8, 16})
    for (int scale : {1, 2}) {
      StepConfig c = shape(E, wpb, scale);
      bool dup = false;
      for (auto& d : cand) dup |= (d.warps_per_block == c.warps_per_block && d.grid == c.grid);
      if (!dup) cand.push_back(c);
    }
  cudaEvent_t a, b;
  CU(cudaEventCreate(&a));
  CU(cudaEventCreate(&b));
  float best = 1e30f;
  StepConfig best_cfg = E->step;
  lbm_status st = LBM_OK;
  for (int rep = 0; rep < 2 && st == LBM_OK; ++rep) {  // first pass warms up
    for (const StepConfig& c : cand) {
      E->step = c;
      cudaEventRecord(a, E->stream);
      for (int k = 0; k < 16 && st == LBM_OK; ++k) st = launch_pair(E, 0);
      cudaEventRecord(b, E->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) st = fail(LBM_ERR_CUDA, "autotune timing");
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep == 1 && ms < best) {
        best = ms;
        best_cfg = c;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  for (int i = 0; i < E->n; ++i) {
    cudaMemcpyAsync(E->m[i]->f, backups[i], 9 * E->m[i]->plane * sb, cudaMemcpyDeviceToDevice, E->stream);
  }
  cudaStreamSynchronize(E->stream);
  for (void* q : backups) cudaFree(q);
  E->step = best_cfg;
  for (auto& g : E->graphs)  // captured with the previous shape
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return st;
}

lbm_status initial_state(Engine* E) {
  const size_t sb = storage_bytes(E->precision);
  for (Member* m : E->m) {
    CU(cudaMemcpyAsync(m->mask_base, m->mask0_base, m->mask_bytes, cudaMemcpyDeviceToDevice, E->stream));
    CU(cudaMemsetAsync(m->f, 0, 9 * m->plane * sb, E->stream));  // shifted equilibrium at rest: g = 0
    for (float* a : {m->drho, m->ux, m->uy, m->ux_prev, m->uy_prev})
      CU(cudaMemsetAsync(a, 0, m->plane * sizeof(float), E->stream));
    m->steps_done = 0;
  }
  lbm_status st = rebuild_worklist(E);
  if (st != LBM_OK) return st;
  CU(cudaMemcpyAsync(E->h_count, E->fluid_dev, sizeof(unsigned long long) * E->n, cudaMemcpyDeviceToHost,
                     E->stream));
  CU(cudaStreamSynchronize(E->stream));
  for (int i = 0; i < E->n; ++i) E->m[i]->fluid_cells = (int64_t)E->h_count[i];
  E->solved = false;
  return LBM_OK;
}

lbm_status engine_create(int n, const lbm_params* params, const uint8_t* const* cells, void* cuda_stream,
                         Engine** out) {
  *out = nullptr;
  if (n < 1) return fail(LBM_ERR_ARG, "need at least one lattice");
  for (int i = 1; i < n; ++i)
    if (params[i].precision != params[0].precision || params[i].residual_every != params[0].residual_every)
      return fail(LBM_ERR_ARG, "all lattices of a batch share precision and residual_every");
  for (int i = 0; i < n; ++i)
    if (!cells[i]) return fail(LBM_ERR_ARG, "cell_types is NULL");
  Engine* E = new Engine();
  E->precision = params[0].precision;
  E->residual_every = params[0].residual_every;
  E->n = n;
#define CUE(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      delete E;                                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                    \
  } while (0)
  int dev = 0;
  CUE(cudaGetDevice(&dev));
  CUE(cudaDeviceGetAttribute(&E->sm_count, cudaDevAttrMultiProcessorCount, dev));
  if (cuda_stream) {
    E->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    CUE(cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking));
    E->own_stream = true;
  }
  long long max_cells = 0;
  for (int i = 0; i < n; ++i) max_cells = std::max<long long>(max_cells, (long long)params[i].nx * params[i].ny);
  for (int i = 0; i < n; ++i)
    if (check_params(params[i]) != LBM_OK) {
      delete E;
      return LBM_ERR_ARG;
    }
  CUE(dalloc(E->allocs, &E->cells_dev, (size_t)max_cells));
  CUE(dalloc(E->allocs, &E->dense_f, (size_t)max_cells * 4));
  for (int i = 0; i < n; ++i) {
    Member* mb = nullptr;
    lbm_status st = member_create(params[i], cells[i], E->cells_dev, E->stream, &mb);
    if (st != LBM_OK) {
      delete E;
      return st;
    }
    E->m.push_back(mb);
  }
  // set-level layout
  std::vector<int> woff(n + 1, 0), swoff(n + 1, 0);
  long long sel = 0, words = 0, swords = 0;
  for (int i = 0; i < n; ++i) {
    Member* mb = E->m[i];
    mb->view.word_off = (int)words;
    mb->view.seg_word_off = (int)swords;
    mb->view.sel_off = (int)sel;
    words += (long long)mb->ny * mb->wpr;
    swords += (long long)(mb->ny - 2) * mb->wpr;
    sel += sel_capacity(mb->nx, mb->ny);
    E->total_cells += (long long)mb->nx * mb->ny;
    woff[i + 1] = (int)words;
    swoff[i + 1] = (int)swords;
  }
  if (words >= (1ll << 31) || sel >= (1ll << 31) || E->total_cells >= (1ll << 31)) {
    delete E;
    return fail(LBM_ERR_ARG, "batch too large: total cells must stay below 2^31");
  }
  E->total_words = (int)words;
  E->total_seg_words = (int)swords;
  CUE(dalloc(E->allocs, &E->views, sizeof(LatticeView) * n));
  CUE(dalloc(E->allocs, &E->word_off, sizeof(int) * (n + 1)));
  CUE(dalloc(E->allocs, &E->seg_word_off, sizeof(int) * (n + 1)));
  CUE(dalloc(E->allocs, &E->segs, sizeof(SegRef) * std::max(1, E->total_seg_words)));
  CUE(dalloc(E->allocs, &E->n_segs, sizeof(int)));
  CUE(dalloc(E->allocs, &E->seg_scratch, segment_scratch_ints(E->total_seg_words) * sizeof(int)));
  CUE(dalloc(E->allocs, &E->partials, sizeof(double) * 2 * kResidualBlocks * n));
  CUE(dalloc(E->allocs, &E->result, sizeof(double) * kResultDoubles * n));
  CUE(dalloc(E->allocs, &E->fluid_dev, sizeof(unsigned long long) * n));
  CUE(dalloc(E->allocs, &E->n_swap_dev, sizeof(int) * n));
  OcScratch& oc = E->oc;
  CUE(dalloc(E->allocs, &oc.cnt_f, (size_t)words * 4));
  CUE(dalloc(E->allocs, &oc.cnt_s, (size_t)words * 4));
  CUE(dalloc(E->allocs, &oc.off_f, (size_t)(words + 1) * 4));
  CUE(dalloc(E->allocs, &oc.off_s, (size_t)(words + 1) * 4));
  CUE(dalloc(E->allocs, &oc.key_f, (size_t)E->total_cells * 8));
  CUE(dalloc(E->allocs, &oc.key_s, (size_t)E->total_cells * 8));
  CUE(dalloc(E->allocs, &oc.idx_f, (size_t)E->total_cells * 4));
  CUE(dalloc(E->allocs, &oc.idx_s, (size_t)E->total_cells * 4));
  CUE(dalloc(E->allocs, &oc.sel_f, (size_t)sel * 4));
  CUE(dalloc(E->allocs, &oc.sel_s, (size_t)sel * 4));
  CUE(dalloc(E->allocs, &oc.info, (size_t)8 * n * 4));
  CUE(dalloc(E->allocs, &oc.scan_tmp, scan_tmp_ints(words) * 4));
  CUE(cudaMallocHost((void**)&E->h_result, sizeof(double) * kResultDoubles * n));
  CUE(cudaMallocHost((void**)&E->h_info, sizeof(int) * 8 * n));
  CUE(cudaMallocHost((void**)&E->h_count, sizeof(unsigned long long) * n));
  CUE(cudaMallocHost((void**)&E->h_nswap, sizeof(int) * n));
  CUE(cudaEventCreate(&E->ev_begin));
  CUE(cudaEventCreate(&E->ev_end));
  std::vector<LatticeView> vs(n);
  for (int i = 0; i < n; ++i) vs[i] = E->m[i]->view;
  CUE(cudaMemcpyAsync(E->views, vs.data(), sizeof(LatticeView) * n, cudaMemcpyHostToDevice, E->stream));
  CUE(cudaMemcpyAsync(E->word_off, woff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, E->stream));
  CUE(cudaMemcpyAsync(E->seg_word_off, swoff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, E->stream));
#undef CUE
  E->step = shape(E, kStepWarps, 1);
  lbm_status st = initial_state(E);
  if (st != LBM_OK) {
    delete E;
    return st;
  }
  *out = E;
  return LBM_OK;
}

// after the stream has been synchronised: add the steps' device time
void account_steps(Engine* E, int64_t n_steps) {
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, E->ev_begin, E->ev_end) == cudaSuccess) E->step_ms += ms;
  E->step_launches += n_steps;
  for (Member* m : E->m) E->fluid_updates += n_steps * m->fluid_cells;
}

void fill_result(Engine* E, int i, lbm_solve_result* out) {
  const double* r = E->h_result + (size_t)i * kResultDoubles;
  const Member* m = E->m[i];
  std::memset(out, 0, sizeof(*out));
  out->dp = r[0];
  out->m_in = r[1];
  out->residual = r[2];
  out->n_outlets = (int)m->out_start.size();
  out->theta = r[8];
  out->dg = r[9];
  for (int j = 0; j < out->n_outlets; ++j) out->m_out[j] = r[10 + j];
  out->steps_done = m->steps_done;
  out->fluid_cells = m->fluid_cells;
}

// Enqueue n_steps (even) and the reductions; copy the results to pinned host
// memory.  The caller synchronises.
lbm_status enqueue_solve(Engine* E, int64_t n_steps) {
  if (!E->tuned && n_steps >= 256) {
    lbm_status st = autotune(E);
    if (st != LBM_OK) return st;
  }
  const int K = E->residual_every;
  const bool with_res = K >= 2 && (K % 2) == 0 && n_steps >= (int64_t)K + 2;
  lbm_status st;
  CU(cudaEventRecord(E->ev_begin, E->stream));
  if (with_res) {
    if ((st = run_plain_pairs(E, (n_steps - K) / 2 - 1)) != LBM_OK) return st;
    if ((st = launch_pair(E, 2)) != LBM_OK) return st;
    if ((st = run_plain_pairs(E, K / 2 - 1)) != LBM_OK) return st;
  } else {
    if ((st = run_plain_pairs(E, n_steps / 2 - 1)) != LBM_OK) return st;
  }
  if ((st = launch_pair(E, 1)) != LBM_OK) return st;
  CU(cudaEventRecord(E->ev_end, E->stream));
  if (with_res) {
    CU(launch_residual_partials(E->views, E->n, E->partials, E->stream));
    DEBUG_SYNC(E, "residual partials");
  }
  CU(launch_finalize(E->views, E->n, E->partials, with_res ? 1 : 0, E->result, E->stream));
  DEBUG_SYNC(E, "finalize");
  CU(cudaMemcpyAsync(E->h_result, E->result, sizeof(double) * kResultDoubles * E->n, cudaMemcpyDeviceToHost,
                     E->stream));
  return LBM_OK;
}

lbm_status engine_solve(Engine* E, int64_t n_steps, lbm_solve_result* out) {
  if (n_steps < 2 || (n_steps % 2) != 0) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  lbm_status st = enqueue_solve(E, n_steps);
  if (st != LBM_OK) return st;
  CU(cudaStreamSynchronize(E->stream));
  for (Member* m : E->m) m->steps_done += n_steps;
  E->solved = true;
  account_steps(E, n_steps);
  bool bad = false;
  for (int i = 0; i < E->n; ++i) {
    fill_result(E, i, out + i);
    bad |= E->h_result[(size_t)i * kResultDoubles + 7] != 0.0;
  }
  if (bad) return fail(LBM_ERR_DIVERGED, "non-finite pressure drop, flow rate or residual");
  return LBM_OK;
}

lbm_status engine_optimize(Engine* E, const int32_t* n_swap, int64_t n_steps, lbm_opt_result* out) {
  if (n_steps < 2 || (n_steps % 2) != 0) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  for (int i = 0; i < E->n; ++i)
    if (n_swap[i] < 0) return fail(LBM_ERR_ARG, "n_swap must be >= 0");
  if (!E->solved) return fail(LBM_ERR_ARG, "an exchange needs a field: solve first");
  for (int i = 0; i < E->n; ++i) E->h_nswap[i] = n_swap[i];
  CU(cudaMemcpyAsync(E->n_swap_dev, E->h_nswap, sizeof(int) * E->n, cudaMemcpyHostToDevice, E->stream));
  CU(launch_oc_select(E->views, E->word_off, E->n, E->total_words, E->n_swap_dev, E->oc, E->stream));
  DEBUG_SYNC(E, "selection");
  CU(launch_oc_apply(E->precision, E->views, E->n, E->oc, E->stream));
  DEBUG_SYNC(E, "exchange");
  const size_t sb = storage_bytes(E->precision);
  for (Member* m : E->m)
    if (m->p.reinit == LBM_REINIT_COLD) CU(cudaMemsetAsync(m->f, 0, 9 * m->plane * sb, E->stream));
  lbm_status st = rebuild_worklist(E);
  if (st != LBM_OK) return st;
  CU(cudaMemcpyAsync(E->h_info, E->oc.info, sizeof(int) * 8 * E->n, cudaMemcpyDeviceToHost, E->stream));
  CU(cudaMemcpyAsync(E->h_count, E->fluid_dev, sizeof(unsigned long long) * E->n, cudaMemcpyDeviceToHost,
                     E->stream));
  st = enqueue_solve(E, n_steps);
  if (st != LBM_OK) return st;
  CU(cudaStreamSynchronize(E->stream));
  bool nan = false, count_changed = false, bad = false;
  for (int i = 0; i < E->n; ++i) {
    Member* m = E->m[i];
    m->steps_done += n_steps;
    const int64_t before = m->fluid_cells;
    m->fluid_cells = (int64_t)E->h_count[i];
    count_changed |= m->fluid_cells != before;
    nan |= E->h_info[8 * i + 3] != 0;
    bad |= E->h_result[(size_t)i * kResultDoubles + 7] != 0.0;
  }
  account_steps(E, n_steps);
  for (int i = 0; i < E->n; ++i) {
    std::memset(out + i, 0, sizeof(lbm_opt_result));
    out[i].n_swapped = E->h_info[8 * i];
    out[i].fluid_count = E->m[i]->fluid_cells;
    fill_result(E, i, &out[i].solve);
  }
  if (nan) return fail(LBM_ERR_DIVERGED, "a dynamic-pressure or stress score is NaN");
  if (count_changed) return fail(LBM_ERR_CUDA, "fluid cell count changed by the exchange");
  if (bad) return fail(LBM_ERR_DIVERGED, "non-finite pressure drop, flow rate or residual");
  return LBM_OK;
}

lbm_status engine_read(Engine* E, int i, uint32_t which, void* dst, size_t dst_bytes) {
  if (i < 0 || i >= E->n) return fail(LBM_ERR_ARG, "member out of range");
  if (!dst) return fail(LBM_ERR_ARG, "dst is NULL");
  Member* m = E->m[i];
  const size_t nx = m->nx, ny = m->ny, ncell = nx * ny;
  const size_t sb = storage_bytes(E->precision);
  switch (which) {
    case LBM_FIELD_MASK:
      if (dst_bytes < ncell) return fail(LBM_ERR_ARG, "dst too small");
      CU(launch_unpack_mask(m->mask, m->nx, m->ny, m->wpr, E->cells_dev, E->stream));
      CU(cudaMemcpyAsync(dst, E->cells_dev, ncell, cudaMemcpyDefault, E->stream));
      break;
    case LBM_FIELD_RHO:
      if (dst_bytes < ncell * 4) return fail(LBM_ERR_ARG, "dst too small");
      CU(launch_rho_from_drho(m->drho, (float)m->p.rho0, m->mask, m->nx, m->ny, m->pitch, m->wpr, E->dense_f,
                              E->stream));
      CU(cudaMemcpyAsync(dst, E->dense_f, ncell * 4, cudaMemcpyDefault, E->stream));
      break;
    case LBM_FIELD_DRHO:
    case LBM_FIELD_UX:
    case LBM_FIELD_UY: {
      if (dst_bytes < ncell * 4) return fail(LBM_ERR_ARG, "dst too small");
      const float* src = which == LBM_FIELD_DRHO ? m->drho : which == LBM_FIELD_UX ? m->ux : m->uy;
      CU(cudaMemcpy2DAsync(dst, nx * 4, src, (size_t)m->pitch * 4, nx * 4, ny, cudaMemcpyDefault, E->stream));
      break;
    }
    case LBM_FIELD_POPS:
      if (dst_bytes < 9 * ncell * sb) return fail(LBM_ERR_ARG, "dst too small");
      for (int k = 0; k < 9; ++k)
        CU(cudaMemcpy2DAsync(static_cast<char*>(dst) + k * ncell * sb, nx * sb,
                             static_cast<const char*>(m->f) + k * m->plane * sb, (size_t)m->pitch * sb, nx * sb,
                             ny, cudaMemcpyDefault, E->stream));
      break;
    default:
      return fail(LBM_ERR_ARG, "which must be exactly one LBM_FIELD_* value");
  }
  CU(cudaStreamSynchronize(E->stream));
  return LBM_OK;
}

lbm_status engine_kernel_time(Engine* E, int reset, double* ms, int64_t* launches, int64_t* fluid_updates) {
  if (ms) *ms = E->step_ms;
  if (launches) *launches = E->step_launches;
  if (fluid_updates) *fluid_updates = E->fluid_updates;
  if (reset) {
    E->step_ms = 0.0;
    E->step_launches = 0;
    E->fluid_updates = 0;
  }
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
  return initial_state(h->e);
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
    CU(cudaMemcpy2DAsync(static_cast<char*>(m->f) + i * m->plane * sb, (size_t)m->pitch * sb,
                         static_cast<const char*>(pops) + i * ncell * sb, nx * sb, nx * sb, ny,
                         cudaMemcpyDefault, E->stream));
  CU(cudaStreamSynchronize(E->stream));
  return LBM_OK;
}

lbm_status lbm_kernel_time(lbm_handle h, int reset, double* ms, int64_t* launches, int64_t* fluid_updates) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  return engine_kernel_time(h->e, reset, ms, launches, fluid_updates);
}

lbm_status lbm_step_config(lbm_handle h, int32_t* warps_per_block, int32_t* grid) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  if (warps_per_block) *warps_per_block = h->e->step.warps_per_block;
  if (grid) *grid = h->e->step.grid;
  return LBM_OK;
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
  CU(cudaMalloc(&tmp, 3 * m->plane * sizeof(float)));
  if (cudaMalloc(&vdev, sizeof(LatticeView)) != cudaSuccess) {
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
    step(cudaMemcpy2DAsync(tmp + k * m->plane, (size_t)m->pitch * 4, srcs[k], nx * 4, nx * 4, ny,
                           cudaMemcpyDefault, E->stream), "copy field");
  step(cudaMemcpyAsync(vdev, &v, sizeof(v), cudaMemcpyHostToDevice, E->stream), "view");
  E->h_nswap[0] = n_swap;
  step(cudaMemcpyAsync(E->n_swap_dev, E->h_nswap, sizeof(int), cudaMemcpyHostToDevice, E->stream), "n_swap");
  // one lattice: E->word_off is {0, words}
  step(launch_oc_select(vdev, E->word_off, 1, E->total_words, E->n_swap_dev, E->oc, E->stream), "select");
  step(cudaMemcpyAsync(E->h_info, E->oc.info, 8 * sizeof(int), cudaMemcpyDeviceToHost, E->stream), "info");
  step(cudaStreamSynchronize(E->stream), "sync");
  const int n = st == LBM_OK ? E->h_info[0] : 0;
  if (st == LBM_OK && n > 0) {
    step(cudaMemcpyAsync(fluid_idx_out, E->oc.sel_f, n * sizeof(int), cudaMemcpyDefault, E->stream), "out");
    step(cudaMemcpyAsync(solid_idx_out, E->oc.sel_s, n * sizeof(int), cudaMemcpyDefault, E->stream), "out");
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
  return initial_state(b->e);
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

lbm_status lbm_batch_step_config(lbm_batch b, int32_t* warps_per_block, int32_t* grid) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  if (warps_per_block) *warps_per_block = b->e->step.warps_per_block;
  if (grid) *grid = b->e->step.grid;
  return LBM_OK;
}

}  // extern "C"
