// Engine: members, set layouts, time-step graphs, autotuning, solve,
// exchange and read-back.  Host code only: it validates arguments, owns
// device memory and enqueues the kernels of step.cu, worklist.cu, reduce.cu
// and oc.cu on the engine's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"

namespace lbm {

static std::atomic<uint64_t> g_launches{0};
thread_local bool t_capturing = false;
thread_local std::string t_last_error;

void count_launches(uint64_t n) {
  if (!t_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
uint64_t launches_total() { return g_launches.load(); }

static std::atomic<uint64_t> g_h2d{0}, g_d2h{0};

namespace {
bool is_host_memory(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

void count_transfer(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  bool from_host = kind == cudaMemcpyHostToDevice || kind == cudaMemcpyHostToHost;
  bool to_host = kind == cudaMemcpyDeviceToHost || kind == cudaMemcpyHostToHost;
  if (kind == cudaMemcpyDefault) {
    from_host = is_host_memory(src);
    to_host = is_host_memory(dst);
  }
  if (from_host && !to_host) g_h2d.fetch_add(bytes, std::memory_order_relaxed);
  if (to_host && !from_host) g_d2h.fetch_add(bytes, std::memory_order_relaxed);
}
}  // namespace

cudaError_t xfer(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t stream) {
  const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, stream);
  if (e == cudaSuccess && kind != cudaMemcpyDeviceToDevice) count_transfer(dst, src, bytes, kind);
  return e;
}

cudaError_t xfer2d(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t height,
                   cudaMemcpyKind kind, cudaStream_t stream) {
  const cudaError_t e = cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, stream);
  if (e == cudaSuccess && kind != cudaMemcpyDeviceToDevice) count_transfer(dst, src, width * height, kind);
  return e;
}

void transfer_bytes(uint64_t* h2d, uint64_t* d2h) {
  if (h2d) *h2d = g_h2d.load();
  if (d2h) *d2h = g_d2h.load();
}

void set_last_error(const std::string& msg) { t_last_error = msg; }

bool debug_sync() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_DEBUG_SYNC");
    return e && e[0] == '1';
  }();
  return on;
}

// LBM_PERSISTENT=0 keeps the persistent step kernel out of the tuner's candidates.
bool persistent_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_PERSISTENT");
    return !(e && e[0] == '0');
  }();
  return on;
}

// LBM_RESIDENT=0 keeps the on-chip resident steps out of the tuner's candidates.
bool resident_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_RESIDENT");
    return !(e && e[0] == '0');
  }();
  return on;
}

bool autotune_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  return on;
}

static std::atomic<int> g_barrier_timeout{0};
void set_barrier_timeout_test(int on) { g_barrier_timeout.store(on ? 1 : 0); }
int barrier_timeout_test() { return g_barrier_timeout.load(); }

// Test hook for the failure paths: the allocation that brings the countdown
// from 0 to -1 fails as if the device were full.
static std::atomic<int64_t> g_fail_after{-1};

void set_alloc_failure(int64_t after) { g_fail_after.store(after < 0 ? -1 : after); }

cudaError_t dev_malloc(void** p, size_t bytes) {
  int64_t v = g_fail_after.load();
  while (v >= 0 && !g_fail_after.compare_exchange_weak(v, v - 1)) {
  }
  if (v == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

lbm_status fail(lbm_status s, const std::string& msg) {
  t_last_error = msg;
  return s;
}

size_t storage_bytes(int precision) { return precision == LBM_F32 ? 4 : 2; }

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

// With LBM_DEBUG_SYNC=1: wait for the work just enqueued and name it on failure.
#define DEBUG_SYNC(E, what)                                                              \
  do {                                                                                   \
    if (debug_sync() && !t_capturing) {                                                  \
      cudaError_t e_ = cudaStreamSynchronize((E)->stream);                               \
      if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    }                                                                                    \
  } while (0)

namespace {

// Pairs per captured step graph: a programmatic launch overlaps its
// predecessor only within one graph, so long solves run in few, large graphs.
constexpr int kGraphPairs[4] = {512, 64, 8, 1};
// Untuned launch shape: kStepWarps warps per block, the grid twice the blocks
// resident at once (the tuner's usual choice; it leaves the tail of a step
// to blocks that start as the first ones finish).
constexpr int kDefaultGridScale = 2;
constexpr size_t kAlign = 256;
#ifdef LBM_CHECK_BOUNDS
constexpr size_t kCanaryBytes = 256;
#else
constexpr size_t kCanaryBytes = 0;
#endif
constexpr unsigned char kCanaryByte = 0xA5;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Sub-arrays of a member's allocation, as byte offsets.  The bounds-checked
// build puts a canary block (kCanaryBytes of kCanaryByte) on each side of
// the population planes and checks both after every solve.
struct SlabPlan {
  size_t canary_lo, f, canary_hi, mask, mask0, fields, u_in, d_out, cells, total;
};

SlabPlan plan_slab(const lbm_params& p) {
  const size_t pitch = (size_t)(p.nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
  const size_t plane = pitch * (size_t)p.ny;
  const size_t wpr = (size_t)(p.nx + 31) / 32;
  const size_t mask_bytes = (size_t)mask_alloc_words((int)wpr, p.ny) * 4;
  SlabPlan s{};
  size_t o = 0;
  s.canary_lo = o; o += kCanaryBytes;
  s.f = o;      o += align_up(9 * plane * storage_bytes(p.precision));
  s.canary_hi = o; o += kCanaryBytes;
  s.mask = o;   o += align_up(mask_bytes);
  s.mask0 = o;  o += align_up(mask_bytes);
  s.fields = o; o += 5 * align_up(plane * 4);  // drho, ux, uy, ux_prev, uy_prev
  s.u_in = o;   o += align_up((size_t)p.ny * 4);
  s.d_out = o;  o += align_up(2 * LBM_MAX_OUTLETS * 4);
  s.cells = o;  o += align_up((size_t)p.nx * p.ny);
  s.total = o;
  return s;
}

// Geometry rules of include/lbm.h; also finds the inlet runs (parabolic
// profile of Sec. 3.3 per run) and the outlet runs.
lbm_status check_and_describe(Member& m, const uint8_t* cells, std::vector<float>& u_in) {
  const int nx = m.nx, ny = m.ny;
  for (int x = 0; x < nx; ++x)
    if ((!m.p.mirror && !cells[x]) || !cells[(size_t)(ny - 1) * nx + x])
      return fail(LBM_ERR_GEOMETRY, "rows 0 and ny-1 must be solid (row 0 may be fluid next to a symmetry plane)");
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
    // a run touching the symmetry plane is half of a run twice as wide centred on it
    const bool half = m.p.mirror && y_lo == 0;
    const int lo = half ? -width : y_lo, w = half ? 2 * width : width;
    for (int yy = y_lo; yy < y; ++yy) {
      const double s = ((double)(yy - lo) + 0.5) / (double)w;
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

// Offsets and views of a member list, uploaded into the layout's buffers.
lbm_status layout_build(SetLayout& S, const std::vector<Member*>& ms, cudaStream_t stream) {
  ++S.gen;
  const int n = (int)ms.size();
  S.n = n;
  S.h_views.resize(std::max(1, n));
  S.h_woff.assign(n + 1, 0);
  S.h_swoff.assign(n + 1, 0);
  long long words = 0, swords = 0, sel = 0, cells = 0;
  for (int i = 0; i < n; ++i) {
    const Member* mb = ms[i];
    LatticeView v = mb->view;
    v.word_off = (int)words;
    v.seg_word_off = (int)swords;
    v.sel_off = (int)sel;
    S.h_views[i] = v;
    words += (long long)mb->ny * mb->wpr;
    swords += (long long)(mb->ny - 1 - first_step_row(mb->view)) * mb->wpr;
    sel += sel_capacity(mb->nx, mb->ny);
    cells += (long long)mb->nx * mb->ny;
    S.h_woff[i + 1] = (int)std::min<long long>(words, INT32_MAX);
    S.h_swoff[i + 1] = (int)std::min<long long>(swords, INT32_MAX);
  }
  if (words >= (1ll << 31) || sel >= (1ll << 31) || cells >= (1ll << 31))
    return fail(LBM_ERR_ARG, "set too large: total cells must stay below 2^31");
  S.total_words = (int)words;
  S.total_seg_words = (int)swords;
  S.total_sel = sel;
  S.total_cells = cells;
  CU(S.views.reserve(sizeof(LatticeView) * std::max(1, n)));
  CU(S.word_off.reserve(sizeof(int) * (n + 1)));
  CU(S.seg_word_off.reserve(sizeof(int) * (n + 1)));
  if (n > 0)
    CU(xfer(S.views.p, S.h_views.data(), sizeof(LatticeView) * n, cudaMemcpyHostToDevice, stream));
  CU(xfer(S.word_off.p, S.h_woff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, stream));
  CU(xfer(S.seg_word_off.p, S.h_swoff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, stream));
  return LBM_OK;
}

// Exchange scratch for a layout, carved from one growing buffer.
lbm_status reserve_oc(Engine* E, const SetLayout& X) {
  const size_t words = (size_t)X.total_words, cells = (size_t)X.total_cells, sel = (size_t)X.total_sel;
  size_t o = 0;
  size_t off[12];
  const size_t sz[12] = {words * 4,     words * 4,     (words + 1) * 4, (words + 1) * 4,
                         cells * 8,     cells * 8,     cells * 4,       cells * 4,
                         sel * 4,       sel * 4,       8 * (size_t)std::max(1, X.n) * 4,
                         scan_tmp_ints((long long)words) * 4};
  for (int k = 0; k < 12; ++k) {
    off[k] = o;
    o += align_up(std::max<size_t>(sz[k], 16));
  }
  CU(E->oc_buf.reserve(o));
  char* b = static_cast<char*>(E->oc_buf.p);
  OcScratch& s = E->oc;
  s.cnt_f = reinterpret_cast<int*>(b + off[0]);
  s.cnt_s = reinterpret_cast<int*>(b + off[1]);
  s.off_f = reinterpret_cast<int*>(b + off[2]);
  s.off_s = reinterpret_cast<int*>(b + off[3]);
  s.key_f = reinterpret_cast<unsigned long long*>(b + off[4]);
  s.key_s = reinterpret_cast<unsigned long long*>(b + off[5]);
  s.idx_f = reinterpret_cast<int*>(b + off[6]);
  s.idx_s = reinterpret_cast<int*>(b + off[7]);
  s.sel_f = reinterpret_cast<int*>(b + off[8]);
  s.sel_s = reinterpret_cast<int*>(b + off[9]);
  s.info = reinterpret_cast<int*>(b + off[10]);
  s.scan_tmp = reinterpret_cast<int*>(b + off[11]);
  return LBM_OK;
}

lbm_status launch_pair(Engine* E, int moments) {
  // moments: 0 none, 1 into drho/ux/uy, 2 into drho/ux_prev/uy_prev
  const LatticeView* views = static_cast<const LatticeView*>(E->L.views.p);
  const SegRef* segs = static_cast<const SegRef*>(E->segs.p);
  const int* n_segs = static_cast<const int*>(E->n_segs.p);
  if (E->step.persistent == 3) {  // compacted fluid-cell tasks (the list is built before any capture)
    const CellRef* cells = static_cast<const CellRef*>(E->cell_list.p);
    const int* cpre = static_cast<const int*>(E->cell_scan.p) + std::max(1, E->L.total_seg_words);
    CU(launch_stream_collide_cells(E->precision, 0, 0, views, cells, n_segs, cpre, E->step, E->stream));
    DEBUG_SYNC(E, "stream-collide phase A (cell tasks)");
    // staging pays in the shifted phase only (measured): the local phase loads directly
    StepConfig local = E->step;
    local.stages = 0;
    CU(launch_stream_collide_cells(E->precision, 1, moments, views, cells, n_segs, cpre, local, E->stream));
    DEBUG_SYNC(E, "stream-collide phase B (cell tasks)");
    return LBM_OK;
  }
  if (E->step.persistent == 4) {  // paired tasks (the list is built before any capture)
    const SegRef* tasks = static_cast<const SegRef*>(E->pair_list.p);
    const int* n_tasks = static_cast<const int*>(E->pair_scan.p) + 2 * (size_t)std::max(1, E->L.total_seg_words);
    // one lattice: its view by value (a graph captured with it is keyed by the layout build)
    const LatticeView* one = E->n() == 1 ? &E->L.h_views[0] : nullptr;
    CU(launch_stream_collide_pairs(E->precision, 0, 0, views, one, tasks, n_tasks, E->step, E->stream));
    DEBUG_SYNC(E, "stream-collide phase A (paired tasks)");
    CU(launch_stream_collide_pairs(E->precision, 1, moments, views, one, tasks, n_tasks, E->step, E->stream));
    DEBUG_SYNC(E, "stream-collide phase B (paired tasks)");
    return LBM_OK;
  }
  CU(launch_stream_collide(E->precision, 0, 0, views, segs, n_segs, E->step, E->stream));
  DEBUG_SYNC(E, "stream-collide phase A");
  CU(launch_stream_collide(E->precision, 1, moments, views, segs, n_segs, E->step, E->stream));
  DEBUG_SYNC(E, "stream-collide phase B");
  return LBM_OK;
}

void drop_graphs(Engine* E) {
  for (auto& g : E->graphs)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// A captured graph is valid while the buffers and the launch shape it was
// captured with are unchanged.
lbm_status ensure_graph(Engine* E, int which) {
  const bool cells = E->step.persistent == 3, paired = E->step.persistent == 4;
  const void* key[6] = {E->L.views.p, cells ? E->cell_list.p : paired ? E->pair_list.p : E->segs.p, E->n_segs.p,
                        reinterpret_cast<const void*>((intptr_t)E->step.persistent << 56 |
                                                      (intptr_t)E->step.stages << 52 |
                                                      (intptr_t)E->step.cells_per_thread << 48 |
                                                      (intptr_t)E->step.warps_per_block << 32 |
                                                      (intptr_t)(uint32_t)E->step.grid),
                        cells ? E->cell_scan.p : paired ? E->pair_scan.p : nullptr,
                        reinterpret_cast<const void*>((uintptr_t)E->L.gen)};
  if (!std::equal(key, key + 6, E->graph_key)) {
    drop_graphs(E);
    std::copy(key, key + 6, E->graph_key);
  }
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

lbm_status run_persistent(Engine* E, int64_t pairs) {
  // the barrier counter counts 2 * pairs * grid arrivals per launch: keep it below 2^32
  const int64_t max_pairs = std::max<int64_t>(1, ((int64_t)1 << 31) / std::max(1, E->step.grid) - 1);
  while (pairs > 0) {
    const int64_t k = std::min(pairs, max_pairs);
    CU(launch_stream_collide_persistent(E->precision, static_cast<const LatticeView*>(E->L.views.p),
                                        static_cast<const SegRef*>(E->segs.p),
                                        static_cast<const int*>(E->n_segs.p), (int)k, E->step,
                                        static_cast<StepBarrier*>(E->bar.p), E->stream));
    E->bar_used = true;
    pairs -= k;
  }
  return LBM_OK;
}

// One resident launch of n_steps steps (moments at the last step and, when
// mom_prev >= 0, into the *_prev fields at that step).
lbm_status run_resident(Engine* E, int64_t n_steps, int mom_prev) {
  if (n_steps < 1) return LBM_OK;
  if (n_steps >= (int64_t)1 << 30) return fail(LBM_ERR_ARG, "resident steps: at most 2^30 steps per solve");
  if ((uint64_t)E->halo_epoch + (uint64_t)n_steps + 2 >= (1ull << 32)) {  // tags would wrap: start afresh
    CU(cudaMemsetAsync(E->halo.p, 0, E->halo.cap, E->stream));
    E->halo_epoch = 1;
  }
  const unsigned epoch0 = E->halo_epoch;
  E->halo_epoch += (unsigned)n_steps + 1;
  StepBarrier* bar = static_cast<StepBarrier*>(E->bar.p);
  CU(cudaMemsetAsync(&bar->error, 0, sizeof(int), E->stream));
  const int* scratch = static_cast<const int*>(E->seg_scratch.p);
  CU(launch_stream_collide_resident(E->precision, static_cast<const LatticeView*>(E->L.views.p),
                                    static_cast<const SegRef*>(E->segs.p), static_cast<const int*>(E->n_segs.p),
                                    static_cast<const int*>(E->L.seg_word_off.p), scratch,
                                    scratch + E->L.total_seg_words, E->rshape,
                                    static_cast<unsigned long long*>(E->halo.p), E->halo_cap, epoch0, (int)n_steps,
                                    mom_prev, &bar->error, E->stream));
  E->bar_used = true;
  DEBUG_SYNC(E, "resident steps");
  return LBM_OK;
}

StepConfig resident_config(const Engine* E) {
  StepConfig c{};
  c.warps_per_block = E->rshape.warps;
  c.grid = E->rshape.grid;
  c.persistent = 2;
  c.cells_per_thread = 2;
  c.stages = 0;
  c.features = 0;
  return c;
}

lbm_status run_plain_pairs(Engine* E, int64_t pairs) {
  if (E->step.persistent == 2 && !debug_sync()) return run_resident(E, 2 * pairs, -1);
  if (E->step.persistent == 1 && !debug_sync()) return run_persistent(E, pairs);
  if (debug_sync()) {
    for (int64_t k = 0; k < pairs; ++k) {
      lbm_status st = launch_pair(E, 0);
      if (st != LBM_OK) return st;
    }
    return LBM_OK;
  }
  for (int which = 0; which < 4 && pairs > 0; ++which) {
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

// Block shapes the step kernels take: per-phase launches 4, 8, 12, 16 or 32
// warps per block with one cell per thread, 4, 8, 12 or 24 with two; the
// persistent kernel 8 or 16 (8 with two cells per thread).
bool step_shape_allowed(int wpb, int cpt, int persistent) {
  if (persistent == 3) return cpt == 1 && (wpb == 4 || wpb == 8 || wpb == 12 || wpb == 16 || wpb == 32);
  if (persistent == 4) return cpt == 2 && (wpb == 4 || wpb == 8 || wpb == 12 || wpb == 24);
  if (persistent) return wpb == 8 || (wpb == 16 && cpt == 1);
  return cpt == 1 ? (wpb == 4 || wpb == 8 || wpb == 12 || wpb == 16 || wpb == 32)
                  : (wpb == 4 || wpb == 8 || wpb == 12 || wpb == 24);
}

// Launch shape: every segment its own warp, but never more blocks than fit
// on the device at once; a fixed-grid engine always takes the device-sized
// grid, so its captured graphs outlive changes of the member list.
StepConfig shape(Engine* E, int wpb, int blocks_per_sm_scale, int cpt = 1, int stages = 0) {
  const int bps = stream_collide_blocks_per_sm(E->precision, 0, 0, wpb, cpt, stages, E->features);
  const long long cap = (long long)E->sm_count * bps * blocks_per_sm_scale;
  const long long tasks = ((long long)E->L.total_seg_words + cpt - 1) / cpt;
  const long long need = (tasks + wpb - 1) / wpb;
  StepConfig c;
  c.warps_per_block = wpb;
  c.grid = (int)(E->fixed_grid ? cap : std::max<long long>(1, std::min(need, cap)));
  c.persistent = 0;
  c.cells_per_thread = cpt;
  c.stages = stages;
  c.features = E->features;
  return c;
}

// The persistent shape: one cooperative launch per run of pairs, as many
// blocks as are resident at once.
StepConfig persistent_shape(Engine* E, int wpb, int cpt = 1) {
  StepConfig c;
  c.warps_per_block = wpb;
  c.grid = stream_collide_persistent_grid(E->precision, wpb, cpt);
  c.persistent = 1;
  c.cells_per_thread = cpt;
  c.stages = 0;
  c.features = 0;
  return c;
}

// The compacted-task shape: one cell per thread, 32 fluid cells a warp.
StepConfig cells_shape(Engine* E, int wpb, int blocks_per_sm_scale, int stages = 0) {
  const int bps = stream_collide_cells_blocks_per_sm(E->precision, 0, 0, wpb, stages);
  const long long cap = (long long)E->sm_count * bps * blocks_per_sm_scale;
  long long fluid = 0;
  for (const Member* m : E->m) fluid += m->fluid_cells;
  const long long need = ((fluid + 31) / 32 + wpb - 1) / wpb;
  StepConfig c;
  c.warps_per_block = wpb;
  c.grid = (int)(E->fixed_grid ? cap : std::max<long long>(1, std::min(need, cap)));
  c.persistent = 3;
  c.cells_per_thread = 1;
  c.stages = stages;
  c.features = 0;
  return c;
}

// The paired-task shape: two cells a lane on interior windows, one segment
// a warp elsewhere; at most one task per warp of the grid, the segment list
// bounding the tasks.
StepConfig pairs_shape(Engine* E, int wpb, int blocks_per_sm_scale, int stages = 0) {
  const int bps = stream_collide_pairs_blocks_per_sm(E->precision, 0, 0, wpb, stages);
  const long long cap = (long long)E->sm_count * bps * blocks_per_sm_scale;
  const long long need = ((long long)E->L.total_seg_words + wpb - 1) / wpb;
  StepConfig c;
  c.warps_per_block = wpb;
  c.grid = (int)(E->fixed_grid ? cap : std::max<long long>(1, std::min(need, cap)));
  c.persistent = 4;
  c.cells_per_thread = 2;
  c.stages = stages;
  c.features = 0;
  return c;
}

// Pick the step launch shape by timing candidate shapes on the engine's own
// lattices.  The populations are saved and restored around the trials, and
// every shape computes the same values per cell, so tuning changes no result.
// Shapes already tuned in this process, by set signature: device,
// precision, kernel build, member count and each member's size and
// fluid-cell count.  A new
// engine over the same lattices takes the stored shape instead of timing the
// candidates again (LBM_TUNE_CACHE=0 turns the cache off).
std::mutex g_tune_mu;
std::map<std::vector<long long>, StepConfig> g_tune_cache;

bool tune_cache_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_TUNE_CACHE");
    return !(e && e[0] == '0');
  }();
  return on;
}

bool tune_log_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_TUNE_LOG");
    return e && e[0] == '1';
  }();
  return on;
}

std::vector<long long> tune_key(const Engine* E) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<long long> k{dev, E->precision, E->features, E->fixed_grid ? 1 : 0, (long long)E->m.size()};
  for (const Member* m : E->m) {
    k.push_back(m->nx);
    k.push_back(m->ny);
    k.push_back(m->fluid_cells);
  }
  return k;
}

lbm_status autotune(Engine* E) {
  NvtxRange nvtx("lbm_autotune");
  E->tuned = true;
  E->step = shape(E, kStepWarps, kDefaultGridScale);
  if (!autotune_enabled() || debug_sync()) return LBM_OK;
  const std::vector<long long> key = tune_key(E);
  if (tune_cache_enabled()) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      E->step = it->second;
      return LBM_OK;
    }
  }
  const size_t sb = storage_bytes(E->precision);
  const int n = E->n();
  std::vector<void*> backups(n, nullptr);
  for (int i = 0; i < n; ++i) {
    const size_t bytes = 9 * E->m[i]->plane * sb;
    if (dev_malloc(&backups[i], bytes) != cudaSuccess) {  // no room: keep the default shape
      for (void* b : backups) cudaFree(b);
      cudaGetLastError();
      return LBM_OK;
    }
    if (xfer(backups[i], E->m[i]->f, bytes, cudaMemcpyDeviceToDevice, E->stream) != cudaSuccess) {
      for (void* b : backups) cudaFree(b);
      return fail(LBM_ERR_CUDA, "autotune: saving the populations");
    }
  }
  std::vector<StepConfig> cand;
  // the builds with features (collision models, symmetry plane) have one
  // kernel shape: one cell per thread, register loads, one launch per phase
  const bool only_plain = E->features != 0;
  // (one block per SM, the whole register budget: 32 warps with one cell
  // per thread, 24 with two)
  for (int cpt : {1, 2})
    for (int wpb : {4, 8, 12, 16, 24, 32})
      for (int scale : {1, 2, 4}) {
        if (!step_shape_allowed(wpb, cpt, 0) || (cpt == 2 && scale == 4) || (only_plain && cpt == 2) ||
            (wpb >= 24 && scale != 1))
          continue;
        StepConfig c = shape(E, wpb, scale, cpt);
        bool dup = false;
        for (auto& d : cand)
          dup |= (d.warps_per_block == c.warps_per_block && d.grid == c.grid &&
                  d.cells_per_thread == c.cells_per_thread);
        if (!dup) cand.push_back(c);
      }
  if (!only_plain)
    for (int stages : {2, 3})
      for (int wpb : {4, 8}) cand.push_back(shape(E, wpb, 1, 1, stages));
  if (persistent_enabled() && !only_plain && !E->in_group)
    for (int cpt : {1, 2}) {
      StepConfig c = persistent_shape(E, 8, cpt);
      if (c.grid > 0) cand.push_back(c);
    }
  if (cells_eligible(E)) {
    lbm_status cst = ensure_cells(E);
    if (cst != LBM_OK) {
      for (void* b : backups) cudaFree(b);
      return cst;
    }
    for (int stages : {0, 2, 3})
      for (int wpb : {4, 8, 16, 32})
        for (int scale : {1, 2}) {
          if ((wpb == 32 && (scale != 1 || stages)) || (stages && scale != 1)) continue;
          cand.push_back(cells_shape(E, wpb, scale, stages));
        }
  }
  if (pairs_eligible(E)) {
    lbm_status pst = ensure_pairs(E);
    if (pst != LBM_OK) {
      for (void* b : backups) cudaFree(b);
      return pst;
    }
    for (int stages : {0, 2, 3})
      for (int wpb : {4, 8, 12, 24})
        for (int scale : {1, 2}) {
          if (wpb == 24 && scale != 1) continue;
          cand.push_back(pairs_shape(E, wpb, scale, stages));
        }
  }
  if (resident_enabled() && !only_plain && !E->in_group) {
    bool ok = false;
    lbm_status st = resident_prepare(E, &ok);
    if (st != LBM_OK) {
      for (void* b : backups) cudaFree(b);
      return st;
    }
    if (ok) cand.push_back(resident_config(E));
  }
  cudaEvent_t a, b;
  CU(cudaEventCreate(&a));
  CU(cudaEventCreate(&b));
  // Each per-phase candidate runs as a CUDA graph of kTunePairs pairs -- as
  // the solves do -- so that host launch costs do not favour one shape; the
  // persistent candidates are one launch anyway.  One untimed pass, then
  // kTunePasses timed passes over all candidates (slow moments of the device
  // hit every candidate alike); a candidate's time is its fastest pass.
  constexpr int kTunePasses = 5, kTunePairs = 64;
  std::vector<cudaGraphExec_t> tg(cand.size(), nullptr);
  lbm_status st = LBM_OK;
  for (size_t ci = 0; ci < cand.size() && st == LBM_OK; ++ci) {
    if (cand[ci].persistent == 1 || cand[ci].persistent == 2) continue;  // one launch per run: no graph
    E->step = cand[ci];
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(E->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = fail(LBM_ERR_CUDA, "autotune capture");
      break;
    }
    t_capturing = true;
    for (int k = 0; k < kTunePairs && st == LBM_OK; ++k) st = launch_pair(E, 0);
    t_capturing = false;
    const cudaError_t e = cudaStreamEndCapture(E->stream, &g);
    if (st == LBM_OK && (e != cudaSuccess || cudaGraphInstantiate(&tg[ci], g, 0) != cudaSuccess))
      st = fail(LBM_ERR_CUDA, "autotune graph");
    if (g) cudaGraphDestroy(g);
  }
  std::vector<float> t_min(cand.size(), 1e30f);
  for (int rep = 0; rep <= kTunePasses && st == LBM_OK; ++rep) {
    for (size_t ci = 0; ci < cand.size() && st == LBM_OK; ++ci) {
      const StepConfig& c = cand[ci];
      E->step = c;
      cudaEventRecord(a, E->stream);
      if (c.persistent == 2) {
        st = run_resident(E, 2 * kTunePairs, -1);
      } else if (c.persistent == 1) {
        st = run_persistent(E, kTunePairs);
      } else if (cudaGraphLaunch(tg[ci], E->stream) != cudaSuccess) {
        st = fail(LBM_ERR_CUDA, "autotune graph launch");
      } else {
        count_launches(2 * kTunePairs);
      }
      cudaEventRecord(b, E->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) st = fail(LBM_ERR_CUDA, "autotune timing");
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      if ((c.persistent == 1 || c.persistent == 2) && st == LBM_OK) {  // a barrier that gave up would look fast: never pick it
        int err = 0;
        if (cudaMemcpy(&err, &static_cast<StepBarrier*>(E->bar.p)->error, sizeof(int), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
          st = fail(LBM_ERR_CUDA, "autotune barrier flag");
        if (err != 0) st = fail(LBM_ERR_TIMEOUT, "step kernel: a bounded device wait gave up");
      }
      if (rep > 0) t_min[ci] = std::min(t_min[ci], ms);
    }
  }
  for (cudaGraphExec_t g : tg)
    if (g) cudaGraphExecDestroy(g);
  // The fastest candidate, except that a shape with two cells per thread,
  // staged loads or one persistent launch must beat the fastest plain shape
  // (one cell per thread, register loads, per-phase launches) by kMargin:
  // near-ties are within the timing noise, and the plain shape is the one
  // the profiles and the default use.  LBM_TUNE_LOG=1 prints every
  // candidate's time to stderr.
  constexpr float kMargin = 0.985f;
  if (tune_log_enabled())
    for (size_t ci = 0; ci < cand.size(); ++ci)
      std::fprintf(stderr, "lbm tune: wpb %d grid %d cpt %d stages %d persistent %d: %.3f us per step\n",
                   cand[ci].warps_per_block, cand[ci].grid, cand[ci].cells_per_thread, cand[ci].stages,
                   cand[ci].persistent, 1000.0 * t_min[ci] / (2 * kTunePairs));
  StepConfig best_cfg = cand[0], best_plain = cand[0];
  float best = 1e30f, best_p = 1e30f;
  for (size_t ci = 0; ci < cand.size(); ++ci) {
    const StepConfig& c = cand[ci];
    if (t_min[ci] < best) {
      best = t_min[ci];
      best_cfg = c;
    }
    if (!c.persistent && c.cells_per_thread == 1 && c.stages == 0 && t_min[ci] < best_p) {
      best_p = t_min[ci];
      best_plain = c;
    }
  }
  if (best_p < 1e30f && best > kMargin * best_p) best_cfg = best_plain;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  E->bar_used = false;
  for (int i = 0; i < n; ++i)
    xfer(E->m[i]->f, backups[i], 9 * E->m[i]->plane * sb, cudaMemcpyDeviceToDevice, E->stream);
  cudaStreamSynchronize(E->stream);
  for (void* q : backups) cudaFree(q);
  E->step = best_cfg;
  if (st == LBM_OK && tune_cache_enabled()) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_cfg;
  }
  return st;
}

lbm_status ensure_pinned(Engine* E, size_t n) {
  if (n <= E->pinned_n) return LBM_OK;
  const size_t cap = std::max(n, E->pinned_n + E->pinned_n / 2);
  if (E->h_result) cudaFreeHost(E->h_result);
  if (E->h_info) cudaFreeHost(E->h_info);
  if (E->h_count) cudaFreeHost(E->h_count);
  if (E->h_nswap) cudaFreeHost(E->h_nswap);
  if (E->h_bar_error) cudaFreeHost(E->h_bar_error);
  E->h_bar_error = nullptr;
  E->h_result = nullptr;
  E->h_info = nullptr;
  E->h_count = nullptr;
  E->h_nswap = nullptr;
  E->pinned_n = 0;
  CU(cudaMallocHost((void**)&E->h_result, sizeof(double) * kResultDoubles * cap));
  CU(cudaMallocHost((void**)&E->h_info, sizeof(int) * 8 * cap));
  CU(cudaMallocHost((void**)&E->h_count, sizeof(unsigned long long) * cap));
  CU(cudaMallocHost((void**)&E->h_nswap, sizeof(int) * cap));
  CU(cudaMallocHost((void**)&E->h_bar_error, sizeof(int)));
  *E->h_bar_error = 0;
  E->pinned_n = cap;
  return LBM_OK;
}

}  // namespace

// ---- members -------------------------------------------------------------

Member::~Member() {
  if (slab) cudaFree(slab);
}

size_t member_footprint(const lbm_params& p) { return plan_slab(p).total; }

lbm_status check_params(const lbm_params& p) {
  if (p.nx < 4 || p.ny < 3 || (int64_t)p.nx * p.ny >= (int64_t)1 << 31 || p.nx > (32 << kSegWordBits) ||
      p.ny >= (1 << (31 - kSegWordBits)))
    return fail(LBM_ERR_ARG, "need 4 <= nx <= 131072, 3 <= ny < 524288, nx*ny < 2^31");
  // the zero-gradient outlet cell takes the streamed populations of cell
  // nx-2 from the lane to its left: both must lie in one 32-cell segment
  if (p.outlet == LBM_OUT_NEUMANN && (p.nx & 31) == 1)
    return fail(LBM_ERR_ARG, "with the zero-gradient outlet, nx mod 32 must not be 1");
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
  if (p.guard != 0 && p.guard != 1) return fail(LBM_ERR_ARG, "guard must be 0 or 1");
  if (p.collision != LBM_COLLIDE_BGK && p.collision != LBM_COLLIDE_REGULARIZED &&
      p.collision != LBM_COLLIDE_SMAGORINSKY)
    return fail(LBM_ERR_ARG, "collision");
  if (p.mirror != 0 && p.mirror != 1) return fail(LBM_ERR_ARG, "mirror must be 0 or 1");
  if (!std::isfinite(p.c_smag) || p.c_smag < 0) return fail(LBM_ERR_ARG, "c_smag must be finite and >= 0");
  return LBM_OK;
}

lbm_status member_check(const lbm_params& p, const uint8_t* cells) {
  if (!cells) return fail(LBM_ERR_ARG, "cell_types is NULL");
  lbm_status st = check_params(p);
  if (st != LBM_OK) return st;
  Member m;
  m.p = p;
  m.nx = p.nx;
  m.ny = p.ny;
  std::vector<float> u_in;
  return check_and_describe(m, cells, u_in);
}

lbm_status member_create(const lbm_params& p, const uint8_t* cells, cudaStream_t stream, Member** out) {
  *out = nullptr;
  if (!cells) return fail(LBM_ERR_ARG, "cell_types is NULL");
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
  const SlabPlan s = plan_slab(p);
  CUM(dev_malloc(&m->slab, s.total));
  m->slab_bytes = s.total;
  char* b = static_cast<char*>(m->slab);
  m->f = b + s.f;
  m->canary_lo = b + s.canary_lo;
  m->canary_hi = b + s.canary_hi;
  if (kCanaryBytes) {
    CUM(cudaMemsetAsync(m->canary_lo, kCanaryByte, kCanaryBytes, stream));
    CUM(cudaMemsetAsync(m->canary_hi, kCanaryByte, kCanaryBytes, stream));
  }
  m->mask_bytes = (size_t)mask_alloc_words(m->wpr, m->ny) * 4;
  m->mask_base = reinterpret_cast<uint32_t*>(b + s.mask);
  m->mask0_base = reinterpret_cast<uint32_t*>(b + s.mask0);
  const size_t fstride = align_up(m->plane * 4);
  float** fields[5] = {&m->drho, &m->ux, &m->uy, &m->ux_prev, &m->uy_prev};
  for (int k = 0; k < 5; ++k) *fields[k] = reinterpret_cast<float*>(b + s.fields + k * fstride);
  m->u_in = reinterpret_cast<float*>(b + s.u_in);
  m->d_out = reinterpret_cast<int*>(b + s.d_out);
  m->cells = reinterpret_cast<uint8_t*>(b + s.cells);
  m->mask = m->mask_base + mask_origin(m->wpr);
  m->mask0 = m->mask0_base + mask_origin(m->wpr);
  CUM(cudaMemsetAsync(m->mask_base, 0xff, m->mask_bytes, stream));  // padding = wall
  CUM(cudaMemsetAsync(m->mask0_base, 0xff, m->mask_bytes, stream));
  std::vector<int> outs(2 * LBM_MAX_OUTLETS, 0);
  std::copy(m->out_start.begin(), m->out_start.end(), outs.begin());
  std::copy(m->out_len.begin(), m->out_len.end(), outs.begin() + LBM_MAX_OUTLETS);
  // pageable sources: each call returns once its source has been staged
  CUM(xfer(m->u_in, u_in.data(), (size_t)m->ny * 4, cudaMemcpyHostToDevice, stream));
  CUM(xfer(m->d_out, outs.data(), outs.size() * 4, cudaMemcpyHostToDevice, stream));
  CUM(xfer(m->cells, cells, (size_t)m->nx * m->ny, cudaMemcpyHostToDevice, stream));
  CUM(launch_pack_mask(m->cells, m->nx, m->ny, m->wpr, m->mask0, stream));
  if (p.mirror) {  // the padding row below row 0 is row 0's mirror image (the exchange never moves row 0)
    const size_t row = (size_t)mask_stride(m->wpr) * 4;
    CUM(xfer(m->mask0_base, m->mask0_base + mask_stride(m->wpr), row, cudaMemcpyDeviceToDevice, stream));
  }
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
  v.guard = p.guard;
  v.mirror = p.mirror;
  v.collision = p.collision;
  v.c_smag = (float)p.c_smag;
  *out = m;
  return LBM_OK;
}

lbm_status member_reset(Member* m, cudaStream_t stream) {
  CU(xfer(m->mask_base, m->mask0_base, m->mask_bytes, cudaMemcpyDeviceToDevice, stream));
  CU(cudaMemsetAsync(m->f, 0, 9 * m->plane * storage_bytes(m->p.precision), stream));  // g = 0: rest at rho0
  CU(cudaMemsetAsync(m->drho, 0, 5 * align_up(m->plane * 4), stream));                 // the five fields
  m->steps_done = 0;
  return LBM_OK;
}

// ---- growing buffers -------------------------------------------------------

cudaError_t GrowBuf::reserve(size_t bytes, bool* moved) {
  if (moved) *moved = false;
  if (bytes <= cap && p) return cudaSuccess;
  const size_t want = std::max<size_t>(std::max<size_t>(bytes, 256), cap + cap / 2);
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = dev_malloc(&p, want);
  if (e != cudaSuccess) {
    p = nullptr;
    return e;
  }
  cap = want;
  if (moved) *moved = true;
  return cudaSuccess;
}

void GrowBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
}

// ---- engine ----------------------------------------------------------------

Engine::~Engine() {
  if (stream) cudaStreamSynchronize(stream);
  for (Engine* g : groups) delete g;  // they do not own the members
  for (auto& g : graphs)
    if (g) cudaGraphExecDestroy(g);
  if (own_members)
    for (Member* x : m) delete x;
  for (GrowBuf* b : {&L.views, &L.word_off, &L.seg_word_off, &XL.views, &XL.word_off, &XL.seg_word_off, &segs,
                     &n_segs, &seg_scratch, &partials, &result, &fluid_dev, &n_swap_dev, &dense_f, &oc_buf, &bar,
                     &best, &rplan, &halo, &cell_list, &cell_scan, &pair_list, &pair_scan})
    b->release();
  if (h_rplan) cudaFreeHost(h_rplan);
  if (h_bar_error) cudaFreeHost(h_bar_error);
  if (h_result) cudaFreeHost(h_result);
  if (h_info) cudaFreeHost(h_info);
  if (h_count) cudaFreeHost(h_count);
  if (h_nswap) cudaFreeHost(h_nswap);
  if (ev_begin) cudaEventDestroy(ev_begin);
  if (ev_end) cudaEventDestroy(ev_end);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

lbm_status engine_new(int precision, int residual_every, void* cuda_stream, bool fixed_grid, Engine** out) {
  *out = nullptr;
  Engine* E = new Engine();
  E->precision = precision;
  E->residual_every = residual_every;
  E->fixed_grid = fixed_grid;
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
  CUE(cudaEventCreate(&E->ev_begin));
  CUE(cudaEventCreate(&E->ev_end));
  CUE(E->n_segs.reserve(2 * sizeof(int)));
  CUE(E->bar.reserve(sizeof(StepBarrier)));
  CUE(cudaMemsetAsync(E->bar.p, 0, sizeof(StepBarrier), E->stream));
#undef CUE
  E->step = shape(E, kStepWarps, kDefaultGridScale);
  *out = E;
  return LBM_OK;
}

lbm_status rebuild_worklist(Engine* E) {
  E->rplan_valid = false;
  E->cells_valid = false;
  E->pairs_valid = false;
  for (Engine* g : E->groups) {  // the groups' lists follow the members' masks
    lbm_status st = rebuild_worklist(g);
    if (st != LBM_OK) return st;
  }
  if (E->n() == 0) return LBM_OK;
  CU(launch_build_segments(static_cast<const LatticeView*>(E->L.views.p), static_cast<const int*>(E->L.seg_word_off.p),
                           E->n(), E->L.total_seg_words, std::max(1, E->L.total_seg_words),
                           static_cast<int*>(E->seg_scratch.p), static_cast<SegRef*>(E->segs.p),
                           static_cast<int*>(E->n_segs.p), E->stream));
  CU(launch_count_fluid(static_cast<const LatticeView*>(E->L.views.p), static_cast<const int*>(E->L.word_off.p),
                        E->n(), E->L.total_words, static_cast<unsigned long long*>(E->fluid_dev.p), E->stream));
  DEBUG_SYNC(E, "work-list");
  return LBM_OK;
}

bool cells_eligible(const Engine* E) {
  if (E->features != 0 || E->n() == 0 || E->n() >= (1 << kCellLatticeBits) || debug_sync()) return false;
  for (const Member* m : E->m)
    if (m->p.outlet == LBM_OUT_NEUMANN) return false;  // its shuffle needs cell nx-2 in the lane to the left
  return true;
}

lbm_status ensure_cells(Engine* E) {
  if (E->cells_valid) return LBM_OK;
  const int cap = std::max(1, E->L.total_seg_words);
  long long fluid = 0;
  for (const Member* m : E->m) fluid += m->fluid_cells;
  CU(E->cell_scan.reserve((2 * ((size_t)cap + 1) + scan_tmp_ints(cap)) * sizeof(int)));
  CU(E->cell_list.reserve((size_t)std::max<long long>(1, fluid) * sizeof(CellRef)));
  int* cnt = static_cast<int*>(E->cell_scan.p);
  CU(launch_build_cells(static_cast<const LatticeView*>(E->L.views.p), static_cast<const SegRef*>(E->segs.p),
                        static_cast<const int*>(E->n_segs.p), cap, cnt, cnt + cap, cnt + 2 * ((size_t)cap + 1),
                        static_cast<CellRef*>(E->cell_list.p), E->stream));
  DEBUG_SYNC(E, "cell list");
  E->cells_valid = true;
  return LBM_OK;
}

bool pairs_eligible(const Engine* E) {
  return E->features == 0 && E->n() > 0 && E->n() < kPairTask;
}

lbm_status ensure_pairs(Engine* E) {
  if (E->pairs_valid) return LBM_OK;
  const int cap = std::max(1, E->L.total_seg_words);
  CU(E->pair_scan.reserve((2 * (size_t)cap + 1 + scan_tmp_ints(cap)) * sizeof(int)));
  CU(E->pair_list.reserve((size_t)cap * sizeof(SegRef)));
  int* emit = static_cast<int*>(E->pair_scan.p);
  CU(launch_build_pairs(static_cast<const LatticeView*>(E->L.views.p), static_cast<const SegRef*>(E->segs.p),
                        static_cast<const int*>(E->n_segs.p), cap, emit, emit + cap, emit + 2 * (size_t)cap + 1,
                        static_cast<SegRef*>(E->pair_list.p), E->stream));
  DEBUG_SYNC(E, "paired list");
  E->pairs_valid = true;
  return LBM_OK;
}

lbm_status resident_prepare(Engine* E, bool* ok) {
  *ok = false;
  if (E->features != 0 || E->fixed_grid || E->n() == 0 || debug_sync()) return LBM_OK;
  if (!E->rplan_valid) {
    NvtxRange nvtx("lbm_resident_plan");
    CU(E->rplan.reserve(4 * sizeof(int)));
    if (!E->h_rplan) CU(cudaMallocHost((void**)&E->h_rplan, 4 * sizeof(int)));
    const int* scratch = static_cast<const int*>(E->seg_scratch.p);
    CU(launch_resident_plan(static_cast<const LatticeView*>(E->L.views.p), static_cast<const SegRef*>(E->segs.p),
                            static_cast<const int*>(E->n_segs.p), static_cast<const int*>(E->L.seg_word_off.p),
                            scratch, scratch + E->L.total_seg_words, E->sm_count, static_cast<int*>(E->rplan.p),
                            E->stream));
    CU(xfer(E->h_rplan, E->rplan.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, E->stream));
    CU(cudaStreamSynchronize(E->stream));
    const int nseg = E->h_rplan[0];
    ResidentShape rs{};
    rs.grid = resident_grid(nseg, E->sm_count);
    const int own = (nseg + rs.grid - 1) / std::max(1, rs.grid);
    rs.warps = std::max(1, (own + 1) / 2);
    rs.words = E->h_rplan[1];
    rs.pairs = E->h_rplan[2];
    bool fits = nseg > 0 && E->h_rplan[3] == 1 && own <= kResidentMaxOwn && rs.words <= 65536 &&
                resident_smem_bytes(E->precision, rs.words, rs.pairs) <= (size_t)std::max(0, resident_max_smem());
    if (fits) {
      bool moved = false;
      const size_t bytes = (size_t)2 * nseg * 9 * 32 * sizeof(unsigned long long);
      CU(E->halo.reserve(bytes, &moved));
      if (moved) {  // fresh memory: no tag in it may match a future one
        CU(cudaMemsetAsync(E->halo.p, 0, E->halo.cap, E->stream));
        E->halo_epoch = 1;
      }
      E->halo_cap = (int)(E->halo.cap / (2 * 9 * 32 * sizeof(unsigned long long)));
    }
    E->rshape = rs;
    E->rplan_ok = fits;
    E->rplan_valid = true;
    if (tune_log_enabled())
      std::fprintf(stderr, "lbm resident plan: segments %d blocks %d warps %d words %d ghost rows %d fits %d\n",
                   nseg, rs.grid, rs.warps, rs.words, rs.pairs, fits ? 1 : 0);
  }
  *ok = E->rplan_ok;
  return LBM_OK;
}

lbm_status engine_set_members(Engine* E, const std::vector<Member*>& members) {
  int features = 0;
  for (Member* mb : members) {
    if (mb->p.precision != E->precision) return fail(LBM_ERR_ARG, "all lattices of a set share one precision");
    if (mb->p.collision != LBM_COLLIDE_BGK) features |= 1;
    if (mb->p.mirror) features |= 2;
  }
  if (features != E->features) {  // a different kernel build: the tuned shape and graphs no longer apply
    E->features = features;
    E->tuned = false;
    E->step.cells_per_thread = 1;
    E->step.stages = 0;
    E->step.persistent = 0;
  }
  E->m = members;
  const size_t n = members.size();
  lbm_status st = layout_build(E->L, E->m, E->stream);
  if (st != LBM_OK) return st;
  long long max_cells = 0;
  for (Member* mb : members) max_cells = std::max<long long>(max_cells, (long long)mb->nx * mb->ny);
  const size_t nn = std::max<size_t>(1, n);
  CU(E->segs.reserve(segment_list_bytes(std::max(1, E->L.total_seg_words))));
  CU(E->seg_scratch.reserve(segment_scratch_ints(E->L.total_seg_words) * sizeof(int)));
  CU(E->partials.reserve(sizeof(double) * 2 * kResidualBlocks * nn));
  CU(E->result.reserve(sizeof(double) * kResultDoubles * nn));
  CU(E->fluid_dev.reserve(sizeof(unsigned long long) * nn));
  CU(E->n_swap_dev.reserve(sizeof(int) * nn));
  CU(E->dense_f.reserve((size_t)std::max<long long>(1, max_cells) * 4));
  st = ensure_pinned(E, nn);
  if (st != LBM_OK) return st;
  if (E->fixed_grid) {
    // the request loop's engine is never tuned (its members change every
    // tick): compacted cell tasks at 4 warps a block, the tuner's pick for
    // L2-resident sets of candidate distributors, where every request allows
    // them; the grid is sized for the device either way
    const char* e = std::getenv("LBM_SERVER_CELLS");
    const bool cells = !(e && e[0] == '0') && cells_eligible(E);
    E->step = cells ? cells_shape(E, 4, kDefaultGridScale) : shape(E, kStepWarps, kDefaultGridScale);
  } else if (!E->tuned) {
    E->step = shape(E, E->step.warps_per_block, kDefaultGridScale);
  }
  if (n == 0) return LBM_OK;
  st = rebuild_worklist(E);
  if (st != LBM_OK) return st;
  CU(xfer(E->h_count, E->fluid_dev.p, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost,
                     E->stream));
  CU(cudaStreamSynchronize(E->stream));
  for (size_t i = 0; i < n; ++i) E->m[i]->fluid_cells = (int64_t)E->h_count[i];
  return LBM_OK;
}

lbm_status engine_reset(Engine* E) {
  for (Member* mb : E->m) {
    lbm_status st = member_reset(mb, E->stream);
    if (st != LBM_OK) return st;
  }
  lbm_status st = rebuild_worklist(E);
  if (st != LBM_OK) return st;
  CU(xfer(E->h_count, E->fluid_dev.p, sizeof(unsigned long long) * E->n(), cudaMemcpyDeviceToHost,
                     E->stream));
  CU(cudaStreamSynchronize(E->stream));
  for (int i = 0; i < E->n(); ++i) E->m[i]->fluid_cells = (int64_t)E->h_count[i];
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
  // every argument and geometry rule before any device call
  for (int i = 0; i < n; ++i) {
    lbm_status st = member_check(params[i], cells[i]);
    if (st != LBM_OK) return st;
  }
  Engine* E = nullptr;
  lbm_status st = engine_new(params[0].precision, params[0].residual_every, cuda_stream, false, &E);
  if (st != LBM_OK) return st;
  std::vector<Member*> ms;
  for (int i = 0; i < n && st == LBM_OK; ++i) {
    Member* mb = nullptr;
    st = member_create(params[i], cells[i], E->stream, &mb);
    if (st == LBM_OK) {
      ms.push_back(mb);
      st = member_reset(mb, E->stream);
    }
  }
  E->m = ms;  // owned from here on, also on failure
  if (st == LBM_OK) st = engine_set_members(E, ms);
  if (st == LBM_OK) st = reserve_oc(E, E->L);
  if (st != LBM_OK) {
    delete E;
    return st;
  }
  *out = E;
  return LBM_OK;
}

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

// Member groups (decided once, at the first solve of 256 steps or more).
// A batch is split when its members' population bytes exceed 1.5 times the
// group budget and every member is below a quarter of it: members in order,
// each group up to the budget.  The budget is a third of the L2 cache of
// FP32 populations, two thirds of that with 16-bit storage: a group's other
// per-cell data (cell-list entry, flags) does not shrink with the storage,
// and on the 256 candidates the 16-bit groups ran fastest at about 4/3 of
// the FP32 groups' cells (budget 14 / 21 / 28 / 42 MB: 61.3 / 62.6 / 65.8 /
// 62.2 GLUPS; FP32 at 28 / 42 MB: 77.1 / 79.0).  32-48 candidates at a
// time step 1.5x faster (FP32) than all 256, which stream from DRAM.
// LBM_GROUPS=0 turns grouping off; LBM_GROUP_BYTES sets the budget (tests).
bool groups_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LBM_GROUPS");
    return !(e && e[0] == '0');
  }();
  return on;
}

lbm_status ensure_groups(Engine* E) {
  if (E->groups_decided) return LBM_OK;
  E->groups_decided = true;
  if (E->n() < 2 || E->fixed_grid || E->in_group || E->shape_fixed || !groups_enabled()) return LBM_OK;
  double budget = 0.0;
  if (const char* e = std::getenv("LBM_GROUP_BYTES")) budget = std::atof(e);
  if (budget <= 0.0) {
    int dev = 0, l2 = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    budget = l2 / 3.0 * (E->precision == LBM_F32 ? 1.0 : 2.0 / 3.0);
  }
  const double sb = 9.0 * (double)storage_bytes(E->precision);
  double total = 0.0, largest = 0.0;
  for (const Member* m : E->m) {
    total += sb * (double)m->fluid_cells;
    largest = std::max(largest, sb * (double)m->fluid_cells);
  }
  if (total <= 1.5 * budget || largest > 0.25 * budget) return LBM_OK;
  std::vector<std::vector<Member*>> parts(1);
  double acc = 0.0;
  for (Member* m : E->m) {
    const double b = sb * (double)m->fluid_cells;
    if (!parts.back().empty() && acc + b > budget) {
      parts.emplace_back();
      acc = 0.0;
    }
    parts.back().push_back(m);
    acc += b;
  }
  for (const auto& part : parts) {
    Engine* g = nullptr;
    lbm_status st = engine_new(E->precision, E->residual_every, E->stream, false, &g);
    if (st == LBM_OK) {
      g->own_members = false;
      g->in_group = true;
      E->groups.push_back(g);  // owned by E from here on
      st = engine_set_members(g, part);
    }
    if (st != LBM_OK) {  // no half-built grouping: the batch steps as one set
      for (Engine* x : E->groups) delete x;
      E->groups.clear();
      return st;
    }
  }
  return LBM_OK;
}

int engine_step_groups(const Engine* E) { return E->groups.empty() ? 1 : (int)E->groups.size(); }

// The time steps of a solve of E's members (moments at the last step and,
// with the residual, K steps before it).
lbm_status enqueue_steps(Engine* E, int64_t n_steps, bool with_res) {
  const int K = E->residual_every;
  lbm_status st;
  bool resident = false;
  if (E->step.persistent == 2 && !debug_sync()) {
    if ((st = resident_prepare(E, &resident)) != LBM_OK) return st;
    if (!resident) E->step = shape(E, kStepWarps, kDefaultGridScale);  // the list outgrew the chip
  }
  if (E->step.persistent == 3) {
    if (!cells_eligible(E)) E->step = shape(E, kStepWarps, kDefaultGridScale);
    else if ((st = ensure_cells(E)) != LBM_OK) return st;
  }
  if (E->step.persistent == 4) {
    if (!pairs_eligible(E)) E->step = shape(E, kStepWarps, kDefaultGridScale);
    else if ((st = ensure_pairs(E)) != LBM_OK) return st;
  }
  if (resident) {
    if ((st = run_resident(E, n_steps, with_res ? (int)(n_steps - K - 1) : -1)) != LBM_OK) return st;
  } else if (with_res) {
    if ((st = run_plain_pairs(E, (n_steps - K) / 2 - 1)) != LBM_OK) return st;
    if ((st = launch_pair(E, 2)) != LBM_OK) return st;
    if ((st = run_plain_pairs(E, K / 2 - 1)) != LBM_OK) return st;
  } else {
    if ((st = run_plain_pairs(E, n_steps / 2 - 1)) != LBM_OK) return st;
  }
  if (!resident && (st = launch_pair(E, 1)) != LBM_OK) return st;
  return LBM_OK;
}

lbm_status enqueue_steps_and_reduce(Engine* E, int64_t n_steps, bool with_res) {
  lbm_status st;
  E->bar_used = false;
  {
    NvtxRange nvtx("lbm_time_steps");
    CU(cudaEventRecord(E->ev_begin, E->stream));
    if (E->groups.empty()) {
      if ((st = enqueue_steps(E, n_steps, with_res)) != LBM_OK) return st;
    } else {
      for (Engine* g : E->groups)  // one group after the other: each stays in L2 for its steps
        if ((st = enqueue_steps(g, n_steps, with_res)) != LBM_OK) return st;
    }
    CU(cudaEventRecord(E->ev_end, E->stream));
  }
  NvtxRange nvtx_red("lbm_reductions");
  const LatticeView* views = static_cast<const LatticeView*>(E->L.views.p);
  double* partials = static_cast<double*>(E->partials.p);
  if (with_res) {
    CU(launch_residual_partials(views, E->n(), partials, E->stream));
    DEBUG_SYNC(E, "residual partials");
  }
  CU(launch_finalize(views, E->n(), partials, with_res ? 1 : 0, static_cast<double*>(E->result.p), E->stream));
  DEBUG_SYNC(E, "finalize");
  CU(xfer(E->h_result, E->result.p, sizeof(double) * kResultDoubles * E->n(), cudaMemcpyDeviceToHost,
                     E->stream));
  if (E->bar_used)
    CU(xfer(E->h_bar_error, &static_cast<StepBarrier*>(E->bar.p)->error, sizeof(int),
                       cudaMemcpyDeviceToHost, E->stream));
  else
    *E->h_bar_error = 0;
  return LBM_OK;
}

lbm_status enqueue_solve(Engine* E, int64_t n_steps) {
  if (n_steps >= 256) {
    lbm_status st = ensure_groups(E);
    if (st != LBM_OK) return st;
  }
  if (!E->groups.empty()) {
    for (Engine* g : E->groups)
      if (!g->tuned && n_steps >= 256) {
        lbm_status st = autotune(g);
        if (st != LBM_OK) return st;
      }
  } else if (!E->tuned && n_steps >= 256) {
    lbm_status st = autotune(E);
    if (st != LBM_OK) return st;
  }
  const int K = E->residual_every;
  const bool with_res = K >= 2 && (K % 2) == 0 && n_steps >= (int64_t)K + 2;
  return enqueue_steps_and_reduce(E, n_steps, with_res);
}

lbm_status enqueue_exchange(Engine* E, const std::vector<int>& which, const int32_t* n_swap) {
  NvtxRange nvtx("lbm_exchange");
  const int nx_ = (int)which.size();
  bool all = nx_ == E->n();
  for (int k = 0; all && k < nx_; ++k) all = which[k] == k;
  const SetLayout* X = &E->L;
  if (!all) {
    std::vector<Member*> xm;
    for (int i : which) xm.push_back(E->m[i]);
    lbm_status st = layout_build(E->XL, xm, E->stream);
    if (st != LBM_OK) return st;
    X = &E->XL;
  }
  lbm_status st = reserve_oc(E, *X);
  if (st != LBM_OK) return st;
  for (int k = 0; k < nx_; ++k) E->h_nswap[k] = n_swap[k];
  CU(xfer(E->n_swap_dev.p, E->h_nswap, sizeof(int) * nx_, cudaMemcpyHostToDevice, E->stream));
  const LatticeView* xv = static_cast<const LatticeView*>(X->views.p);
  CU(launch_oc_select(xv, static_cast<const int*>(X->word_off.p), nx_, X->total_words,
                      static_cast<const int*>(E->n_swap_dev.p), E->oc, E->stream));
  DEBUG_SYNC(E, "selection");
  CU(launch_oc_apply(E->precision, xv, nx_, E->oc, E->stream));
  DEBUG_SYNC(E, "exchange");
  const size_t sb = storage_bytes(E->precision);
  for (int i : which) {
    Member* m = E->m[i];
    if (m->p.reinit == LBM_REINIT_COLD) CU(cudaMemsetAsync(m->f, 0, 9 * m->plane * sb, E->stream));
  }
  st = rebuild_worklist(E);
  if (st != LBM_OK) return st;
  CU(xfer(E->h_info, E->oc.info, sizeof(int) * 8 * nx_, cudaMemcpyDeviceToHost, E->stream));
  CU(xfer(E->h_count, E->fluid_dev.p, sizeof(unsigned long long) * E->n(), cudaMemcpyDeviceToHost,
                     E->stream));
  return LBM_OK;
}

lbm_status check_canaries(Engine* E) {
  if (!kCanaryBytes) return LBM_OK;
  std::vector<unsigned char> h(2 * kCanaryBytes);
  for (int i = 0; i < E->n(); ++i) {
    const Member* m = E->m[i];
    CU(cudaMemcpy(h.data(), m->canary_lo, kCanaryBytes, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(h.data() + kCanaryBytes, m->canary_hi, kCanaryBytes, cudaMemcpyDeviceToHost));
    for (unsigned char c : h)
      if (c != kCanaryByte)
        return fail(LBM_ERR_CUDA, "lattice " + std::to_string(i) +
                                      ": a canary next to the population planes was overwritten");
  }
  return LBM_OK;
}

lbm_status debug_task_counts(Engine* E, int32_t* segments, int32_t* windows) {
  int32_t n[2] = {0, 0};  // list segments, paired tasks
  if (E->n() > 0) {
    const bool paired = pairs_eligible(E);
    if (paired) {
      lbm_status st = ensure_pairs(E);
      if (st != LBM_OK) return st;
    }
    CU(xfer(&n[0], E->n_segs.p, sizeof(int32_t), cudaMemcpyDeviceToHost, E->stream));
    if (paired)
      CU(xfer(&n[1], static_cast<const int*>(E->pair_scan.p) + 2 * (size_t)std::max(1, E->L.total_seg_words),
              sizeof(int32_t), cudaMemcpyDeviceToHost, E->stream));
    else
      n[1] = n[0];
    CU(cudaStreamSynchronize(E->stream));
  }
  if (segments) *segments = n[0];
  if (windows) *windows = n[0] - n[1];  // each window merges two list segments into one task
  return LBM_OK;
}

lbm_status debug_damage_canary(Engine* E) {
  if constexpr (kCanaryBytes == 0) {
    return fail(LBM_ERR_ARG, "canaries exist only in the bounds-checked build");
  } else {
    CU(cudaStreamSynchronize(E->stream));
    CU(cudaMemset(E->m[0]->canary_hi, 0, 4));
    return LBM_OK;
  }
}

lbm_status engine_solve(Engine* E, int64_t n_steps, lbm_solve_result* out) {
  NvtxRange nvtx("lbm_solve");
  if (n_steps < 2 || (n_steps % 2) != 0) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  lbm_status st = enqueue_solve(E, n_steps);
  if (st != LBM_OK) return st;
  CU(cudaStreamSynchronize(E->stream));
  for (Member* m : E->m) m->steps_done += n_steps;
  E->solved = true;
  account_steps(E, n_steps);
  if (*E->h_bar_error != 0) return fail(LBM_ERR_TIMEOUT, "step kernel: a bounded device wait gave up");
  lbm_status cst = check_canaries(E);
  if (cst != LBM_OK) return cst;
  bool bad = false;
  for (int i = 0; i < E->n(); ++i) {
    fill_result(E, i, out + i);
    bad |= E->h_result[(size_t)i * kResultDoubles + 7] != 0.0;
  }
  if (bad) return fail(LBM_ERR_DIVERGED, "non-finite pressure drop, flow rate or residual");
  return LBM_OK;
}

lbm_status engine_optimize(Engine* E, const int32_t* n_swap, int64_t n_steps, lbm_opt_result* out) {
  NvtxRange nvtx("lbm_optimize_step");
  if (n_steps < 2 || (n_steps % 2) != 0) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  for (int i = 0; i < E->n(); ++i)
    if (n_swap[i] < 0) return fail(LBM_ERR_ARG, "n_swap must be >= 0");
  if (!E->solved) return fail(LBM_ERR_ARG, "an exchange needs a field: solve first");
  std::vector<int> all(E->n());
  for (int i = 0; i < E->n(); ++i) all[i] = i;
  lbm_status st = enqueue_exchange(E, all, n_swap);
  if (st != LBM_OK) return st;
  st = enqueue_solve(E, n_steps);
  if (st != LBM_OK) return st;
  CU(cudaStreamSynchronize(E->stream));
  bool nan = false, count_changed = false, bad = false;
  for (int i = 0; i < E->n(); ++i) {
    Member* m = E->m[i];
    m->steps_done += n_steps;
    const int64_t before = m->fluid_cells;
    m->fluid_cells = (int64_t)E->h_count[i];
    count_changed |= m->fluid_cells != before;
    nan |= E->h_info[8 * i + 3] != 0;
    bad |= E->h_result[(size_t)i * kResultDoubles + 7] != 0.0;
  }
  account_steps(E, n_steps);
  if (*E->h_bar_error != 0) return fail(LBM_ERR_TIMEOUT, "step kernel: a bounded device wait gave up");
  lbm_status cst = check_canaries(E);
  if (cst != LBM_OK) return cst;
  for (int i = 0; i < E->n(); ++i) {
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

namespace {

// A member's state: populations, current mask and the moment fields of the
// last step (drho, ux, uy: the first three field planes of the slab).
struct StateCopy {
  size_t f, mask, fields;
};

StateCopy state_sizes(const Member* m) {
  return {9 * m->plane * storage_bytes(m->p.precision), m->mask_bytes, 3 * align_up(m->plane * 4)};
}

lbm_status save_state(Engine* E, const Member* m) {
  const StateCopy z = state_sizes(m);
  CU(E->best.reserve(z.f + z.mask + z.fields));
  char* b = static_cast<char*>(E->best.p);
  CU(xfer(b, m->f, z.f, cudaMemcpyDeviceToDevice, E->stream));
  CU(xfer(b + z.f, m->mask_base, z.mask, cudaMemcpyDeviceToDevice, E->stream));
  CU(xfer(b + z.f + z.mask, m->drho, z.fields, cudaMemcpyDeviceToDevice, E->stream));
  return LBM_OK;
}

lbm_status restore_state(Engine* E, Member* m) {
  const StateCopy z = state_sizes(m);
  const char* b = static_cast<const char*>(E->best.p);
  CU(xfer(m->f, b, z.f, cudaMemcpyDeviceToDevice, E->stream));
  CU(xfer(m->mask_base, b + z.f, z.mask, cudaMemcpyDeviceToDevice, E->stream));
  CU(xfer(m->drho, b + z.f + z.mask, z.fields, cudaMemcpyDeviceToDevice, E->stream));
  lbm_status st = rebuild_worklist(E);
  if (st != LBM_OK) return st;
  CU(xfer(E->h_count, E->fluid_dev.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, E->stream));
  CU(cudaStreamSynchronize(E->stream));
  m->fluid_cells = (int64_t)E->h_count[0];
  return LBM_OK;
}

}  // namespace

lbm_status engine_optimize_loop(Engine* E, const lbm_opt_plan& P, double* hist, lbm_opt_summary* out) {
  if (E->n() != 1) return fail(LBM_ERR_ARG, "the optimisation loop runs on a single lattice");
  if (P.n_steps < 2 || (P.n_steps % 2) != 0 || P.max_iter < 0 || P.n_swap < 1 || P.patience < 1 ||
      (P.adapt != 0 && P.adapt != 1) || (P.keep_best != 0 && P.keep_best != 1) || P.reserved != 0 ||
      !std::isfinite(P.tol))
    return fail(LBM_ERR_ARG, "plan: n_steps even >= 2, max_iter >= 0, n_swap >= 1, patience >= 1, flags 0/1");
  std::memset(out, 0, sizeof(*out));
  Member* m = E->m[0];
  lbm_solve_result r;
  lbm_status st = engine_solve(E, P.n_steps, &r);
  if (st != LBM_OK) return st;
  std::vector<double> h{r.dp};
  if (hist) hist[0] = r.dp;
  int best = 0, calm = 0;
  int32_t n_swap = P.n_swap;
  if (P.keep_best && (st = save_state(E, m)) != LBM_OK) return st;
  for (int k = 1; k <= P.max_iter; ++k) {
    lbm_opt_result o;
    out->iterations = k - 1;
    out->n_swap_final = n_swap;
    st = engine_optimize(E, &n_swap, P.n_steps, &o);
    if (st != LBM_OK) return st;
    out->swapped += o.n_swapped;
    const double dp = o.solve.dp;
    h.push_back(dp);
    if (hist) hist[k] = dp;
    if (dp < h[best]) {
      best = k;
      if (P.keep_best && (st = save_state(E, m)) != LBM_OK) return st;
    }
    if (P.adapt && dp > h[k - 1]) n_swap = std::max(1, n_swap / 2);
    if (P.tol > 0.0) {
      calm = std::fabs(dp - h[k - 1]) <= P.tol * std::fabs(dp) ? calm + 1 : 0;
      if (calm >= P.patience) {
        out->stopped = 1;
        break;
      }
    }
  }
  out->iterations = (int32_t)h.size() - 1;
  out->n_swap_final = n_swap;
  out->best_iter = best;
  out->dp_first = h.front();
  out->dp_best = h[best];
  out->dp_last = h.back();
  if (P.keep_best && best != out->iterations && (st = restore_state(E, m)) != LBM_OK) return st;
  return LBM_OK;
}

lbm_status engine_read(Engine* E, int i, uint32_t which, void* dst, size_t dst_bytes) {
  if (i < 0 || i >= E->n()) return fail(LBM_ERR_ARG, "member out of range");
  if (!dst) return fail(LBM_ERR_ARG, "dst is NULL");
  Member* m = E->m[i];
  const size_t nx = m->nx, ny = m->ny, ncell = nx * ny;
  const size_t sb = storage_bytes(E->precision);
  switch (which) {
    case LBM_FIELD_MASK:
      if (dst_bytes < ncell) return fail(LBM_ERR_ARG, "dst too small");
      CU(launch_unpack_mask(m->mask, m->nx, m->ny, m->wpr, m->cells, E->stream));
      CU(xfer(dst, m->cells, ncell, cudaMemcpyDefault, E->stream));
      break;
    case LBM_FIELD_RHO:
      if (dst_bytes < ncell * 4) return fail(LBM_ERR_ARG, "dst too small");
      CU(launch_rho_from_drho(m->drho, (float)m->p.rho0, m->mask, m->nx, m->ny, m->pitch, m->wpr,
                              static_cast<float*>(E->dense_f.p), E->stream));
      CU(xfer(dst, E->dense_f.p, ncell * 4, cudaMemcpyDefault, E->stream));
      break;
    case LBM_FIELD_DRHO:
    case LBM_FIELD_UX:
    case LBM_FIELD_UY: {
      if (dst_bytes < ncell * 4) return fail(LBM_ERR_ARG, "dst too small");
      const float* src = which == LBM_FIELD_DRHO ? m->drho : which == LBM_FIELD_UX ? m->ux : m->uy;
      CU(xfer2d(dst, nx * 4, src, (size_t)m->pitch * 4, nx * 4, ny, cudaMemcpyDefault, E->stream));
      break;
    }
    case LBM_FIELD_POPS:
      if (dst_bytes < 9 * ncell * sb) return fail(LBM_ERR_ARG, "dst too small");
      for (int k = 0; k < 9; ++k)
        CU(xfer2d(static_cast<char*>(dst) + k * ncell * sb, nx * sb,
                             static_cast<const char*>(m->f) + k * m->plane * sb, (size_t)m->pitch * sb, nx * sb,
                             ny, cudaMemcpyDefault, E->stream));
      break;
    default:
      return fail(LBM_ERR_ARG, "which must be exactly one LBM_FIELD_* value");
  }
  CU(cudaStreamSynchronize(E->stream));
  return LBM_OK;
}

lbm_status engine_step_config(Engine* E, int32_t* warps_per_block, int32_t* grid, int32_t* persistent,
                              int32_t* cells_per_thread, int32_t* stages) {
  const StepConfig& c = E->groups.empty() ? E->step : E->groups[0]->step;  // grouped: the first group's
  if (warps_per_block) *warps_per_block = c.warps_per_block;
  if (grid) *grid = c.grid;
  if (persistent) *persistent = c.persistent;
  if (cells_per_thread) *cells_per_thread = c.cells_per_thread;
  if (stages) *stages = c.stages;
  return LBM_OK;
}

lbm_status engine_set_step_config(Engine* E, int32_t warps_per_block, int32_t persistent, int32_t cells_per_thread,
                                  int32_t stages) {
  // a fixed shape applies to the whole set: no member groups
  E->shape_fixed = true;
  E->groups_decided = true;
  for (Engine* g : E->groups) delete g;
  E->groups.clear();
  if (persistent == 2) {  // on-chip resident steps: the shape follows from the work-list
    bool ok = false;
    lbm_status st = resident_prepare(E, &ok);
    if (st != LBM_OK) return st;
    if (!ok)
      return fail(LBM_ERR_ARG, "resident steps need plain BGK lattices whose segments fit in shared memory");
    E->step = resident_config(E);
    E->tuned = true;
    return LBM_OK;
  }
  if (persistent == 4) {  // paired tasks
    if (!pairs_eligible(E)) return fail(LBM_ERR_ARG, "paired tasks need plain BGK lattices");
    if (!step_shape_allowed(warps_per_block, cells_per_thread, 4) || (stages != 0 && (stages < 2 || stages > 4)))
      return fail(LBM_ERR_ARG,
                  "paired tasks take two cells per thread, 4, 8, 12 or 24 warps per block and stages 0 or 2-4");
    lbm_status st = ensure_pairs(E);
    if (st != LBM_OK) return st;
    E->step = pairs_shape(E, warps_per_block, kDefaultGridScale, stages);
    E->tuned = true;
    return LBM_OK;
  }
  if (persistent == 3) {  // compacted fluid-cell tasks
    if (!cells_eligible(E))
      return fail(LBM_ERR_ARG, "cell tasks need plain BGK lattices without a zero-gradient outlet");
    if (!step_shape_allowed(warps_per_block, 1, 3) || cells_per_thread != 1 ||
        (stages != 0 && (stages < 2 || stages > 4 || warps_per_block > 16)))
      return fail(LBM_ERR_ARG,
                  "cell tasks take one cell per thread, 4, 8, 12, 16 or 32 warps per block, and stages 0 or 2-4 "
                  "(at most 16 warps with stages)");
    lbm_status st = ensure_cells(E);
    if (st != LBM_OK) return st;
    E->step = cells_shape(E, warps_per_block, kDefaultGridScale, stages);
    E->tuned = true;
    return LBM_OK;
  }
  if (stages != 0 && stages != 2 && stages != 3) return fail(LBM_ERR_ARG, "stages must be 0, 2 or 3");
  if (stages != 0 && (persistent || cells_per_thread != 1))
    return fail(LBM_ERR_ARG, "staged loads take one cell per thread and per-phase launches");
  if (persistent != 0 && persistent != 1) return fail(LBM_ERR_ARG, "persistent must be 0, 1, 2, 3 or 4");
  if (cells_per_thread != 1 && cells_per_thread != 2) return fail(LBM_ERR_ARG, "cells_per_thread must be 1 or 2");
  if (!step_shape_allowed(warps_per_block, cells_per_thread, persistent))
    return fail(LBM_ERR_ARG,
                persistent ? "the persistent kernel takes 8 or 16 warps per block (8 with two cells per thread)"
                : cells_per_thread == 1 ? "one cell per thread takes 4, 8, 12, 16 or 32 warps per block"
                                        : "two cells per thread take 4, 8, 12 or 24 warps per block");
  if (stages != 0 && warps_per_block > 16) return fail(LBM_ERR_ARG, "staged loads take 4, 8 or 16 warps per block");
  if (E->features && (persistent || cells_per_thread != 1 || stages != 0))
    return fail(LBM_ERR_ARG, "lattices with collision models or a symmetry plane take the plain launch shape");
  StepConfig c = persistent ? persistent_shape(E, warps_per_block, cells_per_thread)
                            : shape(E, warps_per_block, kDefaultGridScale, cells_per_thread, stages);
  if (c.grid < 1) return fail(LBM_ERR_CUDA, "no resident block for the persistent kernel");
  E->step = c;
  E->tuned = true;
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

}  // namespace lbm
