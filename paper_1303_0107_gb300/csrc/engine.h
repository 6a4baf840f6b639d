// The engine behind the C ABI: a set of lattices stepped together.
//
// A Member is one lattice: its populations, mask, fields and port tables in
// one device allocation.  An Engine steps a list of members: it owns one
// descriptor table, one row-segment work-list, one reduction block and one
// exchange scratch for the whole list, so every stage of the loop of Sec. 2.3
// (steps 2-5) is one launch over all members.  The list may change between
// solves (the server adds and removes requests); set-level buffers then grow
// to the new totals and the captured step graphs stay valid for as long as
// the buffers they point to do.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbm {

// A named range on the host timeline for profilers (NVTX: solve, time
// steps, reductions, exchange, tuning, resident plan, server tick).  Costs
// nothing measurable when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

lbm_status fail(lbm_status s, const std::string& msg);
// Every device allocation of the library goes through dev_malloc, so that
// a test can make the n-th one fail (set_alloc_failure).
cudaError_t dev_malloc(void** p, size_t bytes);
void set_alloc_failure(int64_t after);
uint64_t launches_total();
size_t storage_bytes(int precision);
lbm_status check_params(const lbm_params& p);

// One lattice.  All device arrays live in one allocation (`slab`).
struct Member {
  lbm_params p{};
  int nx = 0, ny = 0, pitch = 0, wpr = 0;
  size_t plane = 0;
  std::vector<int> out_start, out_len;
  void* slab = nullptr;
  size_t slab_bytes = 0;
  void* f = nullptr;
  void *canary_lo = nullptr, *canary_hi = nullptr;  // bounds-checked build: guard blocks around f
  uint32_t *mask_base = nullptr, *mask0_base = nullptr, *mask = nullptr, *mask0 = nullptr;
  size_t mask_bytes = 0;
  float *drho = nullptr, *ux = nullptr, *uy = nullptr, *ux_prev = nullptr, *uy_prev = nullptr;
  float* u_in = nullptr;
  int* d_out = nullptr;     // [LBM_MAX_OUTLETS] starts, then [LBM_MAX_OUTLETS] lengths
  uint8_t* cells = nullptr; // [ny][nx] staging for uploads and mask reads
  int64_t fluid_cells = 0;
  int64_t steps_done = 0;
  LatticeView view{};       // word_off / seg_word_off / sel_off are set per set
  ~Member();
};

// Device bytes member_create allocates for a lattice of these parameters.
size_t member_footprint(const lbm_params& p);
// Validate, allocate and upload (cells: host uint8[ny][nx]); the cell map is
// packed on `stream`.  The host copies are staged before the call returns.
lbm_status member_create(const lbm_params& p, const uint8_t* cells, cudaStream_t stream, Member** out);
// The host-side checks of member_create (parameters and geometry rules).
lbm_status member_check(const lbm_params& p, const uint8_t* cells);
// Initial state of Sec. 3.3 on `stream`: cell map of creation, g = 0
// (f = w_i rho0 at rest), fields zero, steps_done = 0.
lbm_status member_reset(Member* m, cudaStream_t stream);

// A device buffer that only grows.
struct GrowBuf {
  void* p = nullptr;
  size_t cap = 0;
  // true if p changed
  cudaError_t reserve(size_t bytes, bool* moved = nullptr);
  void release();
};

// Device description of a list of members: their views (with the list's
// word, segment-word and pick offsets) and the offset arrays.
struct SetLayout {
  int n = 0;
  int total_words = 0, total_seg_words = 0;
  long long total_cells = 0, total_sel = 0;
  GrowBuf views, word_off, seg_word_off;
  std::vector<LatticeView> h_views;
  std::vector<int> h_woff, h_swoff;
  unsigned gen = 0;  // counts builds: kernels that took a view by value belong to one build
};

struct Engine {
  int precision = LBM_F32;
  int residual_every = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool own_members = true;  // handles and batches own their members; the server does not
  bool fixed_grid = false;  // step grid sized for the device, not for the current list
  int sm_count = 0;
  std::vector<Member*> m;

  SetLayout L;   // every member: time steps, reductions, work-list
  SetLayout XL;  // members of the next exchange (server only)
  GrowBuf segs, n_segs, seg_scratch, partials, result, fluid_dev, n_swap_dev, dense_f, bar;
  GrowBuf oc_buf;  // exchange scratch, carved into `oc`
  GrowBuf best;    // saved state of the best iteration (lbm_optimize with keep_best)
  OcScratch oc{};
  size_t pinned_n = 0;
  double* h_result = nullptr;             // pinned [n * kResultDoubles]
  int* h_info = nullptr;                  // pinned [8 n]
  unsigned long long* h_count = nullptr;  // pinned [n]
  int* h_nswap = nullptr;                 // pinned [n]
  int* h_bar_error = nullptr;             // pinned: grid-barrier error flag of the last solve
  bool bar_used = false;                  // the last enqueued solve ran the persistent kernel

  // on-chip resident steps (step.persistent == 2): the plan of the current
  // work-list (valid until the list is rebuilt), the halo buffer of tagged
  // words and the next tag
  GrowBuf rplan, halo;
  int* h_rplan = nullptr;  // pinned [4]
  bool rplan_valid = false, rplan_ok = false;
  ResidentShape rshape{};
  int halo_cap = 0;        // segments the halo buffer holds
  unsigned halo_epoch = 1;

  // compacted fluid-cell tasks (step.persistent == 3): the list and the
  // per-segment counts / prefix / scan scratch, valid until the work-list is rebuilt
  GrowBuf cell_list, cell_scan;
  bool cells_valid = false;
  // paired tasks (step.persistent == 4): the list and its emit flags /
  // offsets / scan scratch (the count in offsets[capacity]), valid until the
  // work-list is rebuilt
  GrowBuf pair_list, pair_scan;
  bool pairs_valid = false;

  cudaGraphExec_t graphs[4] = {nullptr, nullptr, nullptr, nullptr};  // 512, 64, 8 and 1 pairs
  // views, segs (or the cell or paired list), n_segs, shape, cell prefix (or paired count), layout build
  const void* graph_key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  StepConfig step{kStepWarps, 1, 0, 1, 0, 0};
  int features = 0;  // kernel build the members need: 1 collision models, 2 symmetry plane
  bool tuned = false;
  bool shape_fixed = false;  // set with engine_set_step_config: no tuning, no member groups
  // Member groups of a batch whose populations exceed the L2 cache: each
  // group's time steps run on an engine of its own (sharing the members and
  // the stream, with its own work-list and tuned shape) so that they stay
  // L2-resident; reductions and exchanges stay with this engine.
  std::vector<Engine*> groups;
  bool groups_decided = false;
  bool in_group = false;  // this engine steps one group of another engine's members
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  double step_ms = 0.0;
  int64_t step_launches = 0, fluid_updates = 0;
  bool solved = false;

  ~Engine();
  int n() const { return (int)m.size(); }
};

// An engine with no members (add them with engine_set_members).
lbm_status engine_new(int precision, int residual_every, void* cuda_stream, bool fixed_grid, Engine** out);
// Replace the member list; rebuilds the layout, the work-list and the fluid
// counts (synchronises the stream).
lbm_status engine_set_members(Engine* E, const std::vector<Member*>& members);
// Handles and batches: create n members and an engine that owns them.
lbm_status engine_create(int n, const lbm_params* params, const uint8_t* const* cells, void* cuda_stream,
                         Engine** out);
lbm_status engine_reset(Engine* E);
// Number of member groups the time steps run in (1 when not grouped).
int engine_step_groups(const Engine* E);
lbm_status rebuild_worklist(Engine* E);
// Plan the resident launch for the current work-list (synchronises the
// stream when the list changed since the last plan); *ok: the set fits.
lbm_status resident_prepare(Engine* E, bool* ok);
// Compacted fluid-cell tasks: whether the set may use them (plain BGK, no
// zero-gradient outlet), and the list built for the current work-list.
bool cells_eligible(const Engine* E);
lbm_status ensure_cells(Engine* E);
bool pairs_eligible(const Engine* E);
lbm_status ensure_pairs(Engine* E);

// Enqueue n_steps (even) with moments in the last step, optional residual,
// and the reductions of every member; results to pinned h_result.  The
// caller synchronises.
lbm_status enqueue_solve(Engine* E, int64_t n_steps);
// As enqueue_solve without autotuning and without residual.
lbm_status enqueue_steps_and_reduce(Engine* E, int64_t n_steps, bool with_residual);
// Exchange (select + apply + re-init + work-list) on the members listed in
// `which` (indices into E->m) with n_swap[k] for which[k]; info and fluid
// counts copied to h_info (per listed member) and h_count (every member).
lbm_status enqueue_exchange(Engine* E, const std::vector<int>& which, const int32_t* n_swap);
void fill_result(Engine* E, int i, lbm_solve_result* out);
void account_steps(Engine* E, int64_t n_steps);

lbm_status engine_solve(Engine* E, int64_t n_steps, lbm_solve_result* out);
lbm_status engine_optimize(Engine* E, const int32_t* n_swap, int64_t n_steps, lbm_opt_result* out);
// The loop of Sec. 2.3 with the stopping test, n_swap adaptation and
// best-state keeping of lbm_opt_plan (engines of one member).
lbm_status engine_optimize_loop(Engine* E, const lbm_opt_plan& plan, double* history, lbm_opt_summary* out);
lbm_status engine_read(Engine* E, int i, uint32_t which, void* dst, size_t dst_bytes);
lbm_status engine_step_config(Engine* E, int32_t* warps_per_block, int32_t* grid, int32_t* persistent,
                              int32_t* cells_per_thread, int32_t* stages);
lbm_status engine_set_step_config(Engine* E, int32_t warps_per_block, int32_t persistent, int32_t cells_per_thread,
                                  int32_t stages);
lbm_status engine_kernel_time(Engine* E, int reset, double* ms, int64_t* launches, int64_t* fluid_updates);
// Bounds-checked build: overwrite a few bytes of the first member's upper
// canary (host-side memset within the allocation), so that the next solve
// reports the damage; LBM_ERR_ARG in the normal build.
lbm_status debug_damage_canary(Engine* E);
lbm_status debug_task_counts(Engine* E, int32_t* segments, int32_t* windows);

// Copies through which the library moves data between host and device
// memory: cudaMemcpyAsync / cudaMemcpy2DAsync that also count the bytes
// crossing in each direction (process-wide; lbm_transfer_bytes reports
// them).  cudaMemcpyDefault copies are classified by the pointers' memory
// types; device-to-device copies count nothing.
cudaError_t xfer(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t stream);
cudaError_t xfer2d(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t height,
                   cudaMemcpyKind kind, cudaStream_t stream);
void transfer_bytes(uint64_t* h2d, uint64_t* d2h);

// thread-local last error and launch counter state shared with api.cu
extern thread_local bool t_capturing;
extern thread_local std::string t_last_error;
bool autotune_enabled();

}  // namespace lbm
