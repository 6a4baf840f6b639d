// Internal declarations shared by the CUDA translation units of the library.
// Not part of the public ABI (include/lbm.h is).
//
// Every kernel works on a set of lattices described by a device table of
// LatticeView entries: a handle is a set of one, a batch a set of many, and
// each stage of the path (work-list, time steps, reductions, exchange) is one
// launch over the whole set.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "lbm.h"

namespace lbm {

// Work unit of the stream-collide kernel: one row segment, the 32 cells of
// one mask word (row y, cells 32w .. 32w+31), taken by one warp (lane l ->
// cell 32w + l), one or two segments per warp task.  The segment list holds
// only segments with a fluid cell.
// Default block shape (the engine tunes it on its own lattices).
constexpr int kStepWarps = 8;
// Row pitch of every per-cell array, in elements: a multiple of 64 so that
// each row starts on a 128-byte boundary for 16-bit and 32-bit storage.
constexpr int kPitchAlign = 64;

// Cell mask layout: one bit per cell, bit (x & 31) of word x >> 5 of a row,
// set = solid.  Rows are stored with a stride of wpr + 2 words and one solid
// padding word on each side, plus one padding row below row 0 and one above
// row ny-1, both solid -- except that with a symmetry plane below row 0 the
// row below holds a copy of row 0 (its mirror image); the mask pointer
// addresses word 0 of row 0.  Every
// neighbour word a kernel forms (rows y-1..y+1, words w-1..w+1) therefore lies
// inside the allocation and reads as wall outside the lattice.
__host__ __device__ constexpr int mask_stride(int wpr) { return wpr + 2; }
__host__ __device__ constexpr long long mask_alloc_words(int wpr, int ny) {
  return (long long)(ny + 2) * mask_stride(wpr);
}
__host__ __device__ constexpr long long mask_origin(int wpr) { return mask_stride(wpr) + 1; }

// Everything a kernel needs to know about one lattice, in a device table.
// Entries are 16-byte aligned and a multiple of 16 bytes long, so any entry
// of a table can be read with 16-byte loads.
struct alignas(16) LatticeView {
  void* f;                 // 9 population planes [9][ny][pitch] of the storage type
  const uint32_t* mask;    // word (0, 0) of the padded mask (see above)
  float* drho;             // [ny][pitch] rho - rho0 of the last step
  float* ux;               // [ny][pitch]
  float* uy;               // [ny][pitch]
  float* ux_prev;          // [ny][pitch] u of the step K steps before the last (residual)
  float* uy_prev;          // [ny][pitch]
  const float* u_in;       // [ny] inlet u_x per row (0 where the row has no inlet cell)
  const int* out_start;    // [n_outlets] first row of each outlet run
  const int* out_len;      // [n_outlets] rows of each outlet run
  long long plane;         // elements per population plane = ny * pitch
  long long f_elems;       // 9 * plane
  double rho0d;            // rho0 (FP64, for the scores and reductions)
  double mu;               // rho0 (tau - 1/2) / 3 (Eq. 5)
  int nx, ny, pitch, wpr;
  float omega;             // 1 / tau
  float rho0;
  int outlet_rule;         // lbm_outlet_rule
  int port_scheme;         // lbm_port_scheme
  int n_outlets;
  int sel_off;             // start of this lattice's picks in the shared pick arrays
  int word_off;            // start of this lattice's words in the concatenated word space
  int seg_word_off;        // start of its interior-row words (rows 1..ny-2)
  int guard;               // connectivity guard on fluid candidates (lbm_params.guard)
  int mirror;              // symmetry plane below row 0 (lbm_params.mirror)
  int collision;           // lbm_collision
  float c_smag;            // Smagorinsky constant
};

// A row segment: lattice index and (y << 12) | w (w < 4096, so nx <= 131072).
struct alignas(8) SegRef {
  int lattice;
  int yw;
};
constexpr int kSegWordBits = 12;
static_assert(sizeof(LatticeView) % 16 == 0 && alignof(LatticeView) == 16, "LatticeView layout");
static_assert(sizeof(SegRef) == 8, "SegRef layout");

// First row of the step work-list: row 0 is fluid-capable only next to a
// symmetry plane; the last row (ny - 1) is always a wall.
__host__ __device__ inline int first_step_row(const LatticeView& v) { return v.mirror ? 0 : 1; }

// Index of the lattice whose range [off[l], off[l+1]) holds i (off ascending,
// off[0] = 0, n lattices).
__host__ __device__ inline int find_lattice(const int* off, int n, long long i) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---- stream-collide (step.cu) ----------------------------------------------
// phase 0 ("A"): reads the post-collision state from the neighbours, writes
//   the new post-collision values into the slots the neighbours will read
//   (or back into the cell's own slots where the neighbour is solid);
// phase 1 ("B"): reads and writes the cell's own slots only, leaving the
//   canonical layout F[i][cell] = post-collision population i.
// moments (phase B only): 0 none, 1 write drho/ux/uy, 2 write drho/ux_prev/uy_prev.
// Launched as a programmatic dependent of the previous kernel on the stream:
// it reads its work item, descriptor and mask before waiting for that kernel,
// and only then the populations.
struct StepConfig {
  int warps_per_block;  // 4, 8 or 16
  int grid;             // blocks
  int persistent;       // launch mode: 0 one launch per phase over the row segments; 1 all pairs of a
                        //    solve in one cooperative launch; 2 on-chip resident solve (resident.cu);
                        //    3 one launch per phase over compacted fluid-cell tasks (32 cells a warp);
                        //    4 one launch per phase over paired tasks (interior 64-cell windows, two
                        //    cells a lane, and the other segments)
  int cells_per_thread; // 1 or 2: row segments per warp task (2: at most 8 warps per block)
  int stages;           // 0: populations loaded into registers; 2 or 3: staged through shared
                        //    memory that many segments ahead (one cell per thread, per-phase launches)
  int features;         // kernel build: bit 0 collision models beyond BGK, bit 1 symmetry plane
                        //    (non-zero: one cell per thread, register loads, per-phase launches)
};
// A fluid cell of the compacted task list: c = y * pitch + x in its lattice;
// meta = lattice | neighbour flags (kNbE..kNbMirror) << 20 | inlet << 29 |
// outlet << 30.  The list holds a set's fluid cells in segment-list order
// (lattice, row, x), so a warp's 32 cells are consecutive along x within
// runs of fluid.
struct alignas(8) CellRef {
  int c;
  unsigned meta;
};
constexpr int kCellLatticeBits = 20;
// Build the compacted list: per-segment fluid counts cnt[capacity] (0 past
// the list), their exclusive scan cpre[capacity + 1] (cells = cpre[n_segs[0]]),
// and the cells; tmp holds scan_tmp_ints(capacity) ints.  Needs the segment
// list and its neighbour flags (launch_build_segments).
cudaError_t launch_build_cells(const LatticeView* views, const SegRef* segs, const int* n_segs, int capacity,
                               int* cnt, int* cpre, int* tmp, CellRef* cells, cudaStream_t stream);
// One phase over the compacted list (sc.warps_per_block, sc.grid; one cell
// per thread; sc.stages 0: populations into registers, 2-4: copied into
// shared memory that many tasks ahead, at most 16 warps per block), a
// programmatic dependent launch like launch_stream_collide.
// Plain BGK lattices without a zero-gradient outlet only.
cudaError_t launch_stream_collide_cells(int precision, int phase, int moments, const LatticeView* views,
                                        const CellRef* cells, const int* n_segs, const int* cpre, StepConfig sc,
                                        cudaStream_t stream);
int stream_collide_cells_blocks_per_sm(int precision, int phase, int moments, int warps_per_block, int stages);
// Paired tasks: an entry {lattice | kPairTask, (y << kSegWordBits) | p} is
// the interior window of 64 cells of row y, mask words 2p and 2p+1 (its
// cells and all their neighbours fluid), taken by one warp two cells a
// lane; any other entry is a row segment as in the segment list.
constexpr int kPairTask = 1 << 30;
// Build the paired list from the segment list, keeping its order: emit and
// off hold capacity and capacity + 1 ints, tmp scan_tmp_ints(capacity); the
// number of tasks lands in off[capacity].  Plain lattices without a symmetry
// plane (a lattice with one keeps every segment).
cudaError_t launch_build_pairs(const LatticeView* views, const SegRef* segs, const int* n_segs, int capacity,
                               int* emit, int* off, int* tmp, SegRef* tasks, cudaStream_t stream);
// One phase over the paired list (sc.warps_per_block up to 24, sc.grid;
// sc.stages 0: windows loaded into registers, 2-4: copied into shared
// memory that many tasks ahead), a programmatic dependent launch like
// launch_stream_collide; plain BGK lattices.  one: for a set of one
// lattice, a host copy of its view, passed to the kernel by value (NULL:
// the kernel reads the device table views).
cudaError_t launch_stream_collide_pairs(int precision, int phase, int moments, const LatticeView* views,
                                        const LatticeView* one, const SegRef* tasks, const int* n_tasks,
                                        StepConfig sc, cudaStream_t stream);
int stream_collide_pairs_blocks_per_sm(int precision, int phase, int moments, int warps_per_block, int stages);
// Grid barrier state of the persistent kernel (device memory, 16 bytes).
struct StepBarrier {
  unsigned count;  // arrivals since the launch began
  unsigned gen;    // unused
  int error;       // set when a wait gave up (the launch then stops early)
  int extra;       // arrivals awaited beyond the grid: 0, or 1 under the test hook
                   // (lbm_debug_barrier_timeout) so that every wait runs out
};
// lbm_debug_barrier_timeout: the next persistent launches wait for an arrival
// that never comes (the bounded-wait failure path, tested without a fault)
void set_barrier_timeout_test(int on);
int barrier_timeout_test();
cudaError_t launch_stream_collide(int precision, int phase, int moments, const LatticeView* views,
                                  const SegRef* segs, const int* n_segs, StepConfig cfg,
                                  cudaStream_t stream);
int stream_collide_blocks_per_sm(int precision, int phase, int moments, int warps_per_block, int cells_per_thread,
                                 int stages, int features);
// n_pairs time-step pairs (phase A then B, no moments) in one cooperative
// launch with a grid barrier between phases; sc.grid must not exceed
// stream_collide_persistent_grid (every block resident at once), and
// 2 * n_pairs * sc.grid must stay below 2^32.  The
// barrier is reset on the stream first; a barrier wait that gives up sets
// bar->error and ends the launch early.
cudaError_t launch_stream_collide_persistent(int precision, const LatticeView* views, const SegRef* segs,
                                             const int* n_segs, int n_pairs, StepConfig sc, StepBarrier* bar,
                                             cudaStream_t stream);
int stream_collide_persistent_grid(int precision, int warps_per_block, int cells_per_thread);

// ---- on-chip resident time steps (resident.cu) ------------------------------
// A whole solve in one cooperative launch with the populations in shared
// memory: block b of G owns segments [b n / G, (b+1) n / G) of the list
// (at most kResidentMaxOwn), two per warp, and exchanges the rows its
// neighbours need through a halo buffer of tagged words.
constexpr int kResidentMaxOwn = 48;
constexpr int kResidentMaxWarps = kResidentMaxOwn / 2;
// blocks of a resident launch over n segments: as few as hold them, at most one per SM
__host__ __device__ inline int resident_grid(int nseg, int sm_count) {
  const int need = (nseg + kResidentMaxOwn - 1) / kResidentMaxOwn;
  return need < 1 ? 1 : need > sm_count ? sm_count : need;
}
// elements between the two step buffers: words rounded up to 8, a multiple
// of 16 bytes for 16-bit and 32-bit storage
__host__ __device__ inline int resident_buffer_stride(int words) { return (words + 7) & ~7; }
struct ResidentShape {
  int grid;   // blocks
  int warps;  // warps per block (two segments each)
  int words;  // step-buffer size per block (elements of the storage type)
  int pairs;  // ghost rows per block at most
};
// Plan for the current list (out: int[4], device): segments, largest
// step-buffer size, largest ghost-row count, 1 if the list fits.  seg_flags /
// seg_offs: the work-list build's per-word flags and their exclusive scan
// (the list index of every segment word that holds fluid).
cudaError_t launch_resident_plan(const LatticeView* views, const SegRef* segs, const int* n_segs,
                                 const int* seg_word_off, const int* seg_flags, const int* seg_offs, int sm_count,
                                 int* out, cudaStream_t stream);
// Dynamic shared memory of a launch, and the most a block may take.
size_t resident_smem_bytes(int precision, int words, int pairs);
int resident_max_smem();
// n_steps time steps; halo: [2][halo_cap][9][32] words of {value, tag}, tags
// epoch0 + 1 .. epoch0 + n_steps - 1 written by this launch (older tags
// must all be smaller); moments at the last step and at step mom_prev (-1:
// none, else into the *_prev fields); *error is set when a wait gave up.
cudaError_t launch_stream_collide_resident(int precision, const LatticeView* views, const SegRef* segs,
                                           const int* n_segs, const int* seg_word_off, const int* seg_flags,
                                           const int* seg_offs, const ResidentShape& rs,
                                           unsigned long long* halo, int halo_cap, unsigned epoch0, int n_steps,
                                           int mom_prev, int* error, cudaStream_t stream);

// ---- geometry / work-list (worklist.cu) ------------------------------------
cudaError_t launch_pack_mask(const uint8_t* cells, int nx, int ny, int wpr, uint32_t* mask,
                             cudaStream_t stream);
cudaError_t launch_unpack_mask(const uint32_t* mask, int nx, int ny, int wpr, uint8_t* cells,
                               cudaStream_t stream);
// Segment list of a set of lattices: the row segments of rows 1..ny-2 holding
// a fluid cell, lattice by lattice in ascending (y, w) order.  seg_word_off is
// a device copy of the views' seg_word_off plus the total at [n]; scratch
// holds segment_scratch_ints(total) ints, segs room for total entries.
size_t segment_scratch_ints(long long total_words);
// The list buffer holds `capacity` SegRef entries followed by 32 neighbour
// flag words (uint16_t, see kNbE..kNbSE) per entry: those of the cells of
// entry t at flags + 32 t, for phase A.  n_segs[0] receives the count,
// n_segs[1] the capacity (so that kernels find the flags).
cudaError_t launch_build_segments(const LatticeView* views, const int* seg_word_off, int n_lattices,
                                  int total_words, int capacity, int* scratch, SegRef* segs, int* n_segs,
                                  cudaStream_t stream);
inline size_t segment_list_bytes(int capacity) { return (size_t)capacity * (sizeof(SegRef) + 32 * sizeof(uint16_t)); }
__host__ __device__ inline const uint16_t* segment_flags(const SegRef* segs, const int* n_segs) {
  return reinterpret_cast<const uint16_t*>(segs + n_segs[1]);
}
// neighbour solid flags of a cell, bit i-1 = solid(x + c_i), i = 1..8 (E N W S NE NW SW SE);
// kNbMirror marks a cell of row 0 next to a symmetry plane (whose S flag is then set too)
constexpr unsigned kNbE = 1u, kNbN = 2u, kNbW = 4u, kNbS = 8u, kNbNE = 16u, kNbNW = 32u, kNbSW = 64u,
                   kNbSE = 128u, kNbMirror = 256u;
// fluid cells of each lattice into count[l] (zeroed here); word_off as for
// the exchange below
cudaError_t launch_count_fluid(const LatticeView* views, const int* word_off, int n_lattices,
                               int total_words, unsigned long long* count, cudaStream_t stream);
// exclusive scan of n ints; out[n] = total.  Fixed order for any input.
// tmp holds scan_tmp_ints(n) ints.
size_t scan_tmp_ints(long long n);
cudaError_t launch_scan(const int* in, int* out, int n, int* tmp, cudaStream_t stream);
cudaError_t launch_rho_from_drho(const float* drho, float rho0, const uint32_t* mask, int nx, int ny,
                                 int pitch, int wpr, float* rho_dense, cudaStream_t stream);

// ---- reductions (reduce.cu) -------------------------------------------------
constexpr int kResidualBlocks = 128;
// per-lattice results written by launch_finalize, doubles (kResultDoubles each):
//   [0] dp, [1] m_in, [2] residual (or -1), [3] n_in, [4] n_out,
//   [5] sum |du|, [6] sum |u|, [7] nonfinite flag, [8] theta, [9] D_g,
//   [10 .. 10+n_out) m_out
constexpr int kResultDoubles = 10 + LBM_MAX_OUTLETS;
// partials: 2 * kResidualBlocks doubles per lattice
cudaError_t launch_residual_partials(const LatticeView* views, int n_lattices, double* partials,
                                     cudaStream_t stream);
cudaError_t launch_finalize(const LatticeView* views, int n_lattices, const double* partials,
                            int with_residual, double* result, cudaStream_t stream);

// ---- optimality criterion (oc.cu) -------------------------------------------
struct OcScratch {
  int* cnt_f;                 // [total_words]
  int* cnt_s;                 // [total_words]
  int* off_f;                 // [total_words + 1]
  int* off_s;                 // [total_words + 1]
  unsigned long long* key_f;  // [total cells]
  unsigned long long* key_s;  // [total cells]
  int* idx_f;                 // [total cells]
  int* idx_s;                 // [total cells]
  int* sel_f;                 // picks of lattice l from views[l].sel_off (sel_capacity each)
  int* sel_s;
  int* info;                  // [8 per lattice]: n_swapped, nF, nS, NaN flag
  int* scan_tmp;              // scan_tmp_ints(total_words)
};
__host__ __device__ inline int sel_capacity(int nx, int ny) { return (int)((long long)nx * ny / 2 + 1); }
// Selection for every lattice: n_swap (device int[n]) requested per lattice;
// word_off: device copy of the views' word_off plus the total at [n].
cudaError_t launch_oc_select(const LatticeView* views, const int* word_off, int n_lattices,
                             int total_words, const int* n_swap, const OcScratch& s,
                             cudaStream_t stream);
cudaError_t launch_oc_apply(int precision, const LatticeView* views, int n_lattices,
                            const OcScratch& s, cudaStream_t stream);
// The choice alone, on keys and indices already emitted (key_f/idx_f,
// key_s/idx_s in ascending idx order, off_f/off_s their per-word offsets over
// the word space word_off[0 .. n]) -- the D3Q19 exchange uses it with a
// one-entry table whose nx * ny is the cell count.  info must be zeroed
// before the emit stage.
cudaError_t launch_oc_select_only(const LatticeView* views, const int* word_off, int n_lattices, const int* n_swap,
                                  const OcScratch& s, cudaStream_t stream);

// ---- counters / debugging ----------------------------------------------------
void count_launches(uint64_t n);
// message returned by lbm_last_error() on the calling thread
void set_last_error(const std::string& msg);
// LBM_DEBUG_SYNC=1 in the environment: no graphs, synchronise after every
// launch and name the kernel that failed.
bool debug_sync();

#ifdef LBM_CHECK_BOUNDS
// Bounds-checked builds: every global access of the step and reduction
// kernels is checked against its allocation; a violation is printed and the
// access skipped.
__device__ __forceinline__ bool lbm_in_bounds(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  printf("lbm bounds: line %d index %lld extent %lld block %d thread %d\n", line, i, n, blockIdx.x,
         threadIdx.x);
  return false;
}
#define LBM_OK_IDX(i, n) lbm_in_bounds((long long)(i), (long long)(n), __LINE__)
#else
#define LBM_OK_IDX(i, n) true
#endif

}  // namespace lbm
