// Fused D2Q9 stream + collide on a single lattice (AA access pattern).
//
// Method: lattice BGK update of Eq. 1 with the second-order equilibrium of
// Sec. 2.1 and the moments of Eq. 2; halfway bounce-back on solid cells, the
// parabolic velocity inlet, and the constant-density or zero-gradient outlet
// of Sec. 3.3 (ports regularised or plain Zou-He) -- all fused into one pass
// per time step.
//
// Storage.  Populations are kept shifted, g_i = f_i - w_i rho0, in nine planes
// F[i][y][x] (row pitch `pitch`), as FP32, BF16 or FP16; arithmetic is FP32.
// The canonical layout between steps is F[i][cell] = post-collision g_i of
// that cell.  Steps come in pairs:
//   phase A  cell x pulls g_i from F[i][x - c_i] (or, where x - c_i is solid,
//            the reversed F[opp(i)][x]: bounce-back), relaxes, and writes each
//            outgoing g_i into F[opp(i)][x + c_i] -- the very slot it read for
//            direction opp(i) -- or, where x + c_i is solid, into F[i][x];
//   phase B  cell x finds its incoming g_i in F[opp(i)][x], relaxes, and
//            writes g_i back to F[i][x]: the canonical layout again.
// Each slot is read and then written by exactly one thread per phase, so the
// pair needs one lattice and no barrier.  Solid cells are never read.
//
// Thread mapping.  Each warp takes one or two consecutive row segments (the
// 32 cells of one mask word each) from a device-resident list holding only
// segments with fluid cells; lane l handles cell 32w + l of each, so every
// plane access of a warp is one contiguous 32-element row segment (shifted by
// at most one element).  With two segments (two cells per thread) all 18
// loads are in flight before the first cell is updated.  Warps stride over
// the list; the list may span several lattices (batches).  Consecutive steps
// are programmatic dependent launches: a step's warps load their segment,
// descriptor and mask words while the previous step is still finishing, and
// wait for it only before touching populations.  Alternatively one
// cooperative launch runs all steps of a solve with grid barriers between
// phases (the persistent kernel).
#include <cstddef>

#include "d2q9_cell.cuh"

namespace lbm {
namespace {

// population access with optional bounds checks (offset in elements from F)
#define FLD(off) (LBM_OK_IDX((off), s.fe) ? (CG ? P::ldcg(F + (off)) : P::ld(F + (off))) : 0.0f)
#define FST(off, v)                                     \
  do {                                                  \
    if (LBM_OK_IDX((off), s.fe)) P::st(F + (off), (v)); \
  } while (0)

// Kernel builds by feature (template bit mask): kFeatModels -- collision
// models beyond BGK; kFeatMirror -- a symmetry plane below row 0.  The plain
// build has neither, so the common path keeps its registers and branches.
constexpr int kFeatModels = 1, kFeatMirror = 2;

// neighbour solid flags (built with the work-list), bit i-1 = solid(x + c_i),
// i = 1..8 (E N W S NE NW SW SE); kMirror marks a cell of row 0 next to a
// symmetry plane
constexpr unsigned kE = kNbE, kN = kNbN, kW = kNbW, kS = kNbS, kNE = kNbNE, kNW = kNbNW, kSW = kNbSW,
                   kSE = kNbSE, kMirror = kNbMirror;

// Threads per block at most, by cells per thread: the register budget per
// thread is 64 with one cell (1024 threads per SM), 80 with two (768).  The
// per-phase kernel may take the whole budget in one block (one block per SM
// costs less to schedule at every launch than three or four smaller ones),
// the persistent kernel in two or three.
__host__ __device__ constexpr int max_step_threads(int cpt) { return cpt == 1 ? 1024 : 768; }
__host__ __device__ constexpr int max_persistent_threads(int cpt) { return cpt == 1 ? 512 : 256; }
__host__ __device__ constexpr int min_persistent_blocks(int cpt) { return cpt == 1 ? 2 : 3; }

// What one lane knows about its cell of one row segment before touching
// populations: everything here comes from the segment list, the lattice
// descriptor and the mask, none of which a time step writes.
template <class T>
struct SegCtx {
  const LatticeView* L;
  T* F;
  int y, c, pitch, pl;
  unsigned nb;  // solid flags of the 8 neighbours (phase A)
  bool fluid, inlet, outlet;
  float rho0, omega;
  int rule;      // outlet rule
  long long fe;  // population elements (bounds-checked builds)
};

// NBMASK: form the neighbour flags from the mask words at every precision
// (for task lists whose entries are not the segment list's, whose flags
// array is indexed by segment number).
template <class T, int PHASE, int FEAT = 0, bool NBMASK = false>
__device__ __forceinline__ void seg_prologue(const LatticeView* __restrict__ views, const SegRef sr, bool valid,
                                             const int lane, SegCtx<T>& s, const uint16_t* __restrict__ nbs,
                                             int t) {
  const LatticeView* __restrict__ L = views + (valid ? sr.lattice : 0);
  const int y = sr.yw >> kSegWordBits;
  const int w = sr.yw & ((1 << kSegWordBits) - 1);
#ifdef LBM_CHECK_BOUNDS
  if (valid && (sr.lattice < 0 || y < 1 || y > L->ny - 2 || w < 0 || w >= L->wpr)) {
    if (lane == 0) printf("lbm bounds: bad segment: lattice %d y %d w %d\n", sr.lattice, y, w);
    valid = false;
    L = views;
  }
#endif
  s.L = L;
  s.F = static_cast<T*>(L->f);
  s.pitch = L->pitch;
  s.pl = (int)L->plane;  // 32-bit element offsets: lattices are limited to 9 * plane < 2^31
  s.fe = L->f_elems;
  s.rho0 = L->rho0;
  s.omega = L->omega;
  s.rule = L->outlet_rule;
  s.nb = 0;
  if (!valid) {
    s.y = 0;
    s.c = 0;
    s.fluid = s.inlet = s.outlet = false;
    return;
  }
  const int ms = mask_stride(L->wpr);
  const uint32_t* mr = L->mask + (long long)y * ms;
  const uint32_t mc = mr[w];
  const int x = (w << 5) + lane;
  s.y = y;
  s.c = y * s.pitch + x;
  s.fluid = !((mc >> lane) & 1u);  // bits beyond nx are set (solid)
  s.inlet = (x == 0);
  s.outlet = (x == L->nx - 1);
  if (PHASE == 0) {
    if (sizeof(T) == 4 && !NBMASK) {
      // FP32: the neighbour flags built with the work-list (one coalesced
      // 16-bit word per cell, by task number, the symmetry-plane mark below
      // included; builds without the plane drop it).  The 16-bit builds form
      // them from the mask words instead: for them the extra bytes cost more
      // than the saved instructions (measured).
      s.nb = nbs[(long long)t * 32 + lane];
      if (!(FEAT & kFeatMirror)) s.nb &= ~kMirror;
    } else {
      // padded mask: words w-1 and w+1 of rows y-1..y+1 always exist and are
      // solid outside the lattice
      const uint32_t* rn = mr + ms;
      const uint32_t* rs = mr - ms;
      const uint32_t mn = rn[w], msth = rs[w];
      const uint32_t eC = __funnelshift_r(mc, mr[w + 1], 1), wC = __funnelshift_l(mr[w - 1], mc, 1);
      const uint32_t eN = __funnelshift_r(mn, rn[w + 1], 1), wN = __funnelshift_l(rn[w - 1], mn, 1);
      const uint32_t eS = __funnelshift_r(msth, rs[w + 1], 1), wS = __funnelshift_l(rs[w - 1], msth, 1);
      s.nb = ((eC >> lane) & 1u) | (((mn >> lane) & 1u) << 1) | (((wC >> lane) & 1u) << 2) |
             (((msth >> lane) & 1u) << 3) | (((eN >> lane) & 1u) << 4) | (((wN >> lane) & 1u) << 5) |
             (((wS >> lane) & 1u) << 6) | (((eS >> lane) & 1u) << 7);
      // Symmetry plane half a cell below row 0 (the padding row below holds
      // row 0's mirror image, so the SW / SE flags already tell whether the
      // image cell is solid).  What row 0 sends across the plane comes back
      // reflected: straight down returns as straight up into the same cell
      // -- the bounce-back slot -- and a diagonal returns into the row-0
      // neighbour it was heading past: SW into (x-1, 0) as NW, SE into
      // (x+1, 0) as NE.
      if ((FEAT & kFeatMirror) && y == 0 && L->mirror) s.nb |= kS | kMirror;
    }
  }
}

// The nine incoming populations of the lane's cell (0 where unknown or solid).
// CG: read through L2 only (the persistent kernel: within one launch a slot
// written by another block must not be served from this SM's L1).
template <class T, int PHASE, bool CG, int FEAT = 0>
__device__ __forceinline__ void seg_load(const SegCtx<T>& s, float (&g)[9]) {
  using P = Pop<T>;
  const T* __restrict__ F = s.F;
  const int c = s.c, pl = s.pl, pitch = s.pitch;
  const unsigned nb = s.nb;
#pragma unroll
  for (int i = 0; i < 9; ++i) g[i] = 0.0f;
  if (!s.fluid) return;
  if (PHASE == 0) {
    g[0] = FLD(c);
    g[2] = (nb & kS) ? FLD(4 * pl + c) : FLD(2 * pl + c - pitch);
    g[4] = (nb & kN) ? FLD(2 * pl + c) : FLD(4 * pl + c + pitch);
    if (!s.inlet) {  // sources on the west side (unknown at the inlet)
      g[1] = (nb & kW) ? FLD(3 * pl + c) : FLD(1 * pl + c - 1);
      g[5] = (nb & kSW) ? FLD(7 * pl + c)
             : ((FEAT & kFeatMirror) && (nb & kMirror)) ? FLD(8 * pl + c - 1) : FLD(5 * pl + c - pitch - 1);
      g[8] = (nb & kNW) ? FLD(6 * pl + c) : FLD(8 * pl + c + pitch - 1);
    }
    if (!s.outlet) {  // sources on the east side (unknown at the outlet)
      g[3] = (nb & kE) ? FLD(1 * pl + c) : FLD(3 * pl + c + 1);
      g[6] = (nb & kSE) ? FLD(8 * pl + c)
             : ((FEAT & kFeatMirror) && (nb & kMirror)) ? FLD(7 * pl + c + 1) : FLD(6 * pl + c - pitch + 1);
      g[7] = (nb & kNE) ? FLD(5 * pl + c) : FLD(7 * pl + c + pitch + 1);
    }
  } else {
    g[0] = FLD(c);
    g[2] = FLD(4 * pl + c);
    g[4] = FLD(2 * pl + c);
    if (!s.inlet) {
      g[1] = FLD(3 * pl + c);
      g[5] = FLD(7 * pl + c);
      g[8] = FLD(6 * pl + c);
    }
    if (!s.outlet) {
      g[3] = FLD(1 * pl + c);
      g[6] = FLD(8 * pl + c);
      g[7] = FLD(5 * pl + c);
    }
  }
}

// Boundary rules, collision and stores of the lane's cell.  Every lane of the
// warp calls it (the zero-gradient outlet shuffles across lanes).
// OPQ: recompute the store offsets after the collision instead of keeping
// the load offsets alive across it (fewer registers: pays where two cells per
// thread press on the budget, costs a little elsewhere -- measured).
template <class T, int PHASE, int MOM, int FEAT, bool OPQ = false>
__device__ __forceinline__ void seg_update(const SegCtx<T>& s, float (&g)[9]) {
  using P = Pop<T>;
  const LatticeView* __restrict__ L = s.L;
  const int rule = s.rule;
  if (rule == LBM_OUT_NEUMANN) {
    // zero-gradient outlet: the unknown g3, g6, g7 of cell (nx-1, y) are the
    // streamed g3, g6, g7 of cell (nx-2, y), held by the lane to the left
    // (nx mod 32 != 1 is required with this rule, so both cells are in
    // this warp's row segment).
    const float n3 = __shfl_up_sync(0xffffffffu, g[3], 1);
    const float n6 = __shfl_up_sync(0xffffffffu, g[6], 1);
    const float n7 = __shfl_up_sync(0xffffffffu, g[7], 1);
    if (s.outlet) {
      g[3] = n3;
      g[6] = n6;
      g[7] = n7;
    }
  }
  if (!s.fluid) return;
  const float rho0 = s.rho0;
  if (s.inlet) {
    inlet_rule(g, L->u_in[s.y], rho0, L->port_scheme);
  } else if (s.outlet && rule == LBM_OUT_CONST_RHO) {
    outlet_rule(g, rho0, L->port_scheme);
  }
  float drho, ux, uy;
  if ((FEAT & kFeatModels) && L->collision != LBM_COLLIDE_BGK)  // the plain build skips this branch
    collide_other(g, rho0, s.omega, L->collision, L->c_smag, drho, ux, uy);
  else
    bgk(g, rho0, s.omega, drho, ux, uy);

  T* __restrict__ F = s.F;
  int c = s.c, pl = s.pl, pitch = s.pitch;
  if (OPQ) asm volatile("" : "+r"(c), "+r"(pl), "+r"(pitch));
  const unsigned nb = s.nb;
  if (PHASE == 0) {
    FST(c, g[0]);
    if (nb & kN) FST(2 * pl + c, g[2]); else FST(4 * pl + c + pitch, g[2]);
    if (nb & kS) FST(4 * pl + c, g[4]); else FST(2 * pl + c - pitch, g[4]);
    if (!s.outlet) {  // destinations on the east side leave through the outlet
      if (nb & kE) FST(1 * pl + c, g[1]); else FST(3 * pl + c + 1, g[1]);
      if (nb & kNE) FST(5 * pl + c, g[5]); else FST(7 * pl + c + pitch + 1, g[5]);
      if (nb & kSE) FST(8 * pl + c, g[8]);
      else if ((FEAT & kFeatMirror) && (nb & kMirror)) FST(7 * pl + c + 1, g[8]);
      else FST(6 * pl + c - pitch + 1, g[8]);
    }
    if (!s.inlet) {  // destinations on the west side leave through the inlet
      if (nb & kW) FST(3 * pl + c, g[3]); else FST(1 * pl + c - 1, g[3]);
      if (nb & kNW) FST(6 * pl + c, g[6]); else FST(8 * pl + c + pitch - 1, g[6]);
      if (nb & kSW) FST(7 * pl + c, g[7]);
      else if ((FEAT & kFeatMirror) && (nb & kMirror)) FST(8 * pl + c - 1, g[7]);
      else FST(5 * pl + c - pitch - 1, g[7]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) FST(i * pl + c, g[i]);
    if (MOM != 0 && LBM_OK_IDX(c, pl)) {
      L->drho[c] = drho;
      (MOM == 1 ? L->ux : L->ux_prev)[c] = ux;
      (MOM == 1 ? L->uy : L->uy_prev)[c] = uy;
    }
  }
}

// One phase on CPT consecutive segments of the list: their loads are all
// issued before the first cell is updated (more bytes in flight per thread).
template <class T, int PHASE, int MOM, int CPT, bool CG, int FEAT = 0>
__device__ __forceinline__ void phase_task(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                           const uint16_t* __restrict__ nbs, int nseg, int task, int lane,
                                           bool& waited, const SegRef* pre = nullptr) {
  SegCtx<T> s[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int idx = task * CPT + k;
    const bool valid = CPT == 1 || idx < nseg;  // one segment per task: task < nseg already
    seg_prologue<T, PHASE, FEAT>(views, (CPT == 1 && pre) ? *pre : segs[valid ? idx : 0], valid, lane, s[k], nbs,
                                 valid ? idx : 0);
  }
  if (!waited) {  // warp-uniform: populations of the previous step are final from here on
    asm volatile("griddepcontrol.wait;" ::: "memory");
    waited = true;
  }
  float g[CPT][9];
#pragma unroll
  for (int k = 0; k < CPT; ++k) seg_load<T, PHASE, CG, FEAT>(s[k], g[k]);
#pragma unroll
  for (int k = 0; k < CPT; ++k) seg_update<T, PHASE, MOM, FEAT, (CPT > 1)>(s[k], g[k]);
}

// One phase of one time step over the whole segment list.  Launched as a
// programmatic dependent of the previous step: descriptors, segments and
// masks are read before waiting for it, populations after.
// FEAT: the features some lattice of the set uses (kFeatModels, kFeatMirror);
// each combination is a separate build, so that the plain kernels keep their
// register budget and straight-line loads.
template <class T, int PHASE, int MOM, int CPT, int FEAT>
__global__ void __launch_bounds__(max_step_threads(CPT), 1)
    k_stream_collide(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                     const int* __restrict__ n_segs) {
  // The next time step may be scheduled now; it reads populations only after
  // waiting for this grid to complete.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int nseg = *n_segs;
  const uint16_t* nbs = segment_flags(segs, n_segs);
  const int ntask = (nseg + CPT - 1) / CPT;
  const int wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  bool waited = false;
  if (CPT == 1) {
    // one segment per task: the next task's list entry is loaded while this
    // task's populations are in flight
    int t = blockIdx.x * wpb + (threadIdx.x >> 5);
    SegRef nxt = t < ntask ? segs[t] : SegRef{0, 0};
    for (; t < ntask; t += stride) {
      const SegRef cur = nxt;
      if (t + stride < ntask) nxt = segs[t + stride];
      phase_task<T, PHASE, MOM, CPT, false, FEAT>(views, segs, nbs, nseg, t, lane, waited, &cur);
    }
  } else {
    for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < ntask; t += stride)
      phase_task<T, PHASE, MOM, CPT, false, FEAT>(views, segs, nbs, nseg, t, lane, waited);
  }
  // every thread waits once, so this grid completes only after the previous
  // one (the next step relies on that)
  if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
}


// ---- compacted tasks: 32 consecutive fluid cells per warp ----------------
//
// On lattices of narrow channels a row segment holds few fluid cells (a
// quarter to a third of the lanes idle on the batched candidates), and its
// partly used 32-byte sectors cost DRAM bytes.  Here a warp takes 32
// consecutive entries of the set's fluid-cell list: every lane has a cell,
// and the cells run along x within each run of fluid, so the plane accesses
// stay contiguous pieces.  The per-cell work is that of the segment kernel
// (seg_load, seg_update) with the cell's offset and neighbour flags from its
// list entry.
template <class T, int PHASE, int MOM>
__global__ void __launch_bounds__(1024, 1)
    k_stream_collide_cells(const LatticeView* __restrict__ views, const CellRef* __restrict__ cells,
                           const int* __restrict__ n_segs, const int* __restrict__ cpre) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int ncell = cpre[n_segs[0]];
  const int ntask = (ncell + 31) >> 5;
  const int wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  bool waited = false;
  for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < ntask; t += stride) {
    const int e = (t << 5) + lane;
    const bool valid = e < ncell;
    const CellRef cr = cells[valid ? e : 0];
    const LatticeView* __restrict__ L = views + (cr.meta & ((1u << kCellLatticeBits) - 1u));
    SegCtx<T> s;
    s.L = L;
    s.F = static_cast<T*>(L->f);
    s.pitch = L->pitch;
    s.pl = (int)L->plane;
    s.fe = L->f_elems;
    s.rho0 = L->rho0;
    s.omega = L->omega;
    s.rule = L->outlet_rule;
    s.c = cr.c;
    s.nb = (cr.meta >> kCellLatticeBits) & 0x1ffu;
    s.fluid = valid;
    s.inlet = valid && ((cr.meta >> 29) & 1u);
    s.outlet = valid && ((cr.meta >> 30) & 1u);
    s.y = s.inlet ? cr.c / s.pitch : 0;  // the inlet rule looks up the row's speed
    if (!waited) {  // warp-uniform: populations of the previous step are final from here on
      asm volatile("griddepcontrol.wait;" ::: "memory");
      waited = true;
    }
    float g[9];
    seg_load<T, PHASE, false, 0>(s, g);
    seg_update<T, PHASE, MOM, 0>(s, g);
  }
  if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class T>
void* pick_cells(int phase, int moments) {
  if (phase == 0) return (void*)k_stream_collide_cells<T, 0, 0>;
  if (moments == 1) return (void*)k_stream_collide_cells<T, 1, 1>;
  if (moments == 2) return (void*)k_stream_collide_cells<T, 1, 2>;
  return (void*)k_stream_collide_cells<T, 1, 0>;
}


// ---- paired tasks: interior 64-cell windows, two cells a lane ------------
//
// A window of 64 cells (row y, mask words 2p and 2p+1) is interior when its
// cells and all eight neighbours of each are fluid: it has no bounce-back
// and no port cell.  Lane l takes cells x = 64p + 2l and x + 1, so that
// every plane access is one aligned pair of elements (one memory
// instruction for two cells).  Phase B reads and writes the cells' own
// slots.  Phase A's one-column shifts pass one half of each pair to the
// neighbouring lane by a shuffle.  A pull from the west (c_x = +1) takes
// the upper half of lane l-1's pair, and a pull from the east the lower
// half of lane l+1's.  The pushes back pair each lane's value with the
// neighbour's.  Lanes 0 and 31 reach one element past the window.
// Segments outside interior windows are taken by the same launch, one per
// warp, exactly as by k_stream_collide.  The per-cell arithmetic is the
// same everywhere, so every task shape gives the same bits.
#define PLD2(off, lo, hi)                                         \
  do {                                                            \
    if (LBM_OK_IDX((off), fe) && LBM_OK_IDX((off) + 1, fe)) {     \
      P2::ld(F + (off), lo, hi);                                  \
    } else {                                                      \
      lo = 0.0f;                                                  \
      hi = 0.0f;                                                  \
    }                                                             \
  } while (0)
#define PST2(off, lo, hi)                                                             \
  do {                                                                                \
    if (LBM_OK_IDX((off), fe) && LBM_OK_IDX((off) + 1, fe)) P2::st(F + (off), lo, hi); \
  } while (0)
#define PLD1(off) (LBM_OK_IDX((off), fe) ? P::ld(F + (off)) : 0.0f)
#define PST1(off, v)                                   \
  do {                                                 \
    if (LBM_OK_IDX((off), fe)) P::st(F + (off), (v)); \
  } while (0)

// Where a window's populations come from, by slot i (the population g_i of
// the lane's two cells): phase A reads plane i of row y - c_iy (the x
// shift is made by the shuffles of pair_assemble), phase B plane opp(i) of
// row y.
__host__ __device__ constexpr int pair_plane(int phase, int i) {
  return phase == 0 ? i : (i == 0 ? 0 : i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
__host__ __device__ constexpr int pair_row(int phase, int i) {  // row offset of the source, in rows
  return phase == 0 ? (i == 2 || i == 5 || i == 6 ? -1 : i == 4 || i == 7 || i == 8 ? 1 : 0) : 0;
}
// One element past the window (phase A, slot k = 0, 1, 2): lane 0 reads
// direction {1, 5, 8}[k] at x = 64p - 1, lane 31 direction {3, 6, 7}[k] at
// x = 64p + 64 (2 past its lower cell), both in the row of the slot.
__host__ __device__ constexpr int pair_edge_plane(bool first, int k) {
  return first ? (k == 0 ? 1 : k == 1 ? 5 : 8) : (k == 0 ? 3 : k == 1 ? 6 : 7);
}
__host__ __device__ constexpr int pair_edge_row(int k) { return k == 0 ? 0 : k == 1 ? -1 : 1; }

// The nine pairs of a window, straight from global memory into a (lower
// cells) and b (upper cells), and the phase-A edge elements e.
template <class T, int PHASE>
__device__ __forceinline__ void pair_load(const T* __restrict__ F, const int c, const int pitch, const int pl,
                                          const long long fe, const int lane, float (&a)[9], float (&b)[9],
                                          float (&e)[3]) {
  using P = Pop<T>;
  using P2 = Pop2<T>;
  (void)fe;
#pragma unroll
  for (int i = 0; i < 9; ++i) PLD2(pair_plane(PHASE, i) * pl + c + pair_row(PHASE, i) * pitch, a[i], b[i]);
  e[0] = e[1] = e[2] = 0.0f;
  if (PHASE == 0 && (lane == 0 || lane == 31)) {
    const bool first = lane == 0;
    const int d = first ? -1 : 2;
#pragma unroll
    for (int k = 0; k < 3; ++k) e[k] = PLD1(pair_edge_plane(first, k) * pl + c + pair_edge_row(k) * pitch + d);
  }
}

// Phase A's one-column shifts: a pull from the west (1, 5, 8) takes the
// upper half of lane l-1's pair for the lower cell and the lower half of
// the lane's own pair for the upper cell; a pull from the east (3, 6, 7)
// the own upper half for the lower cell and lane l+1's lower half for the
// upper cell; lanes 0 and 31 take the edge elements instead.
template <int PHASE>
__device__ __forceinline__ void pair_assemble(float (&a)[9], float (&b)[9], const float (&e)[3], const int lane) {
  if (PHASE != 0) return;
  constexpr unsigned kAll = 0xffffffffu;
  const bool first = lane == 0, last = lane == 31;
  const int west[3] = {1, 5, 8}, east[3] = {3, 6, 7};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = west[k];
    const float u = __shfl_up_sync(kAll, b[i], 1);
    b[i] = a[i];
    a[i] = first ? e[k] : u;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = east[k];
    const float d = __shfl_down_sync(kAll, a[i], 1);
    a[i] = b[i];
    b[i] = last ? e[k] : d;
  }
}

// Collision of both cells and the stores of the window.
template <class T, int PHASE, int MOM>
__device__ __forceinline__ void pair_finish(const LatticeView* __restrict__ L, T* __restrict__ F, const int c,
                                            const int pitch, const int pl, const long long fe, const int lane,
                                            float (&a)[9], float (&b)[9]) {
  using P = Pop<T>;
  using P2 = Pop2<T>;
  constexpr unsigned kAll = 0xffffffffu;
  (void)fe;
  const bool first = lane == 0, last = lane == 31;
  const float rho0 = L->rho0, omega = L->omega;
  float dra, uxa, uya, drb, uxb, uyb;
  bgk2(a, b, rho0, omega, dra, uxa, uya, drb, uxb, uyb);
  if (PHASE == 0) {
    // pushes g_i to F[opp(i)] at x + c_i
    PST2(c, a[0], b[0]);
    PST2(4 * pl + c + pitch, a[2], b[2]);
    PST2(2 * pl + c - pitch, a[4], b[4]);
    // east-going (1, 5, 8): the pair at x takes lane l-1's upper cell and
    // this lane's lower one; lane 0's lower half is another task's
    const float v1 = __shfl_up_sync(kAll, b[1], 1), v5 = __shfl_up_sync(kAll, b[5], 1),
                v8 = __shfl_up_sync(kAll, b[8], 1);
    if (!first) {
      PST2(3 * pl + c, v1, a[1]);
      PST2(7 * pl + c + pitch, v5, a[5]);
      PST2(6 * pl + c - pitch, v8, a[8]);
    }
    // west-going (3, 6, 7): the pair at x takes this lane's upper cell and
    // lane l+1's lower one; lane 31's upper half is another task's
    const float v3 = __shfl_down_sync(kAll, a[3], 1), v6 = __shfl_down_sync(kAll, a[6], 1),
                v7 = __shfl_down_sync(kAll, a[7], 1);
    if (!last) {
      PST2(1 * pl + c, b[3], v3);
      PST2(8 * pl + c + pitch, b[6], v6);
      PST2(5 * pl + c - pitch, b[7], v7);
    }
    // the single elements: lane 0's lower cell east into x + 1 and west
    // into 64p - 1; lane 31's upper cell east into 64p + 64 and west into
    // its own lower slot
    if (first || last) {
      const int de = first ? 1 : 2, dw = first ? -1 : 0;
      PST1(3 * pl + c + de, first ? a[1] : b[1]);
      PST1(7 * pl + c + pitch + de, first ? a[5] : b[5]);
      PST1(6 * pl + c - pitch + de, first ? a[8] : b[8]);
      PST1(1 * pl + c + dw, first ? a[3] : b[3]);
      PST1(8 * pl + c + pitch + dw, first ? a[6] : b[6]);
      PST1(5 * pl + c - pitch + dw, first ? a[7] : b[7]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) PST2(i * pl + c, a[i], b[i]);
    if (MOM != 0 && LBM_OK_IDX(c + 1, pl)) {
      *reinterpret_cast<float2*>(L->drho + c) = make_float2(dra, drb);
      *reinterpret_cast<float2*>((MOM == 1 ? L->ux : L->ux_prev) + c) = make_float2(uxa, uxb);
      *reinterpret_cast<float2*>((MOM == 1 ? L->uy : L->uy_prev) + c) = make_float2(uya, uyb);
    }
  }
}

template <class T, int PHASE, int MOM>
__device__ __forceinline__ void pair_task(const LatticeView* __restrict__ L, const int y, const int p,
                                          const int lane, bool& waited) {
  T* __restrict__ F = static_cast<T*>(L->f);
  const int pitch = L->pitch, pl = (int)L->plane;
  const long long fe = L->f_elems;  // bounds-checked builds
  const int c = y * pitch + (p << 6) + 2 * lane;  // the lane's lower cell x (even)
  if (!waited) {  // warp-uniform: populations of the previous step are final from here on
    asm volatile("griddepcontrol.wait;" ::: "memory");
    waited = true;
  }
  float a[9], b[9], e[3];  // cells x and x + 1
  pair_load<T, PHASE>(F, c, pitch, pl, fe, lane, a, b, e);
  pair_assemble<PHASE>(a, b, e, lane);
  pair_finish<T, PHASE, MOM>(L, F, c, pitch, pl, fe, lane, a, b);
}
#undef PLD2
#undef PST2
#undef PLD1
#undef PST1

// One phase over the paired task list (interior windows and the other
// segments, in list order); one task per warp at a time, the next task's
// entry loaded while this one's populations are in flight.  ONE: a set of
// one lattice whose descriptor is a kernel parameter (uniform values from
// the constant bank instead of per-task loads of the table entry).
template <class T, int PHASE, int MOM, bool ONE>
__device__ __forceinline__ void pairs_loop(const LatticeView* __restrict__ views, const SegRef* __restrict__ tasks,
                                           const int* __restrict__ n_tasks) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int ntask = *n_tasks;
  const int wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  bool waited = false;
  int t = blockIdx.x * wpb + (threadIdx.x >> 5);
  SegRef nxt = t < ntask ? tasks[t] : SegRef{0, 0};
  for (; t < ntask; t += stride) {
    SegRef cur = nxt;
    if (t + stride < ntask) nxt = tasks[t + stride];
    if (cur.lattice & kPairTask) {
      pair_task<T, PHASE, MOM>(views + (ONE ? 0 : (cur.lattice & ~kPairTask)), cur.yw >> kSegWordBits,
                               cur.yw & ((1 << kSegWordBits) - 1), lane, waited);
    } else {
      if (ONE) cur.lattice = 0;
      SegCtx<T> s;
      seg_prologue<T, PHASE, 0, true>(views, cur, true, lane, s, nullptr, 0);
      if (!waited) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        waited = true;
      }
      float g[9];
      seg_load<T, PHASE, false, 0>(s, g);
      seg_update<T, PHASE, MOM, 0>(s, g);
    }
  }
  if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class T, int PHASE, int MOM>
__global__ void __launch_bounds__(max_step_threads(2), 1)
    k_stream_collide_pairs(const LatticeView* __restrict__ views, const SegRef* __restrict__ tasks,
                           const int* __restrict__ n_tasks) {
  pairs_loop<T, PHASE, MOM, false>(views, tasks, n_tasks);
}

template <class T, int PHASE, int MOM>
__global__ void __launch_bounds__(max_step_threads(2), 1)
    k_stream_collide_pairs_one(const __grid_constant__ LatticeView one, const SegRef* __restrict__ tasks,
                               const int* __restrict__ n_tasks) {
  pairs_loop<T, PHASE, MOM, true>(&one, tasks, n_tasks);
}

template <class T>
void* pick_pairs(int phase, int moments, bool one) {
  if (one) {
    if (phase == 0) return (void*)k_stream_collide_pairs_one<T, 0, 0>;
    if (moments == 1) return (void*)k_stream_collide_pairs_one<T, 1, 1>;
    if (moments == 2) return (void*)k_stream_collide_pairs_one<T, 1, 2>;
    return (void*)k_stream_collide_pairs_one<T, 1, 0>;
  }
  if (phase == 0) return (void*)k_stream_collide_pairs<T, 0, 0>;
  if (moments == 1) return (void*)k_stream_collide_pairs<T, 1, 1>;
  if (moments == 2) return (void*)k_stream_collide_pairs<T, 1, 2>;
  return (void*)k_stream_collide_pairs<T, 1, 0>;
}

// ---- staged variant: populations copied into shared memory ahead of use ----
//
// Each warp keeps NS stages of one row segment each in shared memory (nine
// population words and two context words per lane).  While it updates the
// segment in stage k, the copies for the next NS-1 segments of its list are
// in flight (cp.async, 4 bytes per lane and direction: the word holding the
// lane's element), so the bytes in flight per SM no longer depend on the
// registers a thread can hold.

// Element offset (from F) of direction i's incoming population for the cell
// at offset c, or -1 where it is unknown (the open side of a port cell).
// The same selection as seg_load.
template <int PHASE>
__device__ __forceinline__ int src_off(const int i, const int c, const int pitch, const int pl, const unsigned nb,
                                       const bool inlet, const bool outlet) {
  if (PHASE == 1) {
    switch (i) {
      case 0: return c;
      case 1: return inlet ? -1 : 3 * pl + c;
      case 2: return 4 * pl + c;
      case 3: return outlet ? -1 : 1 * pl + c;
      case 4: return 2 * pl + c;
      case 5: return inlet ? -1 : 7 * pl + c;
      case 6: return outlet ? -1 : 8 * pl + c;
      case 7: return outlet ? -1 : 5 * pl + c;
      default: return inlet ? -1 : 6 * pl + c;
    }
  }
  switch (i) {
    case 0: return c;
    case 1: return inlet ? -1 : (nb & kW) ? 3 * pl + c : 1 * pl + c - 1;
    case 2: return (nb & kS) ? 4 * pl + c : 2 * pl + c - pitch;
    case 3: return outlet ? -1 : (nb & kE) ? 1 * pl + c : 3 * pl + c + 1;
    case 4: return (nb & kN) ? 2 * pl + c : 4 * pl + c + pitch;
    case 5: return inlet ? -1 : (nb & kSW) ? 7 * pl + c : 5 * pl + c - pitch - 1;
    case 6: return outlet ? -1 : (nb & kSE) ? 8 * pl + c : 6 * pl + c - pitch + 1;
    case 7: return outlet ? -1 : (nb & kNE) ? 5 * pl + c : 7 * pl + c + pitch + 1;
    default: return inlet ? -1 : (nb & kNW) ? 6 * pl + c : 8 * pl + c + pitch - 1;
  }
}

constexpr int kStageWords = 9 * 32 + 2 * 32;  // populations, then cell offset and flags per lane

// Copy the 4-byte word holding element `off` of F into shared memory
// (zero-filled, nothing read, where off < 0).
template <class T>
__device__ __forceinline__ void cp_async_word(uint32_t* dst, const T* F, int off, long long fe) {
  if (off >= 0 && !LBM_OK_IDX(off, fe)) off = -1;
  const char* src = reinterpret_cast<const char*>(F) + ((off < 0 ? 0ll : (long long)off * (long long)sizeof(T)) & ~3ll);
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = off < 0 ? 0 : 4;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

template <class T, int PHASE>
__device__ __forceinline__ void stage_issue(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                            const uint16_t* __restrict__ nbs, int nseg, int t, int lane,
                                            uint32_t* buf) {
  const bool valid = t < nseg;
  const SegRef sr = segs[valid ? t : 0];
  SegCtx<T> s;
  seg_prologue<T, PHASE>(views, sr, valid, lane, s, nbs, valid ? t : 0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int off = s.fluid ? src_off<PHASE>(i, s.c, s.pitch, s.pl, s.nb, s.inlet, s.outlet) : -1;
    cp_async_word<T>(buf + i * 32 + lane, s.F, off, s.fe);
  }
  buf[9 * 32 + lane] = (uint32_t)s.c;
  buf[10 * 32 + lane] = s.nb | ((uint32_t)s.fluid << 9) | ((uint32_t)s.inlet << 10) | ((uint32_t)s.outlet << 11) |
                        ((uint32_t)(valid ? sr.lattice : 0) << 12);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <class T, int PHASE, int MOM>
__device__ __forceinline__ void stage_consume(const LatticeView* __restrict__ views, const uint32_t* buf, int lane) {
  using P = Pop<T>;
  const uint32_t fl = buf[10 * 32 + lane];
  SegCtx<T> s;
  const LatticeView* __restrict__ L = views + (fl >> 12);
  s.L = L;
  s.F = static_cast<T*>(L->f);
  s.pitch = L->pitch;
  s.pl = (int)L->plane;
  s.fe = L->f_elems;
  s.rho0 = L->rho0;
  s.omega = L->omega;
  s.rule = L->outlet_rule;
  s.c = (int)buf[9 * 32 + lane];
  s.nb = fl & 0x1ffu;
  s.fluid = (fl >> 9) & 1u;
  s.inlet = (fl >> 10) & 1u;
  s.outlet = (fl >> 11) & 1u;
  s.y = s.inlet ? s.c / s.pitch : 0;  // the inlet rule looks up the row's speed
  float g[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int off = s.fluid ? src_off<PHASE>(i, s.c, s.pitch, s.pl, s.nb, s.inlet, s.outlet) : -1;
    g[i] = off < 0 ? 0.0f : P::from_word(buf[i * 32 + lane], off & 1);
  }
  seg_update<T, PHASE, MOM, 0>(s, g);
}

template <int NS>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");
}

template <class T, int PHASE, int MOM, int NS>
__global__ void __launch_bounds__(512, 2)
    k_stream_collide_staged(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                            const int* __restrict__ n_segs) {
  extern __shared__ uint32_t stage_smem[];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int nseg = *n_segs;
  const int stride = gridDim.x * wpb;
  const int first = blockIdx.x * wpb + warp;
  uint32_t* wbuf = stage_smem + (size_t)warp * NS * kStageWords;
  // populations of the previous step are final from here on
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const uint16_t* nbs = segment_flags(segs, n_segs);
#pragma unroll
  for (int k = 0; k < NS - 1; ++k)
    stage_issue<T, PHASE>(views, segs, nbs, nseg, first + k * stride, lane, wbuf + k * kStageWords);
  for (int k = 0; first + k * stride < nseg; ++k) {
    stage_issue<T, PHASE>(views, segs, nbs, nseg, first + (k + NS - 1) * stride, lane,
                          wbuf + ((k + NS - 1) % NS) * kStageWords);
    cp_async_wait<NS>();  // the stage of task k has landed
    stage_consume<T, PHASE, MOM>(views, wbuf + (k % NS) * kStageWords, lane);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---- staged cell tasks --------------------------------------------------------
//
// The compacted cell tasks of k_stream_collide_cells are bound by memory
// latency on the candidate batches (one cell a lane, nine scalar loads; a
// long-scoreboard stall of 20-28 per issued instruction at a quarter of the
// issue slots).  Here each warp copies the nine incoming populations of its
// task NS-1 tasks ahead into shared memory, as k_stream_collide_staged does
// for row segments; the cell's offset and flags come from its list entry.
template <class T, int PHASE>
__device__ __forceinline__ void cell_stage_issue(const LatticeView* __restrict__ views,
                                                 const CellRef* __restrict__ cells, int ncell, int t, int lane,
                                                 uint32_t* buf) {
  const int e = (t << 5) + lane;
  const bool valid = e < ncell;
  const CellRef cr = cells[valid ? e : 0];
  const unsigned lat = valid ? (cr.meta & ((1u << kCellLatticeBits) - 1u)) : 0u;
  const LatticeView* __restrict__ L = views + lat;
  const T* F = static_cast<const T*>(L->f);
  const unsigned nb = (cr.meta >> kCellLatticeBits) & 0x1ffu;
  const bool inlet = valid && ((cr.meta >> 29) & 1u), outlet = valid && ((cr.meta >> 30) & 1u);
  const int pitch = L->pitch, pl = (int)L->plane;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int off = valid ? src_off<PHASE>(i, cr.c, pitch, pl, nb, inlet, outlet) : -1;
    cp_async_word<T>(buf + i * 32 + lane, F, off, L->f_elems);
  }
  buf[9 * 32 + lane] = valid ? (uint32_t)cr.c : 0u;
  buf[10 * 32 + lane] = nb | ((uint32_t)valid << 9) | ((uint32_t)inlet << 10) | ((uint32_t)outlet << 11) | (lat << 12);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <class T, int PHASE, int MOM, int NS>
__global__ void __launch_bounds__(512, 2)
    k_stream_collide_cells_staged(const LatticeView* __restrict__ views, const CellRef* __restrict__ cells,
                                  const int* __restrict__ n_segs, const int* __restrict__ cpre) {
  extern __shared__ uint32_t stage_smem[];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int ncell = cpre[n_segs[0]];
  const int ntask = (ncell + 31) >> 5;
  const int stride = gridDim.x * wpb;
  const int first = blockIdx.x * wpb + warp;
  uint32_t* wbuf = stage_smem + (size_t)warp * NS * kStageWords;
  // populations of the previous step are final from here on
  asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
  for (int k = 0; k < NS - 1; ++k)
    cell_stage_issue<T, PHASE>(views, cells, ncell, first + k * stride, lane, wbuf + k * kStageWords);
  for (int k = 0; first + k * stride < ntask; ++k) {
    cell_stage_issue<T, PHASE>(views, cells, ncell, first + (k + NS - 1) * stride, lane,
                               wbuf + ((k + NS - 1) % NS) * kStageWords);
    cp_async_wait<NS>();  // this lane's copies of task k have landed (each lane reads only its own)
    stage_consume<T, PHASE, MOM>(views, wbuf + (k % NS) * kStageWords, lane);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <class T, int NS>
void* pick_cells_staged(int phase, int moments) {
  if (phase == 0) return (void*)k_stream_collide_cells_staged<T, 0, 0, NS>;
  if (moments == 1) return (void*)k_stream_collide_cells_staged<T, 1, 1, NS>;
  if (moments == 2) return (void*)k_stream_collide_cells_staged<T, 1, 2, NS>;
  return (void*)k_stream_collide_cells_staged<T, 1, 0, NS>;
}

template <class T>
void* pick_cells_any(int phase, int moments, int stages) {
  switch (stages) {
    case 0: return pick_cells<T>(phase, moments);
    case 2: return pick_cells_staged<T, 2>(phase, moments);
    case 3: return pick_cells_staged<T, 3>(phase, moments);
    case 4: return pick_cells_staged<T, 4>(phase, moments);
    default: return nullptr;
  }
}

void* cells_kernel_for(int precision, int phase, int moments, int stages) {
  switch (precision) {
    case LBM_F32: return pick_cells_any<float>(phase, moments, stages);
    case LBM_BF16_SHIFTED: return pick_cells_any<__nv_bfloat16>(phase, moments, stages);
    case LBM_F16_SHIFTED: return pick_cells_any<__half>(phase, moments, stages);
    default: return nullptr;
  }
}

// ---- staged paired tasks ----------------------------------------------------
//
// The paired kernel keeps one window's pairs in flight per lane (36 bytes
// with 16-bit storage): at the occupancy its registers allow, too few bytes
// per SM to cover the memory latency.  Here each warp copies the pairs of
// the windows NS-1 tasks ahead into shared memory (cp.async: the lane's own
// pair of each slot, lanes 0 and 31 also the edge elements), so that the
// bytes in flight take no registers.  Row segments outside interior
// windows are loaded directly when their turn comes.  A stage holds the
// task entry (words 0-1), the edge words (2-7: lane 0's three, lane 31's
// three) and the nine slots of 32 pairs.
template <class T>
struct PairStage {
  static constexpr int kPairWords = 2 * (int)sizeof(T) / 4;  // 32-bit words per pair
  static constexpr int kHead = 8;
  static constexpr int kWords = kHead + 9 * 32 * kPairWords;  // a multiple of 4: stages stay 16-byte aligned
};

template <int N>
__device__ __forceinline__ void cp_async_n(uint32_t* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = ok ? N : 0;  // 0: fill with zeros, read nothing
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(N), "r"(n) : "memory");
}

// 16 bytes global -> shared, cached in L2 only (ok false: zeros, nothing read)
__device__ __forceinline__ void cp_async_16(uint32_t* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}

// Stage a paired task: the window's nine aligned row pieces (32 pairs, 128 or
// 256 bytes each) in 16-byte chunks spread over the lanes, so a lane may fill
// another lane's words (the loop synchronises the warp around each stage),
// and in phase A the six edge elements by lanes 0 and 31.
template <class T, int PHASE, bool ONE>
__device__ __forceinline__ void pair_stage_issue(const LatticeView* __restrict__ views, const SegRef sr,
                                                 const int lane, uint32_t* sb) {
  constexpr int W = PairStage<T>::kPairWords;
  if (lane == 0) {
    sb[0] = (uint32_t)sr.lattice;
    sb[1] = (uint32_t)sr.yw;
  }
  if (!(sr.lattice & kPairTask)) return;  // a row segment: loaded when its turn comes
  const LatticeView* __restrict__ L = views + (ONE ? 0 : (sr.lattice & ~kPairTask));
  const T* F = static_cast<const T*>(L->f);
  const int pitch = L->pitch, pl = (int)L->plane;
  const long long fe = L->f_elems;
  (void)fe;
  const int y = sr.yw >> kSegWordBits, p = sr.yw & ((1 << kSegWordBits) - 1);
  const int base = y * pitch + (p << 6);  // the window's first cell: rows start 128-byte aligned
  constexpr int kChunks = 8 * W;           // 16-byte chunks per piece
  constexpr int kPer = 16 / (int)sizeof(T);
#pragma unroll
  for (int r = 0; r < (9 * kChunks + 31) / 32; ++r) {
    const int j = lane + 32 * r;
    if (j < 9 * kChunks) {
      const int i = j / kChunks, q = j - i * kChunks;
      const int off = pair_plane(PHASE, i) * pl + base + pair_row(PHASE, i) * pitch + q * kPer;
      const bool ok = LBM_OK_IDX(off, fe) && LBM_OK_IDX(off + kPer - 1, fe);
      cp_async_16(sb + PairStage<T>::kHead + i * 32 * W + 4 * q, F + (ok ? off : 0), ok);
    }
  }
  const int c = base + 2 * lane;
  if (PHASE == 0 && (lane == 0 || lane == 31)) {
    const bool first = lane == 0;
    const int d = first ? -1 : 2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int off = pair_edge_plane(first, k) * pl + c + pair_edge_row(k) * pitch + d;
      const bool ok = LBM_OK_IDX(off, fe);
      // 16-bit: the aligned word holding the element (lane 0: its upper half, lane 31: its lower)
      const int src = sizeof(T) == 4 ? off : (off & ~1);
      cp_async_n<4>(sb + 2 + (first ? k : 3 + k), F + (ok ? src : 0), ok);
    }
  }
}

template <class T, int PHASE, int MOM, bool ONE>
__device__ __forceinline__ void pair_stage_consume(const LatticeView* __restrict__ views, const SegRef sr,
                                                   const uint32_t* sb, const int lane) {
  using P = Pop<T>;
  constexpr int W = PairStage<T>::kPairWords;
  const LatticeView* __restrict__ L = views + (ONE ? 0 : (sr.lattice & ~kPairTask));
  T* __restrict__ F = static_cast<T*>(L->f);
  const int pitch = L->pitch, pl = (int)L->plane;
  const long long fe = L->f_elems;
  const int y = sr.yw >> kSegWordBits, p = sr.yw & ((1 << kSegWordBits) - 1);
  const int c = y * pitch + (p << 6) + 2 * lane;
  float a[9], b[9], e[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < 9; ++i)
    Pop2<T>::ld(reinterpret_cast<const T*>(sb + PairStage<T>::kHead + (i * 32 + lane) * W), a[i], b[i]);
  if (PHASE == 0 && (lane == 0 || lane == 31)) {
    const bool first = lane == 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) e[k] = P::from_word(sb[2 + (first ? k : 3 + k)], first ? 1 : 0);
  }
  pair_assemble<PHASE>(a, b, e, lane);
  pair_finish<T, PHASE, MOM>(L, F, c, pitch, pl, fe, lane, a, b);
}

template <class T, int PHASE, int MOM, int NS, bool ONE>
__device__ __forceinline__ void pairs_staged_loop(const LatticeView* __restrict__ views,
                                                  const SegRef* __restrict__ tasks, const int* __restrict__ n_tasks,
                                                  uint32_t* pair_smem) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int SW = PairStage<T>::kWords;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  const int ntask = *n_tasks;
  uint32_t* wbuf = pair_smem + warp * NS * SW;
  const int t0 = blockIdx.x * wpb + warp;
  // every copy reads populations: wait for the previous step first
  asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    const int t = t0 + k * stride;
    if (t < ntask) pair_stage_issue<T, PHASE, ONE>(views, tasks[t], lane, wbuf + k * SW);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  int ta = t0 + (NS - 1) * stride;  // the next task to stage, its entry loaded one turn early
  SegRef ahead = ta < ntask ? tasks[ta] : SegRef{0, 0};
  for (int k = 0, t = t0; t < ntask; ++k, t += stride) {
    __syncwarp();  // every lane is done with the stage refilled now (task k - 1's)
    if (ta < ntask) pair_stage_issue<T, PHASE, ONE>(views, ahead, lane, wbuf + ((k + NS - 1) % NS) * SW);
    asm volatile("cp.async.commit_group;" ::: "memory");
    ta += stride;
    if (ta < ntask) ahead = tasks[ta];
    cp_async_wait<NS>();  // this lane's copies of task k have landed
    __syncwarp();         // and every lane's
    const uint32_t* sb = wbuf + (k % NS) * SW;
    SegRef cur{(int)sb[0], (int)sb[1]};
    if (cur.lattice & kPairTask) {
      pair_stage_consume<T, PHASE, MOM, ONE>(views, cur, sb, lane);
    } else {
      if (ONE) cur.lattice = 0;
      SegCtx<T> sc;
      seg_prologue<T, PHASE, 0, true>(views, cur, true, lane, sc, nullptr, 0);
      float g[9];
      seg_load<T, PHASE, false, 0>(sc, g);
      seg_update<T, PHASE, MOM, 0>(sc, g);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <class T, int PHASE, int MOM, int NS>
__global__ void __launch_bounds__(max_step_threads(2), 1)
    k_stream_collide_pairs_staged(const LatticeView* __restrict__ views, const SegRef* __restrict__ tasks,
                                  const int* __restrict__ n_tasks) {
  extern __shared__ uint32_t pair_smem[];
  pairs_staged_loop<T, PHASE, MOM, NS, false>(views, tasks, n_tasks, pair_smem);
}

template <class T, int PHASE, int MOM, int NS>
__global__ void __launch_bounds__(max_step_threads(2), 1)
    k_stream_collide_pairs_staged_one(const __grid_constant__ LatticeView one, const SegRef* __restrict__ tasks,
                                      const int* __restrict__ n_tasks) {
  extern __shared__ uint32_t pair_smem[];
  pairs_staged_loop<T, PHASE, MOM, NS, true>(&one, tasks, n_tasks, pair_smem);
}

template <class T, int NS>
void* pick_pairs_staged(int phase, int moments, bool one) {
  if (one) {
    if (phase == 0) return (void*)k_stream_collide_pairs_staged_one<T, 0, 0, NS>;
    if (moments == 1) return (void*)k_stream_collide_pairs_staged_one<T, 1, 1, NS>;
    if (moments == 2) return (void*)k_stream_collide_pairs_staged_one<T, 1, 2, NS>;
    return (void*)k_stream_collide_pairs_staged_one<T, 1, 0, NS>;
  }
  if (phase == 0) return (void*)k_stream_collide_pairs_staged<T, 0, 0, NS>;
  if (moments == 1) return (void*)k_stream_collide_pairs_staged<T, 1, 1, NS>;
  if (moments == 2) return (void*)k_stream_collide_pairs_staged<T, 1, 2, NS>;
  return (void*)k_stream_collide_pairs_staged<T, 1, 0, NS>;
}

template <class T>
void* pick_pairs_any(int phase, int moments, int stages, bool one) {
  switch (stages) {
    case 0: return pick_pairs<T>(phase, moments, one);
    case 2: return pick_pairs_staged<T, 2>(phase, moments, one);
    case 3: return pick_pairs_staged<T, 3>(phase, moments, one);
    case 4: return pick_pairs_staged<T, 4>(phase, moments, one);
    default: return nullptr;
  }
}

void* pairs_kernel_for(int precision, int phase, int moments, int stages, bool one) {
  switch (precision) {
    case LBM_F32: return pick_pairs_any<float>(phase, moments, stages, one);
    case LBM_BF16_SHIFTED: return pick_pairs_any<__nv_bfloat16>(phase, moments, stages, one);
    case LBM_F16_SHIFTED: return pick_pairs_any<__half>(phase, moments, stages, one);
    default: return nullptr;
  }
}

size_t pairs_smem_bytes(int precision, int warps_per_block, int stages) {
  if (stages < 2) return 0;
  const int words = precision == LBM_F32 ? PairStage<float>::kWords : PairStage<__half>::kWords;
  return (size_t)warps_per_block * stages * words * sizeof(uint32_t);
}

size_t staged_smem_bytes(int warps_per_block, int stages) {
  return (size_t)warps_per_block * stages * kStageWords * sizeof(uint32_t);
}

// Grid-wide barrier of the persistent kernel (all blocks co-resident: the
// kernel is launched cooperatively).  One monotonic arrival counter, reset
// before the launch: at its k-th barrier a block publishes its writes,
// arrives, and waits until the counter reaches k * gridDim.x.  The wait gives
// up after kSpinLimit polls (or when another block has given up), flags the
// failure and makes every block leave the kernel at its next barrier.
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_barrier(StepBarrier* b, unsigned& target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    target += gridDim.x + (unsigned)b->extra;
    __threadfence();  // this block's population writes before its arrival
    atomicAdd(&b->count, 1u);
    unsigned spins = 0;
    while (ld_acquire(&b->count) < target) {
      if (++spins > kSpinLimit || ld_acquire(reinterpret_cast<const unsigned*>(&b->error)) != 0) {
        atomicExch(&b->error, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// n_pairs (A, B) time-step pairs in one launch, a grid barrier after every
// phase but the last.  Same per-cell arithmetic as k_stream_collide.
template <class T, int CPT>
__global__ void __launch_bounds__(max_persistent_threads(CPT), min_persistent_blocks(CPT))
    k_stream_collide_persistent(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                const int* __restrict__ n_segs, int n_pairs, StepBarrier* bar) {
  const int lane = threadIdx.x & 31;
  const int nseg = *n_segs;
  const int ntask = (nseg + CPT - 1) / CPT;
  const int wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  const int first = blockIdx.x * wpb + (threadIdx.x >> 5);
  const uint16_t* nbs = segment_flags(segs, n_segs);
  unsigned target = 0;
  bool waited = true;  // a cooperative launch follows the stream order: nothing to wait for
  for (int p = 0; p < n_pairs; ++p) {
    for (int t = first; t < ntask; t += stride) phase_task<T, 0, 0, CPT, true>(views, segs, nbs, nseg, t, lane, waited);
    if (!grid_barrier(bar, target)) return;
    for (int t = first; t < ntask; t += stride) phase_task<T, 1, 0, CPT, true>(views, segs, nbs, nseg, t, lane, waited);
    if (p + 1 < n_pairs && !grid_barrier(bar, target)) return;
  }
}

template <class T, int CPT, int FEAT = 0>
void* pick(int phase, int moments) {
  if (phase == 0) return (void*)k_stream_collide<T, 0, 0, CPT, FEAT>;
  if (moments == 1) return (void*)k_stream_collide<T, 1, 1, CPT, FEAT>;
  if (moments == 2) return (void*)k_stream_collide<T, 1, 2, CPT, FEAT>;
  return (void*)k_stream_collide<T, 1, 0, CPT, FEAT>;
}

template <class T, int NS>
void* pick_staged(int phase, int moments) {
  if (phase == 0) return (void*)k_stream_collide_staged<T, 0, 0, NS>;
  if (moments == 1) return (void*)k_stream_collide_staged<T, 1, 1, NS>;
  if (moments == 2) return (void*)k_stream_collide_staged<T, 1, 2, NS>;
  return (void*)k_stream_collide_staged<T, 1, 0, NS>;
}

template <class T>
void* pick_cpt(int phase, int moments, int cpt, int stages, int features) {
  if (features) {
    if (cpt != 1 || stages != 0) return nullptr;
    switch (features) {
      case kFeatModels: return pick<T, 1, kFeatModels>(phase, moments);
      case kFeatMirror: return pick<T, 1, kFeatMirror>(phase, moments);
      case kFeatModels | kFeatMirror: return pick<T, 1, kFeatModels | kFeatMirror>(phase, moments);
      default: return nullptr;
    }
  }
  if (stages == 2) return cpt == 1 ? pick_staged<T, 2>(phase, moments) : nullptr;
  if (stages == 3) return cpt == 1 ? pick_staged<T, 3>(phase, moments) : nullptr;
  if (stages != 0) return nullptr;
  return cpt == 1 ? pick<T, 1>(phase, moments) : cpt == 2 ? pick<T, 2>(phase, moments) : nullptr;
}

void* kernel_for(int precision, int phase, int moments, int cpt, int stages, int features) {
  switch (precision) {
    case LBM_F32: return pick_cpt<float>(phase, moments, cpt, stages, features);
    case LBM_BF16_SHIFTED: return pick_cpt<__nv_bfloat16>(phase, moments, cpt, stages, features);
    case LBM_F16_SHIFTED: return pick_cpt<__half>(phase, moments, cpt, stages, features);
    default: return nullptr;
  }
}

// Dynamic shared memory of a launch; the kernel is allowed that much once.
size_t launch_smem(void* k, const StepConfig& sc) {
  if (sc.stages == 0) return 0;
  const size_t bytes = staged_smem_bytes(sc.warps_per_block, sc.stages);
  if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return bytes;
}

template <class T>
void* persistent_pick(int cpt) {
  return cpt == 1 ? (void*)k_stream_collide_persistent<T, 1>
                  : cpt == 2 ? (void*)k_stream_collide_persistent<T, 2> : nullptr;
}

void* persistent_kernel_for(int precision, int cpt) {
  switch (precision) {
    case LBM_F32: return persistent_pick<float>(cpt);
    case LBM_BF16_SHIFTED: return persistent_pick<__nv_bfloat16>(cpt);
    case LBM_F16_SHIFTED: return persistent_pick<__half>(cpt);
    default: return nullptr;
  }
}

bool shape_ok(const StepConfig& sc) {
  return (sc.cells_per_thread == 1 || sc.cells_per_thread == 2) && sc.warps_per_block >= 1 &&
         sc.warps_per_block * 32 <=
             (sc.persistent ? max_persistent_threads : max_step_threads)(sc.cells_per_thread) &&
         sc.grid >= 1 &&
         (sc.stages == 0 || ((sc.stages == 2 || sc.stages == 3) && sc.cells_per_thread == 1 && !sc.persistent)) &&
         (!sc.features || (sc.cells_per_thread == 1 && sc.stages == 0 && !sc.persistent));
}

}  // namespace

cudaError_t launch_stream_collide(int precision, int phase, int moments, const LatticeView* views,
                                  const SegRef* segs, const int* n_segs, StepConfig sc,
                                  cudaStream_t stream) {
  void* k = kernel_for(precision, phase, moments, sc.cells_per_thread, sc.stages, sc.features);
  if (!k || !shape_ok(sc)) return cudaErrorInvalidValue;
  void* args[] = {(void*)&views, (void*)&segs, (void*)&n_segs};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sc.grid);
  cfg.blockDim = dim3(32 * sc.warps_per_block);
  cfg.dynamicSmemBytes = launch_smem(k, sc);
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

cudaError_t launch_stream_collide_cells(int precision, int phase, int moments, const LatticeView* views,
                                        const CellRef* cells, const int* n_segs, const int* cpre, StepConfig sc,
                                        cudaStream_t stream) {
  void* k = cells_kernel_for(precision, phase, moments, sc.stages);
  if (!k || sc.warps_per_block < 1 || sc.warps_per_block > (sc.stages ? 16 : 32) || sc.grid < 1)
    return cudaErrorInvalidValue;
  const size_t smem = sc.stages ? staged_smem_bytes(sc.warps_per_block, sc.stages) : 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  void* args[] = {(void*)&views, (void*)&cells, (void*)&n_segs, (void*)&cpre};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sc.grid);
  cfg.blockDim = dim3(32 * sc.warps_per_block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

cudaError_t launch_stream_collide_pairs(int precision, int phase, int moments, const LatticeView* views,
                                        const LatticeView* one, const SegRef* tasks, const int* n_tasks,
                                        StepConfig sc, cudaStream_t stream) {
  void* k = pairs_kernel_for(precision, phase, moments, sc.stages, one != nullptr);
  if (!k || sc.warps_per_block < 1 || 32 * sc.warps_per_block > max_step_threads(2) || sc.grid < 1)
    return cudaErrorInvalidValue;
  const size_t smem = pairs_smem_bytes(precision, sc.warps_per_block, sc.stages);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  void* args[] = {one ? (void*)one : (void*)&views, (void*)&tasks, (void*)&n_tasks};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sc.grid);
  cfg.blockDim = dim3(32 * sc.warps_per_block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

int stream_collide_pairs_blocks_per_sm(int precision, int phase, int moments, int warps_per_block, int stages) {
  void* k = pairs_kernel_for(precision, phase, moments, stages, false);
  const size_t smem = pairs_smem_bytes(precision, warps_per_block, stages);
  int n = 0;
  if (k && smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps_per_block, smem) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

int stream_collide_cells_blocks_per_sm(int precision, int phase, int moments, int warps_per_block, int stages) {
  void* k = cells_kernel_for(precision, phase, moments, stages);
  const size_t smem = stages ? staged_smem_bytes(warps_per_block, stages) : 0;
  int n = 0;
  if (k && smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps_per_block, smem) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

int stream_collide_persistent_grid(int precision, int warps_per_block, int cells_per_thread) {
  void* k = persistent_kernel_for(precision, cells_per_thread);
  int dev = 0, sms = 0, n = 0;
  if (!k || warps_per_block * 32 > max_persistent_threads(cells_per_thread) || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps_per_block, 0) != cudaSuccess)
    return 0;
  return n * sms;
}

cudaError_t launch_stream_collide_persistent(int precision, const LatticeView* views, const SegRef* segs,
                                             const int* n_segs, int n_pairs, StepConfig sc, StepBarrier* bar,
                                             cudaStream_t stream) {
  void* k = persistent_kernel_for(precision, sc.cells_per_thread);
  if (!k || !shape_ok(sc) || sc.features || n_pairs < 1 ||
      sc.grid > stream_collide_persistent_grid(precision, sc.warps_per_block, sc.cells_per_thread) ||
      2ull * (unsigned long long)n_pairs * (unsigned long long)sc.grid >= (1ull << 32))
    return cudaErrorInvalidValue;
  // a fresh barrier: count 0, no error
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(StepBarrier), stream);
  if (e != cudaSuccess) return e;
  if (barrier_timeout_test() &&
      (e = cudaMemsetAsync(reinterpret_cast<char*>(bar) + offsetof(StepBarrier, extra), 1, 1, stream)) != cudaSuccess)
    return e;
  void* args[] = {(void*)&views, (void*)&segs, (void*)&n_segs, (void*)&n_pairs, (void*)&bar};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks co-resident: the barrier can complete
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sc.grid);
  cfg.blockDim = dim3(32 * sc.warps_per_block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelExC(&cfg, k, args);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

int stream_collide_blocks_per_sm(int precision, int phase, int moments, int warps_per_block, int cells_per_thread,
                                 int stages, int features) {
  void* k = kernel_for(precision, phase, moments, cells_per_thread, stages, features);
  StepConfig sc{warps_per_block, 1, 0, cells_per_thread, stages, features};
  int n = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps_per_block, launch_smem(k, sc)) !=
                cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace lbm
