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
// Thread mapping.  Each warp takes one row segment (the 32 cells of one mask
// word) from a device-resident list holding only segments with fluid cells;
// lane l handles cell 32w + l, so every plane access of a warp is one
// contiguous 32-element row segment (shifted by at most one element).  Warps
// stride over the list; the list may span several lattices (batches).
// Consecutive steps are programmatic dependent launches: a step's warps load
// their segment, descriptor and mask words while the previous step is still
// finishing, and wait for it only before touching populations.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {
namespace {

template <class T>
struct Pop;
// ld: plain load; ldcg: load cached in L2 only.  Within one persistent launch
// a slot written by another block must not be served from this SM's L1 (L1
// is not coherent across SMs), so that kernel reads populations with ldcg.
template <>
struct Pop<float> {
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct Pop<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ float ldcg(const __nv_bfloat16* p) { return __bfloat162float(__ldcg(p)); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct Pop<__half> {
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ float ldcg(const __half* p) { return __half2float(__ldcg(p)); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};

constexpr float kW0 = 4.0f / 9.0f;
constexpr float kW1 = 1.0f / 9.0f;
constexpr float kW5 = 1.0f / 36.0f;

// Relax a pair of opposite directions (c_o = -c_i) towards the shifted
// equilibrium  g^eq_i = w (t0 + 3 rho cu + 4.5 rho cu^2),  t0 = drho - 1.5 rho u.u,
// which is f^eq_i(rho, u) - w rho0 written out.
__device__ __forceinline__ void relax_pair(float& gi, float& go, float cu, float w, float rho,
                                           float t0, float omega) {
  const float a = 3.0f * rho * cu;
  const float b = 4.5f * rho * cu * cu;
  const float ei = w * (t0 + a + b);
  const float eo = w * (t0 - a + b);
  gi += omega * (ei - gi);
  go += omega * (eo - go);
}

// Moments (Eq. 2) and BGK relaxation (Eq. 1) of one cell, in place.
__device__ __forceinline__ void bgk(float (&g)[9], float rho0, float omega, float& drho, float& ux,
                                    float& uy) {
  drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const float rho = rho0 + drho;
  const float jx = (g[1] - g[3]) + (g[5] - g[7]) + (g[8] - g[6]);
  const float jy = (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
  const float inv = 1.0f / rho;
  ux = jx * inv;
  uy = jy * inv;
  const float t0 = drho - 1.5f * rho * (ux * ux + uy * uy);
  relax_pair(g[1], g[3], ux, kW1, rho, t0, omega);
  relax_pair(g[2], g[4], uy, kW1, rho, t0, omega);
  relax_pair(g[5], g[7], ux + uy, kW5, rho, t0, omega);
  relax_pair(g[8], g[6], ux - uy, kW5, rho, t0, omega);
  // BGK conserves mass and momentum; rounded FP32 relaxation does not quite,
  // and the drift dominates the FP32 error over thousands of steps.  Close
  // both exactly: g1 and g2 carry the momentum balance, the rest population
  // the mass balance (an identity in exact arithmetic).
  g[1] = jx + g[3] - ((g[5] - g[7]) + (g[8] - g[6]));
  g[2] = jy + g[4] - ((g[5] - g[7]) + (g[6] - g[8]));
  g[0] = drho - (((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
}

// Shifted equilibria of all nine directions for (rho0 + drho, ux, uy).
__device__ __forceinline__ void shifted_equilibria(float (&e)[9], float rho0, float drho, float ux,
                                                   float uy) {
  const float rho = rho0 + drho;
  const float t0 = drho - 1.5f * rho * (ux * ux + uy * uy);
  e[0] = kW0 * t0;
  const float cu[4] = {ux, uy, ux + uy, ux - uy};  // directions 1, 2, 5, 8 (opposites 3, 4, 7, 6)
  const int di[4] = {1, 2, 5, 8}, dopp[4] = {3, 4, 7, 6};
  const float wt[4] = {kW1, kW1, kW5, kW5};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float a = 3.0f * rho * cu[k], b = 4.5f * rho * cu[k] * cu[k];
    e[di[k]] = wt[k] * (t0 + a + b);
    e[dopp[k]] = wt[k] * (t0 - a + b);
  }
}

// Regularised port cell: given the cell's (drho, u) and its populations with
// the unknown ones already filled, replace all nine by
//   g_i = g^eq_i + w_i / (2 c_s^4) Q_i : Pi,   Pi = sum_i c_i c_i (g_i - g^eq_i),
// Q_i = c_i c_i - I/3.  With c_s^2 = 1/3 the coefficients 4.5 w_i Q_i are
//   rest: -(2/3)(Pxx + Pyy); axis x: Pxx/3 - Pyy/6; axis y: Pyy/3 - Pxx/6;
//   diagonals NE/SW: (Pxx + Pyy)/12 + Pxy/4; NW/SE: (Pxx + Pyy)/12 - Pxy/4.
__device__ __forceinline__ void regularize(float (&g)[9], const float (&e)[9]) {
  float n[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) n[i] = g[i] - e[i];
  const float dsum = (n[5] + n[6]) + (n[7] + n[8]);
  const float pxx = (n[1] + n[3]) + dsum;
  const float pyy = (n[2] + n[4]) + dsum;
  const float pxy = (n[5] + n[7]) - (n[6] + n[8]);
  const float tr = pxx + pyy;
  g[0] = e[0] - (2.0f / 3.0f) * tr;
  const float ax = pxx * (1.0f / 3.0f) - pyy * (1.0f / 6.0f);
  const float ay = pyy * (1.0f / 3.0f) - pxx * (1.0f / 6.0f);
  g[1] = e[1] + ax;
  g[3] = e[3] + ax;
  g[2] = e[2] + ay;
  g[4] = e[4] + ay;
  const float dp = tr * (1.0f / 12.0f) + 0.25f * pxy, dm = tr * (1.0f / 12.0f) - 0.25f * pxy;
  g[5] = e[5] + dp;
  g[7] = e[7] + dp;
  g[6] = e[6] + dm;
  g[8] = e[8] + dm;
}

// Inlet (x = 0), imposed velocity (u, 0).  Density from mass and x-momentum of
// the known populations, rho = (f0 + f2 + f4 + 2 (f3 + f6 + f7)) / (1 - u), in
// shifted form drho = (s + rho0 u) / (1 - u).  Zou-He rebuilds f1, f5, f8:
//   f1 = f3 + 2/3 rho u,  f5 = f7 - (f2 - f4)/2 + rho u / 6,
//   f8 = f6 + (f2 - f4)/2 + rho u / 6;
// the regularised scheme takes their non-equilibrium parts from the opposite
// directions and then regularises the cell.
__device__ __forceinline__ void inlet_rule(float (&g)[9], float u, float rho0, int scheme) {
  const float s = (g[0] + g[2] + g[4]) + 2.0f * (g[3] + g[6] + g[7]);
  const float drho = (s + rho0 * u) / (1.0f - u);
  if (scheme == LBM_PORTS_ZOU_HE) {
    const float ru = (rho0 + drho) * u;
    const float d = 0.5f * (g[2] - g[4]);
    g[1] = g[3] + (2.0f / 3.0f) * ru;
    g[5] = g[7] - d + (1.0f / 6.0f) * ru;
    g[8] = g[6] + d + (1.0f / 6.0f) * ru;
  } else {
    float e[9];
    shifted_equilibria(e, rho0, drho, u, 0.0f);
    g[1] = e[1] + (g[3] - e[3]);
    g[5] = e[5] + (g[7] - e[7]);
    g[8] = e[8] + (g[6] - e[6]);
    regularize(g, e);
  }
}

// Outlet (x = nx-1) at density rho0: u = -1 + (f0 + f2 + f4 + 2 (f1 + f5 + f8)) / rho0,
// i.e. rho0 u = s in shifted form.  Zou-He rebuilds f3, f6, f7 (mirror of the
// inlet); the regularised scheme as at the inlet.
__device__ __forceinline__ void outlet_rule(float (&g)[9], float rho0, int scheme) {
  const float ru = (g[0] + g[2] + g[4]) + 2.0f * (g[1] + g[5] + g[8]);
  if (scheme == LBM_PORTS_ZOU_HE) {
    const float d = 0.5f * (g[2] - g[4]);
    g[3] = g[1] - (2.0f / 3.0f) * ru;
    g[7] = g[5] + d - (1.0f / 6.0f) * ru;
    g[6] = g[8] - d - (1.0f / 6.0f) * ru;
  } else {
    float e[9];
    shifted_equilibria(e, rho0, 0.0f, ru / rho0, 0.0f);
    g[3] = e[3] + (g[1] - e[1]);
    g[7] = e[7] + (g[5] - e[5]);
    g[6] = e[6] + (g[8] - e[8]);
    regularize(g, e);
  }
}

// population access with optional bounds checks (offset in elements from F)
#define FLD(off) (LBM_OK_IDX((off), fe) ? (PERSIST ? P::ldcg(F + (off)) : P::ld(F + (off))) : 0.0f)
#define FST(off, v)                                   \
  do {                                                \
    if (LBM_OK_IDX((off), fe)) P::st(F + (off), (v)); \
  } while (0)

// neighbour solid flags, bit i-1 = solid(x + c_i), i = 1..8 (E N W S NE NW SW SE)
constexpr unsigned kE = 1u, kN = 2u, kW = 4u, kS = 8u, kNE = 16u, kNW = 32u, kSW = 64u, kSE = 128u;

// Block size is 128, 256 or 512 threads (chosen per launch); the register
// budget is the same (at most 64 per thread) for all of them.
constexpr int kMaxStepThreads = 512;

// One phase of one time step on one row segment (lane = cell 32w + lane).
// PERSIST: called from the persistent kernel (populations read through L2
// only; no programmatic-launch wait); otherwise from a programmatic dependent
// launch, which waits for the previous step once, just before its first
// population access (`waited`).
template <class T, int PHASE, int MOM, bool PERSIST>
__device__ __forceinline__ void update_segment(const LatticeView* __restrict__ views, const SegRef sr,
                                               const int lane, bool& waited) {
  using P = Pop<T>;
  {
    const LatticeView* __restrict__ L = views + sr.lattice;
    const int y = sr.yw >> kSegWordBits;
    const int w = sr.yw & ((1 << kSegWordBits) - 1);
#ifdef LBM_CHECK_BOUNDS
    if (sr.lattice < 0 || y < 1 || y > L->ny - 2 || w < 0 || w >= L->wpr) {
      if (lane == 0) printf("lbm bounds: bad segment: lattice %d y %d w %d\n", sr.lattice, y, w);
      return;
    }
#endif
    const int ms = mask_stride(L->wpr);
    const uint32_t* mr = L->mask + (long long)y * ms;
    const uint32_t mc = mr[w];
    const int nx = L->nx;
    const int x = (w << 5) + lane;
    const bool fluid = !((mc >> lane) & 1u);  // bits beyond nx are set (solid)
    const bool inlet = (x == 0);
    const bool outlet = (x == nx - 1);

    unsigned nb = 0;  // solid flags of the 8 neighbours (phase A only)
    if (PHASE == 0) {
      // padded mask: words w-1 and w+1 of rows y-1..y+1 always exist and are
      // solid outside the lattice
      const uint32_t* rn = mr + ms;
      const uint32_t* rs = mr - ms;
      const uint32_t mn = rn[w], msth = rs[w];
      const uint32_t eC = __funnelshift_r(mc, mr[w + 1], 1), wC = __funnelshift_l(mr[w - 1], mc, 1);
      const uint32_t eN = __funnelshift_r(mn, rn[w + 1], 1), wN = __funnelshift_l(rn[w - 1], mn, 1);
      const uint32_t eS = __funnelshift_r(msth, rs[w + 1], 1), wS = __funnelshift_l(rs[w - 1], msth, 1);
      nb = ((eC >> lane) & 1u) | (((mn >> lane) & 1u) << 1) | (((wC >> lane) & 1u) << 2) |
           (((msth >> lane) & 1u) << 3) | (((eN >> lane) & 1u) << 4) | (((wN >> lane) & 1u) << 5) |
           (((wS >> lane) & 1u) << 6) | (((eS >> lane) & 1u) << 7);
    }
    // 32-bit element offsets: lattices are limited to 9 * plane < 2^31
    const int pitch = L->pitch;
    const int pl = (int)L->plane;
    const float rho0 = L->rho0;
    const float omega = L->omega;
    const int rule = L->outlet_rule;
    T* __restrict__ F = static_cast<T*>(L->f);
    const long long fe = L->f_elems;
    (void)fe;
    const int c = y * pitch + x;

    if (!PERSIST && !waited) {  // warp-uniform: populations of the previous step are final from here on
      asm volatile("griddepcontrol.wait;" ::: "memory");
      waited = true;
    }

    float g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = 0.0f;
    if (fluid) {
      if (PHASE == 0) {
        g[0] = FLD(c);
        g[2] = (nb & kS) ? FLD(4 * pl + c) : FLD(2 * pl + c - pitch);
        g[4] = (nb & kN) ? FLD(2 * pl + c) : FLD(4 * pl + c + pitch);
        if (!inlet) {  // sources on the west side (unknown at the inlet)
          g[1] = (nb & kW) ? FLD(3 * pl + c) : FLD(1 * pl + c - 1);
          g[5] = (nb & kSW) ? FLD(7 * pl + c) : FLD(5 * pl + c - pitch - 1);
          g[8] = (nb & kNW) ? FLD(6 * pl + c) : FLD(8 * pl + c + pitch - 1);
        }
        if (!outlet) {  // sources on the east side (unknown at the outlet)
          g[3] = (nb & kE) ? FLD(1 * pl + c) : FLD(3 * pl + c + 1);
          g[6] = (nb & kSE) ? FLD(8 * pl + c) : FLD(6 * pl + c - pitch + 1);
          g[7] = (nb & kNE) ? FLD(5 * pl + c) : FLD(7 * pl + c + pitch + 1);
        }
      } else {
        g[0] = FLD(c);
        g[2] = FLD(4 * pl + c);
        g[4] = FLD(2 * pl + c);
        if (!inlet) {
          g[1] = FLD(3 * pl + c);
          g[5] = FLD(7 * pl + c);
          g[8] = FLD(6 * pl + c);
        }
        if (!outlet) {
          g[3] = FLD(1 * pl + c);
          g[6] = FLD(8 * pl + c);
          g[7] = FLD(5 * pl + c);
        }
      }
    }

    if (rule == LBM_OUT_NEUMANN) {
      // zero-gradient outlet: the unknown g3, g6, g7 of cell (nx-1, y) are the
      // streamed g3, g6, g7 of cell (nx-2, y), held by the lane to the left
      // (nx is even, so both cells are in this warp's row segment).
      const float n3 = __shfl_up_sync(0xffffffffu, g[3], 1);
      const float n6 = __shfl_up_sync(0xffffffffu, g[6], 1);
      const float n7 = __shfl_up_sync(0xffffffffu, g[7], 1);
      if (outlet) {
        g[3] = n3;
        g[6] = n6;
        g[7] = n7;
      }
    }

    if (!fluid) return;
    if (inlet) {
      inlet_rule(g, L->u_in[y], rho0, L->port_scheme);
    } else if (outlet && rule == LBM_OUT_CONST_RHO) {
      outlet_rule(g, rho0, L->port_scheme);
    }
    float drho, ux, uy;
    bgk(g, rho0, omega, drho, ux, uy);

    if (PHASE == 0) {
      FST(c, g[0]);
      if (nb & kN) FST(2 * pl + c, g[2]); else FST(4 * pl + c + pitch, g[2]);
      if (nb & kS) FST(4 * pl + c, g[4]); else FST(2 * pl + c - pitch, g[4]);
      if (!outlet) {  // destinations on the east side leave through the outlet
        if (nb & kE) FST(1 * pl + c, g[1]); else FST(3 * pl + c + 1, g[1]);
        if (nb & kNE) FST(5 * pl + c, g[5]); else FST(7 * pl + c + pitch + 1, g[5]);
        if (nb & kSE) FST(8 * pl + c, g[8]); else FST(6 * pl + c - pitch + 1, g[8]);
      }
      if (!inlet) {  // destinations on the west side leave through the inlet
        if (nb & kW) FST(3 * pl + c, g[3]); else FST(1 * pl + c - 1, g[3]);
        if (nb & kNW) FST(6 * pl + c, g[6]); else FST(8 * pl + c + pitch - 1, g[6]);
        if (nb & kSW) FST(7 * pl + c, g[7]); else FST(5 * pl + c - pitch - 1, g[7]);
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
}

template <class T, int PHASE, int MOM>
__global__ void __launch_bounds__(kMaxStepThreads, 2)
    k_stream_collide(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                     const int* __restrict__ n_segs) {
  // The next time step may be scheduled now; it reads populations only after
  // waiting for this grid to complete.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  // the segment list, descriptors and mask are never written by a time step,
  // so they may be read before the previous step has finished
  const int nseg = *n_segs;
  const int wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  bool waited = false;
  for (int sidx = blockIdx.x * wpb + (threadIdx.x >> 5); sidx < nseg; sidx += stride)
    update_segment<T, PHASE, MOM, false>(views, segs[sidx], lane, waited);
  if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Grid-wide barrier of the persistent kernel (all blocks co-resident: the
// kernel is launched cooperatively).  Sense by generation: a block reads the
// generation, publishes its writes, arrives; the last arrival resets the
// count and advances the generation; the others wait for the advance.  The
// wait gives up after kSpinLimit polls, flags the failure and makes every
// block leave the kernel at its next barrier.
constexpr unsigned kSpinLimit = 1u << 24;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_barrier(StepBarrier* b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire(&b->gen);
    __threadfence();  // this block's population writes before its arrival
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      unsigned spins = 0;
      while (ld_acquire(&b->gen) == gen) {
        if (++spins > kSpinLimit || ld_acquire(reinterpret_cast<const unsigned*>(&b->error)) != 0) {
          atomicExch(&b->error, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
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
template <class T>
__global__ void __launch_bounds__(kMaxStepThreads, 2)
    k_stream_collide_persistent(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                const int* __restrict__ n_segs, int n_pairs, StepBarrier* bar) {
  const int lane = threadIdx.x & 31;
  const int nseg = *n_segs;
  const int wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  const int first = blockIdx.x * wpb + (threadIdx.x >> 5);
  bool waited = true;
  for (int p = 0; p < n_pairs; ++p) {
    for (int sidx = first; sidx < nseg; sidx += stride)
      update_segment<T, 0, 0, true>(views, segs[sidx], lane, waited);
    if (!grid_barrier(bar)) return;
    for (int sidx = first; sidx < nseg; sidx += stride)
      update_segment<T, 1, 0, true>(views, segs[sidx], lane, waited);
    if (p + 1 < n_pairs && !grid_barrier(bar)) return;
  }
}


template <class T>
void* pick(int phase, int moments) {
  if (phase == 0) return (void*)k_stream_collide<T, 0, 0>;
  if (moments == 1) return (void*)k_stream_collide<T, 1, 1>;
  if (moments == 2) return (void*)k_stream_collide<T, 1, 2>;
  return (void*)k_stream_collide<T, 1, 0>;
}

void* kernel_for(int precision, int phase, int moments) {
  switch (precision) {
    case LBM_F32: return pick<float>(phase, moments);
    case LBM_BF16_SHIFTED: return pick<__nv_bfloat16>(phase, moments);
    case LBM_F16_SHIFTED: return pick<__half>(phase, moments);
    default: return nullptr;
  }
}

}  // namespace

cudaError_t launch_stream_collide(int precision, int phase, int moments, const LatticeView* views,
                                  const SegRef* segs, const int* n_segs, StepConfig sc,
                                  cudaStream_t stream) {
  void* k = kernel_for(precision, phase, moments);
  if (!k || sc.warps_per_block < 1 || sc.warps_per_block * 32 > kMaxStepThreads || sc.grid < 1)
    return cudaErrorInvalidValue;
  void* args[] = {(void*)&views, (void*)&segs, (void*)&n_segs};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sc.grid);
  cfg.blockDim = dim3(32 * sc.warps_per_block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

namespace {
void* persistent_kernel_for(int precision) {
  switch (precision) {
    case LBM_F32: return (void*)k_stream_collide_persistent<float>;
    case LBM_BF16_SHIFTED: return (void*)k_stream_collide_persistent<__nv_bfloat16>;
    case LBM_F16_SHIFTED: return (void*)k_stream_collide_persistent<__half>;
    default: return nullptr;
  }
}
}  // namespace

int stream_collide_persistent_grid(int precision, int warps_per_block) {
  void* k = persistent_kernel_for(precision);
  int dev = 0, sms = 0, n = 0;
  if (!k || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps_per_block, 0) != cudaSuccess)
    return 0;
  return n * sms;
}

cudaError_t launch_stream_collide_persistent(int precision, const LatticeView* views, const SegRef* segs,
                                             const int* n_segs, int n_pairs, StepConfig sc, StepBarrier* bar,
                                             cudaStream_t stream) {
  void* k = persistent_kernel_for(precision);
  if (!k || n_pairs < 1 || sc.warps_per_block < 1 || sc.warps_per_block * 32 > kMaxStepThreads || sc.grid < 1 ||
      sc.grid > stream_collide_persistent_grid(precision, sc.warps_per_block))
    return cudaErrorInvalidValue;
  // a fresh barrier: count 0, generation 0, no error
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(StepBarrier), stream);
  if (e != cudaSuccess) return e;
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

int stream_collide_blocks_per_sm(int precision, int phase, int moments, int warps_per_block) {
  void* k = kernel_for(precision, phase, moments);
  int n = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps_per_block, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace lbm
