// On-chip resident time steps: a whole solve in one launch, the populations
// held in shared memory from its first step to its last.
//
// Method: the same per-cell update as the step kernels (Eq. 1 with the
// equilibrium of Sec. 2.1, the moments of Eq. 2, halfway bounce-back and the
// port rules of Sec. 3.3; d2q9_cell.cuh), so every cell gets the same bits.
//
// Layout.  A lattice set whose row segments fit in the shared memory of the
// SMs (the 2048 x 1024 distributor: 6976 segments, 5.75 MB of FP32
// populations, against 152 x 227 KB) is split into contiguous ranges of its
// segment list, one range per block (at most kResidentMaxOwn segments, one
// block per SM, all blocks resident: a cooperative launch).  A block keeps
// its segments' nine population rows in two step buffers in shared memory
// (read one, write the other, a plain pull scheme), plus copies of the
// population rows it needs from segments of other blocks ("ghosts": per
// neighbouring segment only the directions that stream across, e.g. the
// three upward directions of the segment below).
//
// Exchange.  After each step a block publishes, for each of its segments
// that another block reads, the directions that block needs, as 64-bit words
// {value, step tag} in a halo buffer in global memory (two step parities).
// Before the next step it polls the words of its ghosts until each carries
// the expected tag: value and tag travel in one single-copy-atomic word, so
// there is no fence and no flag, and a block waits only for its neighbours
// -- no grid-wide barrier.  Two parities suffice: a block can overwrite a
// word of step t only after it has read its neighbours' step t + 1 words,
// which they publish after reading its step t words.  Every wait is bounded:
// a block that gives up sets the error word and leaves, and the others leave
// at their next check of that word.
//
// Per step and block: fetch the ghosts, one __syncthreads, then each warp
// updates its (at most two) segments -- the published ones first, so that
// neighbours can proceed while the rest is computed -- pulling from the
// current buffer through source offsets computed once per launch (own row,
// neighbouring own segment, ghost row, bounce-back into the cell's own slot,
// or a zero word for the unknown populations of port cells).  The lattice
// is read from the canonical global layout at the start of the launch and
// written back to it at the end.
#include "d2q9_cell.cuh"

namespace lbm {
namespace {

constexpr int kSegWords = 9 * 32;  // one segment's populations in a step buffer
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kResidentSpinLimit = 1u << 22;
constexpr int kFetch = 6;  // ghost rows a warp keeps in flight

// Neighbouring segments of (y, w), position p = 0..7: E N W S NE NW SW SE,
// (dy, dw) = (0,1) (1,0) (0,-1) (-1,0) (1,1) (1,-1) (-1,-1) (-1,1).
__device__ __forceinline__ int pos_dy(int p) { return (int)((0x00220121u >> (4 * p)) & 15u) - 1; }
__device__ __forceinline__ int pos_dw(int p) { return (int)((0x20021012u >> (4 * p)) & 15u) - 1; }
// position of (dy, dw) != (0, 0)
__device__ __forceinline__ int pos_of(int dy, int dw) {
  if (dy == 0) return dw > 0 ? 0 : 2;
  if (dw == 0) return dy > 0 ? 1 : 3;
  if (dy > 0) return dw > 0 ? 4 : 5;
  return dw < 0 ? 6 : 7;
}
// Directions a cell pulls from the segment at position p (bit i = direction
// i): from the segment above the three with c_y = -1, from the one below the
// three with c_y = +1, from a side or corner segment only the one direction
// that reaches its edge lane.
__device__ __forceinline__ unsigned need_mask(int p) {
  switch (p) {
    case 0: return 1u << 3;                            // E: W-moving
    case 1: return (1u << 4) | (1u << 7) | (1u << 8);  // N: S, SW, SE
    case 2: return 1u << 1;                            // W: E-moving
    case 3: return (1u << 2) | (1u << 5) | (1u << 6);  // S: N, NE, NW
    case 4: return 1u << 7;                            // NE: SW
    case 5: return 1u << 8;                            // NW: SE
    case 6: return 1u << 5;                            // SW: NE
    default: return 1u << 6;                           // SE: NW
  }
}
__device__ __forceinline__ int opp_pos(int p) { return p ^ 2; }

// D2Q9 velocities and opposites (compile-time indices after unrolling)
__host__ __device__ constexpr int cx_of(int i) { return i == 1 || i == 5 || i == 8 ? 1 : i == 3 || i == 6 || i == 7 ? -1 : 0; }
__host__ __device__ constexpr int cy_of(int i) { return i == 2 || i == 5 || i == 6 ? 1 : i == 4 || i == 7 || i == 8 ? -1 : 0; }
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : i <= 4 ? ((i + 1) & 3) + 1 : ((i - 5 + 2) & 3) + 5; }

template <class T>
__device__ __forceinline__ float round_to_storage(float v);
template <>
__device__ __forceinline__ float round_to_storage<float>(float v) { return v; }
template <>
__device__ __forceinline__ float round_to_storage<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}
template <>
__device__ __forceinline__ float round_to_storage<__half>(float v) { return __half2float(__float2half_rn(v)); }

// Relaxed (L2-coherent) accesses of the halo words and the error word.  No
// memory clobber: each poll's use of its value orders it, and the compiler
// may keep the launch-constant descriptor fields in registers across them.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v));
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// List index of segment (y, w) of lattice `lat`, or -1 (outside the step
// rows, or no fluid cell: such a segment's cells are all solid).
__device__ __forceinline__ int list_index(const LatticeView* __restrict__ views, const int* __restrict__ seg_word_off,
                                          const int* __restrict__ seg_flags, const int* __restrict__ seg_offs, int lat,
                                          int y, int w) {
  const LatticeView& L = views[lat];
  const int y0 = first_step_row(L);
  if (w < 0 || w >= L.wpr || y < y0 || y > L.ny - 2) return -1;
  const int i = seg_word_off[lat] + (y - y0) * L.wpr + w;
  return seg_flags[i] ? seg_offs[i] : -1;
}

// What a block knows about its own segments (t: position in its range).
struct OwnInfo {
  int nbq[kResidentMaxOwn][8];  // list index of each neighbouring segment, or -1
  unsigned pub[kResidentMaxOwn];  // directions other blocks read from segment t
  int npairs[kResidentMaxOwn];    // ghost rows segment t needs
  unsigned remote[kResidentMaxOwn];  // bit p: the neighbour at position p belongs to another block
};

// Fill `oi` for the block's range [s0, s1) (every thread of the block calls).
__device__ void describe_range(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                               const int* __restrict__ seg_word_off, const int* __restrict__ seg_flags,
                               const int* __restrict__ seg_offs, int s0, int s1, OwnInfo& oi) {
  for (int t = threadIdx.x; t < s1 - s0; t += blockDim.x) {
    const SegRef sr = segs[s0 + t];
    const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
    unsigned pub = 0, rem = 0;
    int np = 0;
    for (int p = 0; p < 8; ++p) {
      const int nq = list_index(views, seg_word_off, seg_flags, seg_offs, sr.lattice, y + pos_dy(p), w + pos_dw(p));
      oi.nbq[t][p] = nq;
      if (nq >= 0 && (nq < s0 || nq >= s1)) {
        rem |= 1u << p;
        pub |= need_mask(opp_pos(p));
        np += __popc(need_mask(p));
      }
    }
    oi.pub[t] = pub;
    oi.remote[t] = rem;
    oi.npairs[t] = np;
  }
}

__device__ __forceinline__ void block_range(int nseg, int G, int b, int& s0, int& s1) {
  s0 = (int)((long long)b * nseg / G);
  s1 = (int)((long long)(b + 1) * nseg / G);
}

// The block's ghost rows: the (segment, direction) keys (segment << 4 |
// direction) its segments pull from other blocks, each once, ascending, into
// out; returns their number.  raw and first: scratch of 12 n_own ints each
// (a segment needs at most 3 + 3 + 1 + 1 + 4 x 1 rows).  Every thread calls.
__device__ int collect_ghosts(const OwnInfo& oi, int n_own, int* raw, int* first, int* out) {
  __shared__ int s_base[kResidentMaxOwn + 1];
  __shared__ int s_unique;
  if (threadIdx.x == 0) {
    int b = 0;
    for (int t = 0; t < n_own; ++t) {
      s_base[t] = b;
      b += oi.npairs[t];
    }
    s_base[n_own] = b;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_own; t += blockDim.x) {
    int k = s_base[t];
    for (int p = 0; p < 8; ++p) {
      if (!((oi.remote[t] >> p) & 1u)) continue;
      const unsigned m = need_mask(p);
      for (int i = 1; i <= 8; ++i)
        if ((m >> i) & 1u) raw[k++] = (oi.nbq[t][p] << 4) | i;
    }
  }
  __syncthreads();
  const int n = s_base[n_own];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {  // first occurrence of each key
    int f = 1;
    for (int j = 0; j < i && f; ++j) f = raw[j] != raw[i];
    first[i] = f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (first[i]) {
      int pos = 0;
      for (int j = 0; j < n; ++j) pos += first[j] && raw[j] < raw[i];
      out[pos] = raw[i];
    }
  if (threadIdx.x == 0) {
    int c = 0;
    for (int j = 0; j < n; ++j) c += first[j];
    s_unique = c;
  }
  __syncthreads();
  return s_unique;
}

// Position of key in the ascending out[0 .. n), or -1.
__device__ __forceinline__ int find_ghost(const int* out, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = out[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Plan of a resident launch for the current segment list: out[0] = segments,
// out[1] = largest step-buffer size of any block (words of the storage
// type), out[2] = largest ghost-row count, out[3] = 1 if every block's range
// fits kResidentMaxOwn.  out must be zeroed first.
__global__ void k_resident_plan(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                const int* __restrict__ n_segs, const int* __restrict__ seg_word_off,
                                const int* __restrict__ seg_flags, const int* __restrict__ seg_offs, int sm_count,
                                int* __restrict__ out) {
  __shared__ OwnInfo oi;
  __shared__ int raw[12 * kResidentMaxOwn], first[12 * kResidentMaxOwn], uniq[12 * kResidentMaxOwn];
  const int nseg = n_segs[0];
  const int G = resident_grid(nseg, sm_count);
  if (blockIdx.x >= G) return;
  int s0, s1;
  block_range(nseg, G, blockIdx.x, s0, s1);
  if (s1 - s0 > kResidentMaxOwn) {  // the whole list does not fit on the device
    if (threadIdx.x == 0) atomicMax(out + 0, nseg);
    return;
  }
  __syncthreads();
  describe_range(views, segs, seg_word_off, seg_flags, seg_offs, s0, s1, oi);
  __syncthreads();
  const int np = collect_ghosts(oi, s1 - s0, raw, first, uniq);
  if (threadIdx.x == 0) {
    atomicMax(out + 0, nseg);
    atomicMax(out + 1, (s1 - s0) * kSegWords + np * 32 + 1);
    atomicMax(out + 2, np);
    if (blockIdx.x == 0) atomicMax(out + 3, (int)(((long long)nseg + G - 1) / G <= kResidentMaxOwn));
  }
}

// The resident solve: n_steps time steps of the whole set.  words: step-buffer
// size (storage elements) from the plan; halo: [2][halo_cap][9][32] tagged
// words; tags epoch0 + 1 .. epoch0 + n_steps - 1 are published by this
// launch.  Moments go to drho/ux/uy at the last step and to
// drho/ux_prev/uy_prev at step mom_prev (-1: none).  tag_skew is 0, or 1
// under the bounded-wait test hook (every wait then runs out).
template <class T>
__global__ void __launch_bounds__(kResidentMaxWarps * 32, 1)
    k_stream_collide_resident(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                              const int* __restrict__ n_segs, const int* __restrict__ seg_word_off,
                              const int* __restrict__ seg_flags, const int* __restrict__ seg_offs, int words,
                              unsigned long long* __restrict__ halo, int halo_cap, unsigned epoch0, int n_steps,
                              int mom_prev, int* __restrict__ error, unsigned tag_skew) {
  extern __shared__ __align__(16) unsigned char rsm[];
  __shared__ OwnInfo oi;
  __shared__ int s_order[kResidentMaxOwn], s_slot[kResidentMaxOwn];
  __shared__ float2 s_rw[kResidentMaxOwn];  // (rho0, omega) of each slot's lattice
  using P = Pop<T>;
  const int nseg = n_segs[0];
  const int G = gridDim.x;
  int s0, s1;
  block_range(nseg, G, blockIdx.x, s0, s1);
  const int n_own = s1 - s0;  // <= kResidentMaxOwn (checked by the plan)
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // two step buffers, each a multiple of 16 bytes long (so that buffer 1,
  // and the int scratch the prologue keeps in it, start 16-byte aligned),
  // then the ghost-row table
  const int stride = resident_buffer_stride(words);
  T* buf0 = reinterpret_cast<T*>(rsm);
  T* buf1 = buf0 + stride;
  int* gp = reinterpret_cast<int*>(rsm + 2 * (size_t)stride * sizeof(T));
  const int zero = words - 1;  // a word that stays 0 in both buffers
  const int ghost0 = n_own * kSegWords;

  // ---- once per launch: ranges, slots, ghost rows, source offsets ----
  describe_range(views, segs, seg_word_off, seg_flags, seg_offs, s0, s1, oi);
  __syncthreads();
  if (threadIdx.x == 0) {  // slots: published segments first
    int j = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int t = 0; t < n_own; ++t)
        if ((oi.pub[t] != 0) == (pass == 0)) {
          s_order[j] = t;
          s_slot[t] = j;
          ++j;
        }
  }
  // ghost rows, each once (scratch in step buffer 1, unused until step 0 ends)
  int* raw = reinterpret_cast<int*>(buf1);
  const int npairs = collect_ghosts(oi, n_own, raw, raw + 12 * n_own, gp);
  __syncthreads();  // the scratch is overwritten below
  if (threadIdx.x < 32) {
    P::st(buf0 + zero, 0.0f);
    P::st(buf1 + zero, 0.0f);
  }

  const uint16_t* __restrict__ nbs = segment_flags(segs, n_segs);
  // per slot r (j = warp + r W): source offsets of directions 1..8, packed
  // 16-bit; the cell's offset in its lattice; flags; inlet speed
  uint32_t offw[2][4];
  int cell[2], lat[2], qj[2];
  unsigned bits[2];  // bit 0 fluid, 1 inlet, 2 outlet, 3 zero-gradient outlet rule,
                     // 4 constant-density outlet rule, 5 Zou-He ports; bits 8.. publish mask
  float uin[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = warp + r * W;
    offw[r][0] = offw[r][1] = offw[r][2] = offw[r][3] = 0;
    cell[r] = 0;
    lat[r] = 0;
    qj[r] = 0;
    bits[r] = 0;
    uin[r] = 0.0f;
    if (j >= n_own) continue;
    const int t = s_order[j];
    const int q = s0 + t;
    const SegRef sr = segs[q];
    const LatticeView& L = views[sr.lattice];
    const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
    const int x = (w << 5) + lane;
    const uint32_t mc = L.mask[(long long)y * mask_stride(L.wpr) + w];
    const bool fluid = !((mc >> lane) & 1u);
    const bool inlet = x == 0, outlet = x == L.nx - 1;
    const unsigned nb = nbs[(long long)q * 32 + lane];
    const int base = j * kSegWords;
#pragma unroll
    for (int i = 1; i <= 8; ++i) {
      int off = zero;
      const int cx = cx_of(i), cy = cy_of(i);
      const bool unknown = (inlet && cx > 0) || (outlet && cx < 0);
      if (fluid && !unknown) {
        if ((nb >> (opp_of(i) - 1)) & 1u) {  // the source cell is solid: bounce-back
          off = base + opp_of(i) * 32 + lane;
        } else {
          const int sl = lane - cx, dy = -cy;
          const int dw = sl < 0 ? -1 : sl > 31 ? 1 : 0;
          const int slane = sl & 31;
          if (dy == 0 && dw == 0) {
            off = base + i * 32 + slane;
          } else {
            const int p = pos_of(dy, dw);
            const int nq = oi.nbq[t][p];
            if (nq >= s0 && nq < s1) {
              off = s_slot[nq - s0] * kSegWords + i * 32 + slane;
            } else if (nq >= 0) {
              const int g = find_ghost(gp, npairs, (nq << 4) | i);
              if (g >= 0) off = ghost0 + g * 32 + slane;
            }  // nq < 0 cannot happen for a fluid source; the zero word keeps it harmless
          }
        }
      }
      offw[r][(i - 1) >> 1] |= (uint32_t)off << (16 * ((i - 1) & 1));
    }
    cell[r] = y * L.pitch + x;
    lat[r] = sr.lattice;
    qj[r] = q;
    bits[r] = (fluid ? 1u : 0u) | (inlet ? 2u : 0u) | (outlet ? 4u : 0u) |
              (L.outlet_rule == LBM_OUT_NEUMANN ? 8u : 0u) | (L.outlet_rule == LBM_OUT_CONST_RHO ? 16u : 0u) |
              (L.port_scheme == LBM_PORTS_ZOU_HE ? 32u : 0u) | (oi.pub[t] << 8);
    uin[r] = inlet ? L.u_in[y] : 0.0f;
    if (lane == 0) s_rw[j] = make_float2(L.rho0, L.omega);
    // own populations from the canonical layout into step buffer 0
    const T* F = static_cast<const T*>(L.f);
    const int pl = (int)L.plane;
#pragma unroll
    for (int i = 0; i < 9; ++i) buf0[base + i * 32 + lane] = F[i * pl + cell[r]];
  }
  __syncthreads();  // every source offset is known: the keys below may be replaced
  // ghost rows of step 0 from the canonical layout; each key becomes the
  // row's element offset in a halo parity, (segment * 9 + direction) * 32
  for (int g = warp; g < npairs; g += W) {
    const int e = gp[g];
    const SegRef sr = segs[e >> 4];
    const LatticeView& L = views[sr.lattice];
    const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
    const T* F = static_cast<const T*>(L.f);
    buf0[ghost0 + g * 32 + lane] = F[(e & 15) * (int)L.plane + y * L.pitch + (w << 5) + lane];
    __syncwarp();
    if (lane == 0) gp[g] = ((e >> 4) * 9 + (e & 15)) * 32;
  }

  // ---- the time steps ----
  for (int k = 0; k < n_steps; ++k) {
    T* cur = (k & 1) ? buf1 : buf0;
    T* nxt = (k & 1) ? buf0 : buf1;
    int failed = 0;
    if (k > 0) {  // ghost rows of step k: the words of step k - 1, tag epoch0 + k
      const unsigned want = epoch0 + (unsigned)k + tag_skew;
      const unsigned long long* hb = halo + (size_t)((k - 1) & 1) * halo_cap * kSegWords;
      // a warp's rows are g = warp + u W: up to kFetch of them in flight at once
      for (int g0 = warp; g0 < npairs && !failed; g0 += kFetch * W) {
        unsigned long long v[kFetch];
#pragma unroll
        for (int u = 0; u < kFetch; ++u) {
          const int g = g0 + u * W;
          v[u] = g < npairs ? ld_relaxed_u64(hb + gp[g] + lane) : (unsigned long long)want << 32;
        }
        unsigned spins = 0;
        for (;;) {
          bool ready = true;
#pragma unroll
          for (int u = 0; u < kFetch; ++u) ready &= (unsigned)(v[u] >> 32) == want;
          if (__all_sync(kFull, ready)) break;
#pragma unroll
          for (int u = 0; u < kFetch; ++u) {
            const int g = g0 + u * W;
            if (g < npairs && (unsigned)(v[u] >> 32) != want) v[u] = ld_relaxed_u64(hb + gp[g] + lane);
          }
          ++spins;
          if (spins > kResidentSpinLimit ||
              ((spins & 255u) == 0 && __any_sync(kFull, ld_relaxed_s32(error) != 0))) {
            failed = 1;
            break;
          }
        }
        if (failed) break;
#pragma unroll
        for (int u = 0; u < kFetch; ++u) {
          const int g = g0 + u * W;
          if (g < npairs) P::st(cur + ghost0 + g * 32 + lane, __uint_as_float((unsigned)v[u]));
        }
      }
    }
    if (__syncthreads_or(failed)) {
      if (threadIdx.x == 0) atomicExch(error, 1);
      return;  // the global layout keeps the state from before the launch
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int j = warp + r * W;
      if (j >= n_own) break;
      const int base = j * kSegWords;
      float g[9];
      g[0] = P::ld(cur + base + lane);
#pragma unroll
      for (int i = 1; i <= 8; ++i) g[i] = P::ld(cur + ((offw[r][(i - 1) >> 1] >> (16 * ((i - 1) & 1))) & 0xffffu));
      const bool fluid = bits[r] & 1u, inlet = bits[r] & 2u, outlet = bits[r] & 4u;
      if (bits[r] & 8u) {  // zero-gradient outlet: cell nx-2 is the lane to the left
        const float n3 = __shfl_up_sync(kFull, g[3], 1);
        const float n6 = __shfl_up_sync(kFull, g[6], 1);
        const float n7 = __shfl_up_sync(kFull, g[7], 1);
        if (outlet) {
          g[3] = n3;
          g[6] = n6;
          g[7] = n7;
        }
      }
      if (fluid) {
        const float2 rw = s_rw[j];
        const float rho0 = rw.x;
        const int scheme = (bits[r] & 32u) ? LBM_PORTS_ZOU_HE : LBM_PORTS_REGULARIZED;
        if (inlet) {
          inlet_rule(g, uin[r], rho0, scheme);
        } else if (outlet && (bits[r] & 16u)) {
          outlet_rule(g, rho0, scheme);
        }
        float drho, ux, uy;
        bgk(g, rho0, rw.y, drho, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) P::st(nxt + base + i * 32 + lane, g[i]);
        if (k == n_steps - 1) {
          const LatticeView& L = views[lat[r]];
          L.drho[cell[r]] = drho;
          L.ux[cell[r]] = ux;
          L.uy[cell[r]] = uy;
        } else if (k == mom_prev) {
          const LatticeView& L = views[lat[r]];
          L.drho[cell[r]] = drho;
          L.ux_prev[cell[r]] = ux;
          L.uy_prev[cell[r]] = uy;
        }
      }
      const unsigned pub = bits[r] >> 8;
      if (pub && k + 1 < n_steps) {
        unsigned long long* hd = halo + ((size_t)(k & 1) * halo_cap + qj[r]) * kSegWords + lane;
        const unsigned long long tag = (unsigned long long)(epoch0 + (unsigned)k + 1u) << 32;
#pragma unroll
        for (int i = 1; i <= 8; ++i)
          if ((pub >> i) & 1u)
            st_relaxed_u64(hd + i * 32, tag | __float_as_uint(fluid ? round_to_storage<T>(g[i]) : 0.0f));
      }
    }
  }
  // ---- the final state back to the canonical layout ----
  const T* fin = (n_steps & 1) ? buf1 : buf0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = warp + r * W;
    if (j >= n_own || !(bits[r] & 1u)) continue;
    const LatticeView& L = views[lat[r]];
    T* F = static_cast<T*>(L.f);
    const int pl = (int)L.plane;
#pragma unroll
    for (int i = 0; i < 9; ++i) F[i * pl + cell[r]] = fin[j * kSegWords + i * 32 + lane];
  }
}

template <class T>
void* resident_kernel() {
  return (void*)k_stream_collide_resident<T>;
}

void* resident_kernel_for(int precision) {
  switch (precision) {
    case LBM_F32: return resident_kernel<float>();
    case LBM_BF16_SHIFTED: return resident_kernel<__nv_bfloat16>();
    case LBM_F16_SHIFTED: return resident_kernel<__half>();
    default: return nullptr;
  }
}

}  // namespace

size_t resident_smem_bytes(int precision, int words, int pairs) {
  const size_t sb = precision == LBM_F32 ? 4 : 2;
  return 2 * (size_t)resident_buffer_stride(words) * sb + (size_t)(pairs > 0 ? pairs : 1) * sizeof(int);
}

int resident_max_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  // the kernel's static shared memory (the block's segment table) comes on top
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, resident_kernel_for(LBM_F32)) != cudaSuccess) return 0;
  return v - (int)fa.sharedSizeBytes;
}

cudaError_t launch_resident_plan(const LatticeView* views, const SegRef* segs, const int* n_segs,
                                 const int* seg_word_off, const int* seg_flags, const int* seg_offs, int sm_count,
                                 int* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, 4 * sizeof(int), stream);
  if (e != cudaSuccess) return e;
  k_resident_plan<<<sm_count, 64, 0, stream>>>(views, segs, n_segs, seg_word_off, seg_flags, seg_offs, sm_count, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_stream_collide_resident(int precision, const LatticeView* views, const SegRef* segs,
                                           const int* n_segs, const int* seg_word_off, const int* seg_flags,
                                           const int* seg_offs, const ResidentShape& rs,
                                           unsigned long long* halo, int halo_cap, unsigned epoch0, int n_steps,
                                           int mom_prev, int* error, cudaStream_t stream) {
  void* k = resident_kernel_for(precision);
  // under the test hook every wait expects a tag that nobody writes
  unsigned tag_skew = barrier_timeout_test() ? 1u : 0u;
  if (!k || rs.grid < 1 || rs.warps < 1 || rs.warps > kResidentMaxWarps || rs.words < kSegWords + 1 ||
      rs.words > 65536 || n_steps < 1 || halo_cap < 1)
    return cudaErrorInvalidValue;
  const size_t smem = resident_smem_bytes(precision, rs.words, rs.pairs);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&views, (void*)&segs, (void*)&n_segs, (void*)&seg_word_off, (void*)&seg_flags,
                  (void*)&seg_offs, (void*)&rs.words, (void*)&halo, (void*)&halo_cap, (void*)&epoch0,
                  (void*)&n_steps, (void*)&mom_prev, (void*)&error, (void*)&tag_skew};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every block resident: neighbours' words always come
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(rs.grid);
  cfg.blockDim = dim3(32 * rs.warps);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelExC(&cfg, k, args);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

}  // namespace lbm
