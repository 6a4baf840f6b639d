// Geometry to bit mask, row-segment work-list, fluid count, scans.
//
// The cell map of Sec. 3.3 (fluid / solid cells; inlet and outlet cells are
// the fluid cells of the first and last columns) is kept as one bit per cell:
// word w of row y holds cells x = 32w .. 32w+31, bit set = solid.  Bits past
// the last column are set, so padding behaves as wall.  Kernels over a set of
// lattices number the words of all lattices consecutively and find the
// lattice of a word by binary search in the per-lattice offsets.
#include "lbm_internal.h"

namespace lbm {
namespace {

__global__ void k_pack_mask(const uint8_t* __restrict__ cells, int nx, int ny, int wpr,
                            uint32_t* __restrict__ mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ny * wpr) return;
  const int y = i / wpr, w = i - y * wpr;
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int x = w * 32 + b;
    const bool solid = (x >= nx) || cells[(size_t)y * nx + x] != 0;
    word |= (solid ? 1u : 0u) << b;
  }
  mask[(long long)y * mask_stride(wpr) + w] = word;
}

__global__ void k_unpack_mask(const uint32_t* __restrict__ mask, int nx, int ny, int wpr,
                              uint8_t* __restrict__ cells) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nx * ny) return;
  const int y = (int)(i / nx), x = (int)(i - (long long)y * nx);
  cells[i] = (mask[(long long)y * mask_stride(wpr) + (x >> 5)] >> (x & 31)) & 1u;
}

// Step-row words of all lattices in one index space: word i belongs to
// lattice l = find_lattice(seg_word_off, n, i), row first_step_row + (i - off) / wpr.
__device__ __forceinline__ void seg_word(const LatticeView* __restrict__ views,
                                         const int* __restrict__ seg_word_off, int n, int i, int& l,
                                         int& y, int& w) {
  l = find_lattice(seg_word_off, n, i);
  const int wpr = views[l].wpr;
  const int local = i - seg_word_off[l];
  const int r = local / wpr;
  y = first_step_row(views[l]) + r;
  w = local - r * wpr;
}

// 1 for every row segment (row y in 1..ny-2, word w) holding a fluid cell
__global__ void k_segment_flags(const LatticeView* __restrict__ views, const int* __restrict__ seg_word_off,
                                int n, int total, int* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int l, y, w;
  seg_word(views, seg_word_off, n, i, l, y, w);
  const LatticeView& L = views[l];
  flags[i] = L.mask[(long long)y * mask_stride(L.wpr) + w] != 0xffffffffu ? 1 : 0;
}

__global__ void k_segment_scatter(const LatticeView* __restrict__ views, const int* __restrict__ seg_word_off,
                                  int n, int total, int capacity, const int* __restrict__ flags,
                                  const int* __restrict__ offsets, SegRef* __restrict__ segs,
                                  int* __restrict__ n_segs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    n_segs[0] = offsets[total];
    n_segs[1] = capacity;
  }
  if (i >= total || !flags[i]) return;
  int l, y, w;
  seg_word(views, seg_word_off, n, i, l, y, w);
  SegRef r;
  r.lattice = l;
  r.yw = (y << kSegWordBits) | w;
  segs[offsets[i]] = r;
}

// Neighbour flags of every cell of the list's segments (one warp per entry,
// lane l -> cell 32 w + l): the padded mask makes words w-1, w+1 of rows
// y-1..y+1 exist and read as wall outside the lattice.  Next to a symmetry
// plane, the padding row below row 0 holds row 0's image, and row-0 cells
// are marked (their S neighbour is the plane).
__global__ void k_segment_flags16(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                  const int* __restrict__ n_segs, uint16_t* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int nseg = n_segs[0];
  const int stride = (gridDim.x * blockDim.x) >> 5;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nseg; t += stride) {
    const SegRef sr = segs[t];
    const LatticeView& L = views[sr.lattice];
    const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
    const int ms = mask_stride(L.wpr);
    const uint32_t* mr = L.mask + (long long)y * ms;
    const uint32_t* rn = mr + ms;
    const uint32_t* rs = mr - ms;
    const uint32_t mc = mr[w], mn = rn[w], msth = rs[w];
    const uint32_t eC = __funnelshift_r(mc, mr[w + 1], 1), wC = __funnelshift_l(mr[w - 1], mc, 1);
    const uint32_t eN = __funnelshift_r(mn, rn[w + 1], 1), wN = __funnelshift_l(rn[w - 1], mn, 1);
    const uint32_t eS = __funnelshift_r(msth, rs[w + 1], 1), wS = __funnelshift_l(rs[w - 1], msth, 1);
    unsigned nb = ((eC >> lane) & 1u) | (((mn >> lane) & 1u) << 1) | (((wC >> lane) & 1u) << 2) |
                  (((msth >> lane) & 1u) << 3) | (((eN >> lane) & 1u) << 4) | (((wN >> lane) & 1u) << 5) |
                  (((wS >> lane) & 1u) << 6) | (((eS >> lane) & 1u) << 7);
    if (y == 0 && L.mirror) nb |= kNbS | kNbMirror;
    flags[(long long)t * 32 + lane] = (uint16_t)nb;
  }
}

// fluid cells per lattice over all words (rows 0..ny-1) of all lattices
__global__ void k_count_fluid(const LatticeView* __restrict__ views, const int* __restrict__ word_off, int n,
                              int total, unsigned long long* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int l = find_lattice(word_off, n, i);
  const LatticeView& L = views[l];
  const int local = i - word_off[l];
  const int y = local / L.wpr, w = local - y * L.wpr;
  const int valid = min(32, L.nx - w * 32);
  const uint32_t vmask = valid >= 32 ? 0xffffffffu : ((1u << valid) - 1u);
  const int c = __popc(~L.mask[(long long)y * mask_stride(L.wpr) + w] & vmask);
  if (c) atomicAdd(count + l, (unsigned long long)c);  // integer: order does not matter
}

// Exclusive scan of n ints by one block of 1024 threads; out[n] = total.
// Each thread sums a contiguous chunk, the chunk sums are scanned in shared
// memory, then each thread writes its chunk: a fixed order for any input.
// Used for small inputs and for the top level of the multi-block scan.
__global__ void __launch_bounds__(1024) k_scan_chunked(const int* __restrict__ in, int* __restrict__ out,
                                                       int n) {
  __shared__ int sums[1024];
  const int tid = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int begin = min(n, tid * per), end = min(n, begin + per);
  int s = 0;
  for (int i = begin; i < end; ++i) s += in[i];
  sums[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = tid >= off ? sums[tid - off] : 0;
    __syncthreads();
    sums[tid] += v;
    __syncthreads();
  }
  int run = sums[tid] - s;  // exclusive prefix of this chunk
  for (int i = begin; i < end; ++i) {
    const int v = in[i];
    out[i] = run;
    run += v;
  }
  if (tid == 1023) out[n] = sums[1023];
}

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // elements per block

// Level 1: exclusive scan inside each tile of kScanTile elements; tile sums
// go to block_sums[b].
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int* __restrict__ in,
                                                             int* __restrict__ out, int n,
                                                             int* __restrict__ block_sums) {
  __shared__ int warp_sums[kScanThreads / 32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int v[kScanItems];
  int t = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    t += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = t;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int ws = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += u;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = ws;  // inclusive
  }
  __syncthreads();
  int run = incl - t + (warp > 0 ? warp_sums[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = warp_sums[kScanThreads / 32 - 1];
}

// Level 3: add each tile's offset; out[n] = total.
__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ block_offsets,
                           int nb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += block_offsets[i / kScanTile];
  if (i == 0) out[n] = block_offsets[nb];
}

__global__ void k_rho_from_drho(const float* __restrict__ drho, float rho0,
                                const uint32_t* __restrict__ mask, int nx, int ny, int pitch,
                                int wpr, float* __restrict__ rho) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nx * ny) return;
  const int y = (int)(i / nx), x = (int)(i - (long long)y * nx);
  const bool solid = (mask[(long long)y * mask_stride(wpr) + (x >> 5)] >> (x & 31)) & 1u;
  rho[i] = solid ? 0.0f : rho0 + drho[(size_t)y * pitch + x];
}

// Fluid cells of list segment q into cnt[q] (0 past the list).
__global__ void k_segment_cell_counts(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                      const int* __restrict__ n_segs, int capacity, int* __restrict__ cnt) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= capacity) return;
  int c = 0;
  if (q < n_segs[0]) {
    const SegRef sr = segs[q];
    const LatticeView& L = views[sr.lattice];
    const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
    c = __popc(~L.mask[(long long)y * mask_stride(L.wpr) + w]);  // bits past nx are set: solid
  }
  cnt[q] = c;
}

// The compacted list: one warp per segment, each fluid lane writes its entry
// at cpre[q] + (fluid lanes below it).
__global__ void k_scatter_cells(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                                const int* __restrict__ n_segs, const int* __restrict__ cpre,
                                CellRef* __restrict__ cells) {
  const int lane = threadIdx.x & 31;
  const int nseg = n_segs[0];
  const uint16_t* nbs = segment_flags(segs, n_segs);
  const int stride = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nseg; q += stride) {
    const SegRef sr = segs[q];
    const LatticeView& L = views[sr.lattice];
    const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
    const uint32_t fl = ~L.mask[(long long)y * mask_stride(L.wpr) + w];
    if (!((fl >> lane) & 1u)) continue;
    const int x = (w << 5) + lane;
    CellRef r;
    r.c = y * L.pitch + x;
    r.meta = (unsigned)sr.lattice | ((unsigned)nbs[(long long)q * 32 + lane] << kCellLatticeBits) |
             (x == 0 ? 1u << 29 : 0u) | (x == L.nx - 1 ? 1u << 30 : 0u);
    cells[cpre[q] + __popc(fl & ((1u << lane) - 1u))] = r;
  }
}

// Interior window (row y, words 2p and 2p+1): its 64 cells and all their
// neighbours fluid, i.e. rows y-1..y+1 fluid over cells 64p-1 .. 64p+64.
// The columns beyond the inlet and the outlet read as wall, so such a window
// holds no port cell; words 2p-1 and 2p+2 exist in the padded mask whenever
// word 2p+1 is a lattice word.
__device__ __forceinline__ bool window_interior(const LatticeView& L, int y, int p) {
  const int w = 2 * p;
  if (L.mirror || w + 1 >= L.wpr) return false;
  const int ms = mask_stride(L.wpr);
#pragma unroll
  for (int r = -1; r <= 1; ++r) {
    const uint32_t* m = L.mask + (long long)(y + r) * ms;
    if ((m[w] | m[w + 1]) != 0u || (m[w - 1] >> 31) != 0u || (m[w + 2] & 1u) != 0u) return false;
  }
  return true;
}

// 1 where list segment q opens a paired task: the first word of an interior
// window, or a segment outside interior windows (0 past the list)
__global__ void k_pair_emit(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                            const int* __restrict__ n_segs, int capacity, int* __restrict__ emit) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= capacity) return;
  int e = 0;
  if (q < n_segs[0]) {
    const SegRef sr = segs[q];
    const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
    e = ((w & 1) && window_interior(views[sr.lattice], y, w >> 1)) ? 0 : 1;
  }
  emit[q] = e;
}

// Both words of an interior window are in the list (they hold fluid), next
// to each other; the even one writes the window's entry.
__global__ void k_pair_scatter(const LatticeView* __restrict__ views, const SegRef* __restrict__ segs,
                               const int* __restrict__ n_segs, const int* __restrict__ emit,
                               const int* __restrict__ off, SegRef* __restrict__ tasks) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_segs[0] || !emit[q]) return;
  const SegRef sr = segs[q];
  const int y = sr.yw >> kSegWordBits, w = sr.yw & ((1 << kSegWordBits) - 1);
  SegRef t = sr;
  if (!(w & 1) && window_interior(views[sr.lattice], y, w >> 1)) {
    t.lattice = sr.lattice | kPairTask;
    t.yw = (y << kSegWordBits) | (w >> 1);
  }
  tasks[off[q]] = t;
}

inline int blocks_for(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_pack_mask(const uint8_t* cells, int nx, int ny, int wpr, uint32_t* mask,
                             cudaStream_t stream) {
  k_pack_mask<<<blocks_for((long long)ny * wpr, 256), 256, 0, stream>>>(cells, nx, ny, wpr, mask);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack_mask(const uint32_t* mask, int nx, int ny, int wpr, uint8_t* cells,
                               cudaStream_t stream) {
  k_unpack_mask<<<blocks_for((long long)nx * ny, 256), 256, 0, stream>>>(mask, nx, ny, wpr, cells);
  count_launches(1);
  return cudaGetLastError();
}

size_t scan_tmp_ints(long long n) {
  const size_t nb = (size_t)((n + kScanTile - 1) / kScanTile);
  return 2 * nb + 2;
}

cudaError_t launch_scan(const int* in, int* out, int n, int* tmp, cudaStream_t stream) {
  if (n <= kScanTile) {  // one level is enough
    k_scan_chunked<<<1, 1024, 0, stream>>>(in, out, n);
    count_launches(1);
    return cudaGetLastError();
  }
  const int nb = (n + kScanTile - 1) / kScanTile;
  int* sums = tmp;
  int* offs = tmp + nb + 1;
  k_scan_tiles<<<nb, kScanThreads, 0, stream>>>(in, out, n, sums);
  k_scan_chunked<<<1, 1024, 0, stream>>>(sums, offs, nb);
  k_scan_add<<<blocks_for(n, 256), 256, 0, stream>>>(out, n, offs, nb);
  count_launches(3);
  return cudaGetLastError();
}

size_t segment_scratch_ints(long long total_words) {
  return 2 * (size_t)total_words + 1 + scan_tmp_ints(total_words);
}

cudaError_t launch_build_segments(const LatticeView* views, const int* seg_word_off, int n_lattices,
                                  int total, int capacity, int* scratch, SegRef* segs, int* n_segs,
                                  cudaStream_t stream) {
  int* flags = scratch;
  int* offsets = scratch + total;      // total + 1
  int* tmp = scratch + 2 * total + 1;  // scan_tmp_ints(total)
  k_segment_flags<<<blocks_for(total, 256), 256, 0, stream>>>(views, seg_word_off, n_lattices, total, flags);
  count_launches(1);
  cudaError_t e = launch_scan(flags, offsets, total, tmp, stream);
  if (e != cudaSuccess) return e;
  k_segment_scatter<<<blocks_for(total, 256), 256, 0, stream>>>(views, seg_word_off, n_lattices, total, capacity,
                                                                flags, offsets, segs, n_segs);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_segment_flags16<<<blocks_for((long long)total * 32, 256), 256, 0, stream>>>(
      views, segs, n_segs, reinterpret_cast<uint16_t*>(segs + capacity));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_build_cells(const LatticeView* views, const SegRef* segs, const int* n_segs, int capacity,
                               int* cnt, int* cpre, int* tmp, CellRef* cells, cudaStream_t stream) {
  k_segment_cell_counts<<<blocks_for(capacity, 256), 256, 0, stream>>>(views, segs, n_segs, capacity, cnt);
  count_launches(1);
  cudaError_t e = launch_scan(cnt, cpre, capacity, tmp, stream);
  if (e != cudaSuccess) return e;
  k_scatter_cells<<<blocks_for((long long)capacity * 32, 256), 256, 0, stream>>>(views, segs, n_segs, cpre, cells);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_build_pairs(const LatticeView* views, const SegRef* segs, const int* n_segs, int capacity,
                               int* emit, int* off, int* tmp, SegRef* tasks, cudaStream_t stream) {
  k_pair_emit<<<blocks_for(capacity, 256), 256, 0, stream>>>(views, segs, n_segs, capacity, emit);
  count_launches(1);
  cudaError_t e = launch_scan(emit, off, capacity, tmp, stream);
  if (e != cudaSuccess) return e;
  k_pair_scatter<<<blocks_for(capacity, 256), 256, 0, stream>>>(views, segs, n_segs, emit, off, tasks);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_count_fluid(const LatticeView* views, const int* word_off, int n_lattices, int total,
                               unsigned long long* count, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long) * n_lattices, stream);
  if (e != cudaSuccess) return e;
  k_count_fluid<<<blocks_for(total, 256), 256, 0, stream>>>(views, word_off, n_lattices, total, count);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rho_from_drho(const float* drho, float rho0, const uint32_t* mask, int nx, int ny,
                                 int pitch, int wpr, float* rho_dense, cudaStream_t stream) {
  k_rho_from_drho<<<blocks_for((long long)nx * ny, 256), 256, 0, stream>>>(drho, rho0, mask, nx, ny,
                                                                          pitch, wpr, rho_dense);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace lbm
