// Geometry to bit mask, tile work-list, fluid count, block scan.
//
// The cell map of Sec. 3.3 (fluid / solid cells; inlet and outlet cells are
// the fluid cells of the first and last columns) is kept as one bit per cell:
// word w of row y holds cells x = 32w .. 32w+31, bit set = solid.  Bits past
// the last column are set, so padding behaves as wall.
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

// 1 for every tile (32 x kTileY) with a fluid cell in rows 1..ny-2.
__global__ void k_tile_flags(const uint32_t* __restrict__ mask, int ny, int wpr, int tiles_y,
                             int* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tiles_y * wpr) return;
  const int ty = i / wpr, w = i - ty * wpr;
  int any = 0;
  for (int r = 0; r < kTileY; ++r) {
    const int y = ty * kTileY + r;
    if (y >= 1 && y <= ny - 2 && mask[(long long)y * mask_stride(wpr) + w] != 0xffffffffu) any = 1;
  }
  flags[i] = any;
}

__global__ void k_tile_scatter(const int* __restrict__ flags, const int* __restrict__ offsets,
                               int tiles_y, int wpr, int lattice, TileRef* __restrict__ tiles,
                               int* __restrict__ n_tiles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = tiles_y * wpr;
  if (i == 0) *n_tiles = offsets[n];
  if (i >= n || !flags[i]) return;
  const int ty = i / wpr, w = i - ty * wpr;
  TileRef t;
  t.lattice = lattice;
  t.x0 = w * 32;
  t.y0 = ty * kTileY;
  t.reserved = 0;
  tiles[offsets[i]] = t;
}

__global__ void k_count_fluid(const uint32_t* __restrict__ mask, int nx, int ny, int wpr,
                              unsigned long long* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = 0;
  if (i < ny * wpr) {
    const int y = i / wpr, w = i - y * wpr;
    const int valid = min(32, nx - w * 32);
    const uint32_t vmask = valid >= 32 ? 0xffffffffu : ((1u << valid) - 1u);
    c = __popc(~mask[(long long)y * mask_stride(wpr) + w] & vmask);
  }
  // warp sum, then one atomic per warp (integer: order does not matter)
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// Exclusive scan of n ints by one block of 1024 threads; out[n] = total.
// Each thread sums a contiguous chunk, the chunk sums are scanned in shared
// memory, then each thread writes its chunk: a fixed order for any input.
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ in, int* __restrict__ out, int n) {
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

__global__ void k_rho_from_drho(const float* __restrict__ drho, float rho0,
                                const uint32_t* __restrict__ mask, int nx, int ny, int pitch,
                                int wpr, float* __restrict__ rho) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nx * ny) return;
  const int y = (int)(i / nx), x = (int)(i - (long long)y * nx);
  const bool solid = (mask[(long long)y * mask_stride(wpr) + (x >> 5)] >> (x & 31)) & 1u;
  rho[i] = solid ? 0.0f : rho0 + drho[(size_t)y * pitch + x];
}

inline int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

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

cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t stream) {
  k_scan<<<1, 1024, 0, stream>>>(in, out, n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_build_tiles(const uint32_t* mask, int nx, int ny, int wpr, int lattice,
                               int* counts, TileRef* tiles, int* n_tiles, cudaStream_t stream) {
  (void)nx;
  const int tiles_y = (ny + kTileY - 1) / kTileY;
  const int n = tiles_y * wpr;
  int* flags = counts;
  int* offsets = counts + n;  // counts holds 2n + 1 ints
  k_tile_flags<<<blocks_for(n, 256), 256, 0, stream>>>(mask, ny, wpr, tiles_y, flags);
  k_scan<<<1, 1024, 0, stream>>>(flags, offsets, n);
  k_tile_scatter<<<blocks_for(n, 256), 256, 0, stream>>>(flags, offsets, tiles_y, wpr, lattice, tiles,
                                                         n_tiles);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_count_fluid(const uint32_t* mask, int nx, int ny, int wpr, unsigned long long* count,
                               cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  k_count_fluid<<<blocks_for((long long)ny * wpr, 256), 256, 0, stream>>>(mask, nx, ny, wpr, count);
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
