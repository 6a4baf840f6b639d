// Internal declarations of the D3Q19 path (d3q19.cu kernels, api3d.cu
// handle).  Not part of the public ABI (include/lbm3d.h is).
#pragma once

#include "lbm3d.h"
#include "lbm_internal.h"

namespace lbm {

constexpr int kQ3 = 19;  // D3Q19 populations per cell

// Cell mask of a 3D lattice: one bit per cell, set = solid.  Row (y, z) holds
// the bits of cells x = 0 .. nx-1, bit x & 31 of word 1 + (x >> 5); word 0
// and the words past the last cell are padding (all bits set), and so are the
// bits of x >= nx.  Rows y = -1 .. ny and z = -1 .. nz are stored, the
// padding rows solid: row (y, z) starts at word ((z + 1) (ny + 2) + y + 1) ms,
// ms = words per row.  Every word a kernel forms for a cell of rows
// y in [1, ny-2], z in [1, nz-2] (rows y-1..y+1, z-1..z+1, words w-1..w+1)
// therefore lies inside the allocation; cells outside x = 0 .. nx-1 read as
// solid, which the port rules override.
struct View3 {
  void* f;               // [19][plane] populations, storage type, shifted g = f - w rho0
  uint32_t* mask;        // padded mask (word 0 of row y = -1, z = -1)
  float* drho;           // [plane] rho - rho0 of the last moments step
  float* ux;             // [plane]
  float* uy;             // [plane]
  float* uz;             // [plane]
  const float* u_in;     // [nz * ny] inlet u_x of cell (0, y, z); 0 where no inlet cell
  const uint32_t* nbs;   // [32 per task]: solid flags of the 18 neighbours of each cell of a
                         // segment task that is not open, and of each packed cell (bit i:
                         // x + c_i solid), built with the work-list
  const uint32_t* cidx;  // [32 per packed task]: element indices (z ny + y) nxp + x of the
                         // packed cells, 0xffffffff for padding
  int* flag;             // bit 0: a moments step saw a non-finite value
  long long plane;       // elements per population plane: nz * ny * nxp
  int nx, ny, nz;
  int nxp;               // row pitch in cells: 32 * nsx
  int nsx;               // 32-cell segments per row
  int ms;                // mask words per row: nsx + 2
  float omega, rho0;
  int idx64;             // step kernels index populations in 64 bits (19 planes reach 2^31
                         // elements, or LBM3D_INDEX64=1 in the environment), else in 32
  int collision;         // lbm_collision (non-BGK: the models build of the step kernels)
  int mirror;            // symmetry planes (the mirror build): bit 0 below y = 0, bit 1 below
                         // z = 0; the layer next to a plane may be fluid
  float tau;             // relaxation time (the Smagorinsky root needs it)
  float c_smag;          // Smagorinsky constant
};

__host__ __device__ inline long long mask3_row(int ny, int ms, int y, int z) {
  return ((long long)(z + 1) * (ny + 2) + (y + 1)) * ms;
}
__host__ __device__ inline long long mask3_words(int ny, int nz, int ms) {
  return (long long)(ny + 2) * (nz + 2) * ms;
}
// first row / layer of the step work-list: y = 0 (z = 0) holds fluid only next
// to a symmetry plane below it
__host__ __device__ inline int first_row3(const View3& v) { return (v.mirror & 1) ? 0 : 1; }
__host__ __device__ inline int first_layer3(const View3& v) { return (v.mirror & 2) ? 0 : 1; }
// words of the step work-list's rows: y in [first_row3, ny-2], z in [first_layer3, nz-2]
__host__ __device__ inline int seg3_words(const View3& v) {
  return (v.ny - 1 - first_row3(v)) * (v.nz - 1 - first_layer3(v)) * v.nsx;
}

// Step work-list entry: segment (z * ny + y) * nsx + s (bits 0..29) with
// kSegOpen set when no fluid cell of it has a solid neighbour, and its own
// mask word (bit set = solid), so that the local phase reads no mask.
struct alignas(8) Seg3 {
  int seg;
  uint32_t word;
};
constexpr int kSegIndexMask = (1 << 30) - 1;
constexpr int kSegOpen = 1 << 30;
static_assert(sizeof(Seg3) == 8, "Seg3 layout");

// Step work-list of rows y in [first_row3, ny-2], z in [first_layer3, nz-2]:
// segs lists the segments (z, y, s) holding fluid, in ascending order, one
// warp task each, but for those with fewer than pack_below fluid cells (not
// the first or last word of a row, not on a layer next to a symmetry
// plane): their fluid cells follow as packed tasks of 32 cells, their indices in v.cidx (ascending, padded to whole tasks) and
// their flags in v.nbs after the segment tasks' blocks.  counts = {segment
// tasks, all tasks}.  scratch holds seg3_scratch_ints(total) ints, segs
// total entries, v.nbs 32 total and v.cidx packed3_capacity(fluid cells)
// (packed cells are fluid cells, plus one task's padding), total =
// seg3_words(v).
size_t seg3_scratch_ints(long long total);
size_t packed3_capacity(long long fluid);
cudaError_t launch_build_segments3(const View3& v, int pack_below, int* scratch, Seg3* segs, int* counts,
                                   cudaStream_t stream);

// One time step over the work-list (counts as built above).  phase 0 ("A"): pulls from the
// neighbours' slots and pushes into the slots the neighbours read next
// (its own where the neighbour is solid); phase 1 ("B"): the cell's own
// slots only, leaving F[i][cell] = post-collision population i.  moments
// (phase 1 only): write drho, ux, uy, uz and flag non-finite values.
// Warps stride over the list (blocks of warps_per_block warps); launched as
// a programmatic dependent of the previous kernel on the stream.
cudaError_t launch_step3(int precision, int phase, int moments, const View3& v, const Seg3* segs,
                         const int* counts, int blocks, int warps_per_block, cudaStream_t stream);
// blocks of the given shape resident on the whole device at once (0 on error)
int step3_resident_blocks(int precision, int phase, int moments, int warps_per_block, const View3& v);

// FP64 reductions of the last moments step: result[0] dp, [1] m_in,
// [2 + r] m_out of region r.  in_cells: cells (dense idx) of the inlet, n_in
// of them; out_cells: outlet cells grouped by region, out_off[r] .. out_off[r+1].
cudaError_t launch_observables3(const View3& v, const int* in_cells, int n_in, const int* out_cells,
                                const int* out_off, int n_regions, double* result, cudaStream_t stream);

// Exchange (Sec. 2.2-2.3 on the 6-neighbourhood): candidates and FP64 scores
// from the fields drho/ux/uy/uz given (those of v, or a test field of the
// same layout), then the choice via launch_oc_select_only.  one: a one-entry
// device table (nx = cell count, ny = 1, sel_off = 0); word_off: device
// {0, total} with total = (ny-2)(nz-2) nsx.
cudaError_t launch_oc_select3(const View3& v, const float* drho, const float* ux, const float* uy,
                              const float* uz, double mu, const LatticeView* one, const int* word_off,
                              const int* n_swap, const OcScratch& s, cudaStream_t stream);
cudaError_t launch_oc_apply3(int precision, const View3& v, const OcScratch& s, cudaStream_t stream);

// dense uint8 [nz][ny][nx] <- mask
cudaError_t launch_unpack_mask3(const View3& v, uint8_t* cells, cudaStream_t stream);

}  // namespace lbm
