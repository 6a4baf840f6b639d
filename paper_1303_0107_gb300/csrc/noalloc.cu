// Exchange selection without any device allocation.
//
// Some callers cannot call cudaMalloc: a host application whose caching
// allocator owns all device memory and forbids raw allocations, a loop that
// must never trigger the implicit device synchronisation cudaMalloc/cudaFree
// may cause, or a deployment that reserves every byte of device memory when
// it loads.  lbm_select_swaps_noalloc serves them: the caller passes its own
// device buffers for inputs and outputs, and all intermediate storage (packed
// cell mask, candidate counts, offsets, score keys, indices, picks) lives in
// the file-scope array below, sized for lattices of up to
// LBM_NOALLOC_MAX_CELLS cells.  Every GPU that loads the library holds this
// array until the process exits.
//
// The computation is the same as the handle-based selection (the kernels of
// oc.cu and worklist.cu are reused unchanged), so the chosen cells are
// identical bit for bit.
#include <cstring>
#include <string>

#include "lbm_internal.h"

using namespace lbm;

namespace {

// Scratch layout (byte offsets; every part 256-byte aligned).  Bounds for a
// lattice with nx * ny <= LBM_NOALLOC_MAX_CELLS, nx <= 4096, ny <= 4096:
// mask words (ny + 2) * (ceil(nx / 32) + 2) <= 24576; count / offset words
// ny * ceil(nx / 32) + 1 <= 16384 + 1; candidates per class <= cells; picks
// per class <= cells / 2 + 1.
constexpr int kMaxCells = LBM_NOALLOC_MAX_CELLS;
constexpr int kMaxSide = 4096;
constexpr size_t kAlign = 256;
constexpr size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
constexpr int kMaskWords = 24576;
constexpr int kWordSlots = 16384 + 1;
constexpr int kPickSlots = kMaxCells / 2 + 1;
constexpr size_t kOffView = 0;
constexpr size_t kOffInfo = kOffView + up(sizeof(LatticeView));
constexpr size_t kOffMask = kOffInfo + up(8 * sizeof(int));
constexpr size_t kOffCntF = kOffMask + up((size_t)kMaskWords * 4);
constexpr size_t kOffCntS = kOffCntF + up((size_t)kWordSlots * 4);
constexpr size_t kOffOffF = kOffCntS + up((size_t)kWordSlots * 4);
constexpr size_t kOffOffS = kOffOffF + up((size_t)kWordSlots * 4);
constexpr size_t kOffKeyF = kOffOffS + up((size_t)kWordSlots * 4);
constexpr size_t kOffKeyS = kOffKeyF + up((size_t)kMaxCells * 8);
constexpr size_t kOffIdxF = kOffKeyS + up((size_t)kMaxCells * 8);
constexpr size_t kOffIdxS = kOffIdxF + up((size_t)kMaxCells * 4);
constexpr size_t kOffSelF = kOffIdxS + up((size_t)kMaxCells * 4);
constexpr size_t kOffSelS = kOffSelF + up((size_t)kPickSlots * 4);
constexpr size_t kOffScan = kOffSelS + up((size_t)kPickSlots * 4);
constexpr int kScanTmpInts = 256;  // >= scan_tmp_ints(kWordSlots)
constexpr size_t kOffWords = kOffScan + up((size_t)kScanTmpInts * 4);  // {0, words}, n_swap
constexpr size_t kScratchBytes = kOffWords + up(4 * sizeof(int));

// The shared scratch (about 7.4 MB).  In host code this name is only a
// stand-in for the symbol: its device address comes from
// cudaGetSymbolAddress, looked up on every call below.
static __device__ __align__(256) unsigned char g_select_scratch[kScratchBytes];

lbm_status fail(lbm_status s, const char* what, cudaError_t e = cudaSuccess) {
  std::string msg(what);
  if (e != cudaSuccess) {
    msg += ": ";
    msg += cudaGetErrorString(e);
  }
  set_last_error(msg);  // reported by lbm_last_error()
  return s;
}

// Device address of the scratch array on the current device, looked up on
// every call: once the library's device code is loaded on that device the
// lookup is cheap, and a cached address would dangle after a cudaDeviceReset.
lbm_status scratch_on_current_device(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
  if (e != cudaSuccess || !p) return fail(LBM_ERR_CUDA, "cudaGetSymbolAddress(scratch)", e);
  *out = static_cast<unsigned char*>(p);
  return LBM_OK;
}

// The lattice descriptor and the word table {0, words, n_swap} travel as
// kernel parameters, so the call copies nothing from host memory: one
// thread stores them into the scratch.
__global__ void k_put_descriptor(LatticeView v, int words, int n_swap, LatticeView* __restrict__ view_dst,
                                 int* __restrict__ words_dst) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *view_dst = v;
    words_dst[0] = 0;
    words_dst[1] = words;
    words_dst[2] = n_swap;
  }
}

// picks -> caller's output buffers, count -> *n_out (all on the device)
__global__ void k_copy_picks(const int* __restrict__ info, const int* __restrict__ sel_f,
                             const int* __restrict__ sel_s, int cap, int* __restrict__ fluid_out,
                             int* __restrict__ solid_out, int* __restrict__ n_out) {
  const int n = min(info[0], cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    fluid_out[k] = sel_f[k];
    solid_out[k] = sel_s[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = info[3] ? -1 : n;
}

}  // namespace

extern "C" lbm_status lbm_select_swaps_noalloc(int32_t nx, int32_t ny, double tau, double rho0,
                                               const uint8_t* cell_types, const float* drho,
                                               const float* ux, const float* uy, int32_t n_swap,
                                               int32_t* fluid_idx_out, int32_t* solid_idx_out,
                                               int32_t* n_out, void* cuda_stream) {
  if (!cell_types || !drho || !ux || !uy || !n_out || (n_swap > 0 && (!fluid_idx_out || !solid_idx_out)))
    return fail(LBM_ERR_ARG, "lbm_select_swaps_noalloc: NULL argument");
  if (nx < 4 || ny < 3 || n_swap < 0 || !(tau > 0.5) || !(rho0 > 0))
    return fail(LBM_ERR_ARG, "lbm_select_swaps_noalloc: need nx >= 4, ny >= 3, n_swap >= 0, tau > 1/2, rho0 > 0");
  if (nx > kMaxSide || ny > kMaxSide || (long long)nx * ny > kMaxCells)
    return fail(LBM_ERR_ARG,
                "lbm_select_swaps_noalloc: lattice larger than the built-in scratch allows "
                "(nx, ny <= 4096 and nx * ny <= LBM_NOALLOC_MAX_CELLS)");
  const int wpr = (nx + 31) / 32;
  if (mask_alloc_words(wpr, ny) > kMaskWords || (long long)ny * wpr + 1 > kWordSlots ||
      scan_tmp_ints(ny * wpr) > (size_t)kScanTmpInts)
    return fail(LBM_ERR_ARG, "lbm_select_swaps_noalloc: lattice shape exceeds the built-in scratch");
  unsigned char* base = nullptr;
  lbm_status st = scratch_on_current_device(&base);
  if (st != LBM_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  uint32_t* mask_base = reinterpret_cast<uint32_t*>(base + kOffMask);
  uint32_t* mask = mask_base + mask_origin(wpr);
  LatticeView v;
  std::memset(&v, 0, sizeof(v));
  v.mask = mask;
  v.drho = const_cast<float*>(drho);
  v.ux = const_cast<float*>(ux);
  v.uy = const_cast<float*>(uy);
  v.plane = (long long)nx * ny;
  v.nx = nx;
  v.ny = ny;
  v.pitch = nx;  // the caller's fields are dense [ny][nx]
  v.wpr = wpr;
  v.rho0d = rho0;
  v.mu = rho0 * ((tau - 0.5) / 3.0);
  v.sel_off = 0;
  v.word_off = 0;
  LatticeView* view_dev = reinterpret_cast<LatticeView*>(base + kOffView);
  int* words_dev = reinterpret_cast<int*>(base + kOffWords);  // [0] = 0, [1] = words, [2] = n_swap

  OcScratch s;
  s.cnt_f = reinterpret_cast<int*>(base + kOffCntF);
  s.cnt_s = reinterpret_cast<int*>(base + kOffCntS);
  s.off_f = reinterpret_cast<int*>(base + kOffOffF);
  s.off_s = reinterpret_cast<int*>(base + kOffOffS);
  s.key_f = reinterpret_cast<unsigned long long*>(base + kOffKeyF);
  s.key_s = reinterpret_cast<unsigned long long*>(base + kOffKeyS);
  s.idx_f = reinterpret_cast<int*>(base + kOffIdxF);
  s.idx_s = reinterpret_cast<int*>(base + kOffIdxS);
  s.sel_f = reinterpret_cast<int*>(base + kOffSelF);
  s.sel_s = reinterpret_cast<int*>(base + kOffSelS);
  s.info = reinterpret_cast<int*>(base + kOffInfo);
  s.scan_tmp = reinterpret_cast<int*>(base + kOffScan);

  cudaError_t e;
  // the array keeps the previous call's contents: the mask padding must read
  // as wall, so the whole mask region is reset (the selection clears its own
  // counters; every other part is fully written before it is read)
  k_put_descriptor<<<1, 32, 0, stream>>>(v, ny * wpr, n_swap, view_dev, words_dev);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(LBM_ERR_CUDA, "store lattice descriptor", e);
  if ((e = cudaMemsetAsync(mask_base, 0xff, (size_t)mask_alloc_words(wpr, ny) * 4, stream)) != cudaSuccess)
    return fail(LBM_ERR_CUDA, "reset mask", e);
  if ((e = launch_pack_mask(cell_types, nx, ny, wpr, mask, stream)) != cudaSuccess)
    return fail(LBM_ERR_CUDA, "pack mask", e);
  if ((e = launch_oc_select(view_dev, words_dev, 1, ny * wpr, words_dev + 2, s, stream)) != cudaSuccess)
    return fail(LBM_ERR_CUDA, "selection kernels", e);
  k_copy_picks<<<(n_swap + 255) / 256 > 0 ? (n_swap + 255) / 256 : 1, 256, 0, stream>>>(
      s.info, s.sel_f, s.sel_s, n_swap, fluid_idx_out, solid_idx_out, n_out);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(LBM_ERR_CUDA, "copy picks", e);
  return LBM_OK;
}
