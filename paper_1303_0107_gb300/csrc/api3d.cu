// C ABI of the D3Q19 path (include/lbm3d.h): geometry checks, port tables,
// device buffers of one lattice, and the solve / exchange sequence.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "lbm3d_internal.h"

using namespace lbm;

struct lbm3d_handle_s {
  lbm3d_params p{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  View3 v{};
  size_t elem = 4;        // bytes per stored population
  int total_words = 0;    // words of the work-list's rows = its capacity
  int oc_words = 0;       // words of the movable rows (y, z in [1, n-2]): the exchange's word space
  long long ncells = 0;
  std::vector<void*> allocs;
  Seg3* segs = nullptr;
  int* seg_scratch = nullptr;
  int* n_segs = nullptr;      // device {segment tasks, all tasks}
  int* in_rows = nullptr;
  int n_in = 0;
  int* out_rows = nullptr;
  int* out_off = nullptr;
  int n_regions = 0;
  double* d_result = nullptr;
  OcScratch oc{};
  LatticeView* d_one = nullptr;
  int* d_word_off = nullptr;
  int* d_nswap = nullptr;
  float* t_fields = nullptr;  // [4][plane] test-hook field copies (allocated on first use)
  uint8_t* d_cells = nullptr; // [ncells] unpacked mask (allocated on first use)
  double* h_result = nullptr; // pinned
  int* h_small = nullptr;     // pinned: [0] flag, [1..8] info, [9] n_swap, [10..11] task counts
  long long mask_words = 0;
  void* best_f = nullptr;      // saved state of the optimisation loop (allocated on first use)
  uint32_t* best_mask = nullptr;
  float* best_fields = nullptr;
  int nseg = 0;               // tasks in the work-list (host copy)
  int nseg_rows = 0;          // of them, row-segment tasks
  int pack_below = 16;        // segments with fewer fluid cells go to packed tasks
  int resident[3] = {0, 0, 0};  // resident blocks of phase A, B, B with moments at wpb
  int64_t steps_done = 0;
  int64_t fluid = 0;
  bool solved = false;
  int wpb = 8;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double kt_ms = 0.0;
  int64_t kt_launches = 0, kt_updates = 0;

  ~lbm3d_handle_s() {
    if (stream) cudaStreamSynchronize(stream);
    for (void* a : allocs) cudaFree(a);
    if (h_result) cudaFreeHost(h_result);
    if (h_small) cudaFreeHost(h_small);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
  template <class P>
  cudaError_t alloc(P** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = dev_malloc(&p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    *out = static_cast<P*>(p);
    return cudaSuccess;
  }
};

#define CU3(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

namespace {

struct Geometry3 {
  std::vector<float> u_in;     // [nz * ny]
  std::vector<int> in_rows;    // rows z*ny + y of the inlet cells, ascending
  std::vector<int> out_rows;   // outlet rows grouped by region, ascending within each
  std::vector<int> out_off;    // [regions + 1]
  int64_t fluid = 0;
};

inline size_t cell(const lbm3d_params& p, int x, int y, int z) { return ((size_t)z * p.ny + y) * p.nx + x; }

lbm_status check_params3(const lbm3d_params& p) {
  if (p.nx < 4 || p.ny < 3 || p.nz < 3) return fail(LBM_ERR_ARG, "lattice must be at least 4 x 3 x 3");
  if ((long long)p.nx * p.ny * p.nz >= (1ll << 31)) return fail(LBM_ERR_ARG, "nx * ny * nz must be < 2^31");
  if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return fail(LBM_ERR_ARG, "tau must be > 1/2");
  if (!(p.rho0 > 0.0) || !std::isfinite(p.rho0)) return fail(LBM_ERR_ARG, "rho0 must be > 0");
  if (!std::isfinite(p.u_max) || std::fabs(p.u_max) >= 0.5) return fail(LBM_ERR_ARG, "|u_max| must be < 1/2");
  if (p.precision != LBM_F32 && p.precision != LBM_BF16_SHIFTED && p.precision != LBM_F16_SHIFTED)
    return fail(LBM_ERR_ARG, "unknown precision");
  if (p.reinit != LBM_REINIT_WARM && p.reinit != LBM_REINIT_COLD) return fail(LBM_ERR_ARG, "unknown reinit");
  if (p.collision != LBM_COLLIDE_BGK && p.collision != LBM_COLLIDE_REGULARIZED &&
      p.collision != LBM_COLLIDE_SMAGORINSKY)
    return fail(LBM_ERR_ARG, "unknown collision model");
  if (!(p.c_smag >= 0.0) || !std::isfinite(p.c_smag)) return fail(LBM_ERR_ARG, "c_smag must be >= 0");
  if (p.mirror < 0 || p.mirror > 3) return fail(LBM_ERR_ARG, "mirror must be a mask of bits 0 and 1");
  if (p.reserved) return fail(LBM_ERR_ARG, "reserved fields must be 0");
  return LBM_OK;
}

// The geometry rules of include/lbm3d.h, the inlet speeds and the port tables.
lbm_status geometry3(const lbm3d_params& p, const uint8_t* solid, Geometry3& g) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      const bool frame = (y == 0 && !(p.mirror & 1)) || y == ny - 1 || (z == 0 && !(p.mirror & 2)) || z == nz - 1;
      for (int x = 0; x < nx; ++x) {
        const uint8_t s = solid[cell(p, x, y, z)];
        if (s > 1) return fail(LBM_ERR_GEOMETRY, "cell types must be 0 or 1");
        if (frame && !s)
          return fail(LBM_ERR_GEOMETRY, "the faces y = 0, ny-1, z = 0, nz-1 must be solid (but a plane's)");
        g.fluid += !s;
      }
    }
  g.u_in.assign((size_t)ny * nz, 0.0f);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      if (!solid[cell(p, 0, y, z)]) {
        if (solid[cell(p, 1, y, z)]) return fail(LBM_ERR_GEOMETRY, "an inlet cell needs a fluid cell behind it");
        g.in_rows.push_back(z * ny + y);
        // position of the cell centre in its fluid run along y and along z (Sec. 3.3 per axis)
        int lo = y, hi = y;
        while (lo > 0 && !solid[cell(p, 0, lo - 1, z)]) --lo;
        while (hi < ny && !solid[cell(p, 0, hi, z)]) ++hi;
        if ((p.mirror & 1) && lo == 0) lo = -hi;  // half of a run twice as wide, centred on the plane
        const double sy = ((double)(y - lo) + 0.5) / (double)(hi - lo);
        lo = z;
        hi = z;
        while (lo > 0 && !solid[cell(p, 0, y, lo - 1)]) --lo;
        while (hi < nz && !solid[cell(p, 0, y, hi)]) ++hi;
        if ((p.mirror & 2) && lo == 0) lo = -hi;
        const double sz = ((double)(z - lo) + 0.5) / (double)(hi - lo);
        g.u_in[(size_t)z * ny + y] = (float)(p.u_max * (4.0 * sy * (1.0 - sy)) * (4.0 * sz * (1.0 - sz)));
      }
      if (!solid[cell(p, nx - 1, y, z)] && solid[cell(p, nx - 2, y, z)])
        return fail(LBM_ERR_GEOMETRY, "an outlet cell needs a fluid cell before it");
    }
  if (g.in_rows.empty()) return fail(LBM_ERR_GEOMETRY, "no inlet cell");
  // outlet regions: 4-connected in (y, z), numbered by their first cell
  std::vector<int> id((size_t)ny * nz, -1), stack;
  std::vector<std::vector<int>> regions;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      const int k0 = z * ny + y;
      if (id[k0] >= 0 || solid[cell(p, nx - 1, y, z)]) continue;
      const int r = (int)regions.size();
      if (r >= LBM_MAX_OUTLETS) return fail(LBM_ERR_GEOMETRY, "more than LBM_MAX_OUTLETS outlet regions");
      regions.emplace_back();
      id[k0] = r;
      stack.assign(1, k0);
      while (!stack.empty()) {
        const int k = stack.back();
        stack.pop_back();
        regions[r].push_back(k);
        const int qy = k % ny, qz = k / ny;
        const int dy[4] = {1, -1, 0, 0}, dz[4] = {0, 0, 1, -1};
        for (int d = 0; d < 4; ++d) {
          const int yy = qy + dy[d], zz = qz + dz[d];
          if (yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
          const int kk = zz * ny + yy;
          if (id[kk] < 0 && !solid[cell(p, nx - 1, yy, zz)]) {
            id[kk] = r;
            stack.push_back(kk);
          }
        }
      }
    }
  if (regions.empty()) return fail(LBM_ERR_GEOMETRY, "no outlet cell");
  g.out_off.assign(1, 0);
  for (auto& r : regions) {
    std::sort(r.begin(), r.end());
    g.out_rows.insert(g.out_rows.end(), r.begin(), r.end());
    g.out_off.push_back((int)g.out_rows.size());
  }
  return LBM_OK;
}

size_t storage_bytes3(int precision) { return precision == LBM_F32 ? 4 : 2; }

// blocks of one phase launch: one warp per task, at most what is resident at once
int step_blocks(lbm3d_handle h, int which) {
  const int need = (h->nseg + h->wpb - 1) / h->wpb;
  const int cap = h->resident[which] > 0 ? h->resident[which] : need;
  return std::max(1, std::min(need, cap));
}

lbm_status set_shape(lbm3d_handle h, int wpb) {
  const int phase[3] = {0, 1, 1}, mom[3] = {0, 0, 1};
  int res[3];
  for (int k = 0; k < 3; ++k) {
    res[k] = step3_resident_blocks(h->p.precision, phase[k], mom[k], wpb, h->v);
    if (res[k] <= 0) return fail(LBM_ERR_CUDA, "occupancy query of the step kernel failed");
  }
  h->wpb = wpb;
  std::copy(res, res + 3, h->resident);
  return LBM_OK;
}

// (re)build the step work-list and read its length back
lbm_status build_worklist(lbm3d_handle h) {
  CU3(launch_build_segments3(h->v, h->pack_below, h->seg_scratch, h->segs, h->n_segs, h->stream));
  CU3(cudaMemcpyAsync(h->h_small + 10, h->n_segs, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU3(cudaStreamSynchronize(h->stream));
  h->nseg_rows = h->h_small[10];
  h->nseg = h->h_small[11];
  return LBM_OK;
}

lbm_status run_steps(lbm3d_handle h, int64_t n_steps) {
  const int ba = step_blocks(h, 0), bb = step_blocks(h, 1), bm = step_blocks(h, 2);
  CU3(cudaEventRecord(h->ev0, h->stream));
  for (int64_t k = 0; k < n_steps / 2; ++k) {
    const bool last = k == n_steps / 2 - 1;
    CU3(launch_step3(h->p.precision, 0, 0, h->v, h->segs, h->n_segs, ba, h->wpb, h->stream));
    CU3(launch_step3(h->p.precision, 1, last ? 1 : 0, h->v, h->segs, h->n_segs, last ? bm : bb, h->wpb,
                     h->stream));
    if (debug_sync()) CU3(cudaStreamSynchronize(h->stream));
  }
  CU3(cudaEventRecord(h->ev1, h->stream));
  h->kt_launches += n_steps;
  h->kt_updates += n_steps * h->fluid;
  return LBM_OK;
}

lbm_status solve3(lbm3d_handle h, int64_t n_steps, lbm3d_solve_result* out) {
  if (n_steps < 2 || (n_steps & 1)) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  CU3(cudaMemsetAsync(h->v.flag, 0, sizeof(int), h->stream));
  lbm_status st = run_steps(h, n_steps);
  if (st != LBM_OK) return st;
  CU3(launch_observables3(h->v, h->in_rows, h->n_in, h->out_rows, h->out_off, h->n_regions, h->d_result,
                          h->stream));
  CU3(cudaMemcpyAsync(h->h_result, h->d_result, sizeof(double) * (2 + h->n_regions), cudaMemcpyDeviceToHost,
                      h->stream));
  CU3(cudaMemcpyAsync(h->h_small, h->v.flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU3(cudaStreamSynchronize(h->stream));
  float ms = 0.0f;
  CU3(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  h->kt_ms += ms;
  h->steps_done += n_steps;
  h->solved = true;
  std::memset(out, 0, sizeof(*out));
  out->dp = h->h_result[0];
  out->m_in = h->h_result[1];
  out->n_outlets = h->n_regions;
  for (int r = 0; r < h->n_regions; ++r) out->m_out[r] = h->h_result[2 + r];
  out->steps_done = h->steps_done;
  out->fluid_cells = h->fluid;
  if (h->h_small[0] || !std::isfinite(out->dp) || !std::isfinite(out->m_in))
    return fail(LBM_ERR_DIVERGED, "a density or speed of the last step is not finite");
  return LBM_OK;
}

// selection on the fields given (device, padded layout); info to h_small[1..8]
lbm_status select3(lbm3d_handle h, const float* drho, const float* ux, const float* uy, const float* uz,
                   int32_t n_swap) {
  if (n_swap < 0) return fail(LBM_ERR_ARG, "n_swap must be >= 0");
  h->h_small[9] = n_swap;
  CU3(cudaMemcpyAsync(h->d_nswap, h->h_small + 9, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  const double mu = h->p.rho0 * ((h->p.tau - 0.5) / 3.0);
  CU3(launch_oc_select3(h->v, drho, ux, uy, uz, mu, h->d_one, h->d_word_off, h->d_nswap, h->oc, h->stream));
  CU3(cudaMemcpyAsync(h->h_small + 1, h->oc.info, 8 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU3(cudaStreamSynchronize(h->stream));
  if (h->h_small[1 + 3]) return fail(LBM_ERR_DIVERGED, "a score of the exchange is not finite");
  return LBM_OK;
}

lbm_status copy_field(lbm3d_handle h, const void* src, size_t src_pitch_bytes, size_t row_bytes, size_t rows,
                      void* dst, int dst_is_device) {
  CU3(cudaMemcpy2DAsync(dst, row_bytes, src, src_pitch_bytes, row_bytes, rows,
                        dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CU3(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status create3(const lbm3d_params& p, const uint8_t* cells, void* stream, lbm3d_handle h) {
  lbm_status st = check_params3(p);
  if (st != LBM_OK) return st;
  Geometry3 g;
  if ((st = geometry3(p, cells, g)) != LBM_OK) return st;
  h->p = p;
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    CU3(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  CU3(cudaEventCreate(&h->ev0));
  CU3(cudaEventCreate(&h->ev1));
  View3& v = h->v;
  v.nx = p.nx;
  v.ny = p.ny;
  v.nz = p.nz;
  v.nsx = (p.nx + 31) / 32;
  v.nxp = 32 * v.nsx;
  v.ms = v.nsx + 2;
  v.plane = (long long)p.nz * p.ny * v.nxp;
  const char* force64 = std::getenv("LBM3D_INDEX64");
  v.idx64 = ((long long)kQ3 * v.plane >= (1ll << 31) || (force64 && std::strcmp(force64, "1") == 0)) ? 1 : 0;
  // Segments with fewer fluid cells than this are stepped as packed cells (0:
  // none).  16-bit storage is bound by instruction issue, so filling lanes
  // pays down to fuller segments; FP32 by the row pieces a warp touches, so
  // only the sparsest segments are worth packing (measured on the 384 x 192
  // x 192 tree: thresholds 16 and 24 best).
  h->pack_below = p.precision == LBM_F32 ? 16 : 24;
  if (const char* pb = std::getenv("LBM3D_PACK_BELOW")) {
    char* end = nullptr;
    const long n = std::strtol(pb, &end, 10);
    if (end == pb || *end != '\0' || n < 0 || n > 32) return fail(LBM_ERR_ARG, "LBM3D_PACK_BELOW must be 0 .. 32");
    h->pack_below = (int)n;
  }
  v.mirror = p.mirror;
  v.omega = (float)(1.0 / p.tau);
  v.tau = (float)p.tau;
  v.collision = p.collision;
  v.c_smag = (float)p.c_smag;
  v.rho0 = (float)p.rho0;
  h->elem = storage_bytes3(p.precision);
  h->ncells = (long long)p.nx * p.ny * p.nz;
  h->fluid = g.fluid;
  h->total_words = seg3_words(v);
  h->oc_words = (p.ny - 2) * (p.nz - 2) * v.nsx;
  h->n_in = (int)g.in_rows.size();
  h->n_regions = (int)g.out_off.size() - 1;
  // mask: all padding set, fluid cells cleared
  const long long mw = mask3_words(p.ny, p.nz, v.ms);
  h->mask_words = mw;
  std::vector<uint32_t> mask((size_t)mw, 0xffffffffu);
  for (int z = 0; z < p.nz; ++z)
    for (int y = 0; y < p.ny; ++y) {
      uint32_t* row = mask.data() + mask3_row(p.ny, v.ms, y, z) + 1;
      for (int x = 0; x < p.nx; ++x)
        if (!cells[cell(p, x, y, z)]) row[x >> 5] &= ~(1u << (x & 31));
    }
  // the padding rows past a symmetry plane are the mirror image of the layer next to it
  // (the corner row below both planes the image of row (0, 0))
  if (p.mirror & 1)
    for (int z = 0; z < p.nz; ++z)
      std::copy(mask.begin() + mask3_row(p.ny, v.ms, 0, z), mask.begin() + mask3_row(p.ny, v.ms, 0, z) + v.ms,
                mask.begin() + mask3_row(p.ny, v.ms, -1, z));
  if (p.mirror & 2)
    for (int y = -1; y < p.ny; ++y)
      std::copy(mask.begin() + mask3_row(p.ny, v.ms, y, 0), mask.begin() + mask3_row(p.ny, v.ms, y, 0) + v.ms,
                mask.begin() + mask3_row(p.ny, v.ms, y, -1));
  void* f = nullptr;
  CU3(h->alloc(&f, (size_t)kQ3 * v.plane * h->elem));
  v.f = f;
  CU3(h->alloc(&v.mask, sizeof(uint32_t) * mw));
  float* fields = nullptr;
  CU3(h->alloc(&fields, sizeof(float) * 4 * v.plane));
  v.drho = fields;
  v.ux = fields + v.plane;
  v.uy = fields + 2 * v.plane;
  v.uz = fields + 3 * v.plane;
  float* u_in = nullptr;
  CU3(h->alloc(&u_in, sizeof(float) * g.u_in.size()));
  v.u_in = u_in;
  CU3(h->alloc(&v.flag, sizeof(int)));
  CU3(h->alloc(&h->segs, sizeof(Seg3) * h->total_words));
  uint32_t* nbs = nullptr;
  CU3(h->alloc(&nbs, sizeof(uint32_t) * 32 * (size_t)h->total_words));
  v.nbs = nbs;
  uint32_t* cidx = nullptr;
  CU3(h->alloc(&cidx, sizeof(uint32_t) * packed3_capacity(g.fluid)));  // the exchange keeps the fluid count
  v.cidx = cidx;
  CU3(h->alloc(&h->seg_scratch, sizeof(int) * seg3_scratch_ints(h->total_words)));
  CU3(h->alloc(&h->n_segs, 2 * sizeof(int)));
  CU3(h->alloc(&h->in_rows, sizeof(int) * g.in_rows.size()));
  CU3(h->alloc(&h->out_rows, sizeof(int) * g.out_rows.size()));
  CU3(h->alloc(&h->out_off, sizeof(int) * g.out_off.size()));
  CU3(h->alloc(&h->d_result, sizeof(double) * (2 + LBM_MAX_OUTLETS)));
  const size_t tw = (size_t)h->oc_words;
  const size_t cap = (size_t)sel_capacity((int)h->ncells, 1);
  OcScratch& s = h->oc;
  CU3(h->alloc(&s.cnt_f, sizeof(int) * tw));
  CU3(h->alloc(&s.cnt_s, sizeof(int) * tw));
  CU3(h->alloc(&s.off_f, sizeof(int) * (tw + 1)));
  CU3(h->alloc(&s.off_s, sizeof(int) * (tw + 1)));
  CU3(h->alloc(&s.key_f, sizeof(unsigned long long) * h->ncells));
  CU3(h->alloc(&s.key_s, sizeof(unsigned long long) * h->ncells));
  CU3(h->alloc(&s.idx_f, sizeof(int) * h->ncells));
  CU3(h->alloc(&s.idx_s, sizeof(int) * h->ncells));
  CU3(h->alloc(&s.sel_f, sizeof(int) * cap));
  CU3(h->alloc(&s.sel_s, sizeof(int) * cap));
  CU3(h->alloc(&s.info, sizeof(int) * 8));
  CU3(h->alloc(&s.scan_tmp, sizeof(int) * scan_tmp_ints(h->oc_words)));
  CU3(h->alloc(&h->d_one, sizeof(LatticeView)));
  CU3(h->alloc(&h->d_word_off, sizeof(int) * 2));
  CU3(h->alloc(&h->d_nswap, sizeof(int)));
  CU3(cudaMallocHost(&h->h_result, sizeof(double) * (2 + LBM_MAX_OUTLETS)));
  CU3(cudaMallocHost(&h->h_small, sizeof(int) * 16));
  // one-entry table for the shared selection kernel: nx * ny = cell count
  LatticeView one{};
  one.nx = (int)h->ncells;
  one.ny = 1;
  one.sel_off = 0;
  const int word_off[2] = {0, h->oc_words};
  CU3(cudaMemcpyAsync(v.mask, mask.data(), sizeof(uint32_t) * mw, cudaMemcpyHostToDevice, h->stream));
  CU3(cudaMemcpyAsync(u_in, g.u_in.data(), sizeof(float) * g.u_in.size(), cudaMemcpyHostToDevice, h->stream));
  CU3(cudaMemcpyAsync(h->in_rows, g.in_rows.data(), sizeof(int) * g.in_rows.size(), cudaMemcpyHostToDevice,
                      h->stream));
  CU3(cudaMemcpyAsync(h->out_rows, g.out_rows.data(), sizeof(int) * g.out_rows.size(), cudaMemcpyHostToDevice,
                      h->stream));
  CU3(cudaMemcpyAsync(h->out_off, g.out_off.data(), sizeof(int) * g.out_off.size(), cudaMemcpyHostToDevice,
                      h->stream));
  CU3(cudaMemcpyAsync(h->d_one, &one, sizeof(one), cudaMemcpyHostToDevice, h->stream));
  CU3(cudaMemcpyAsync(h->d_word_off, word_off, sizeof(word_off), cudaMemcpyHostToDevice, h->stream));
  CU3(cudaMemsetAsync(v.f, 0, (size_t)kQ3 * v.plane * h->elem, h->stream));  // rest equilibrium: g = 0
  CU3(cudaMemsetAsync(fields, 0, sizeof(float) * 4 * v.plane, h->stream));
  if ((st = build_worklist(h)) != LBM_OK) return st;  // also waits for the uploads above
  return set_shape(h, 8);
}

// populations, mask and fields copied aside (save) or back (restore) on the device
lbm_status keep_state(lbm3d_handle h, bool save) {
  const size_t fb = (size_t)kQ3 * h->v.plane * h->elem, mb = sizeof(uint32_t) * h->mask_words,
               vb = sizeof(float) * 4 * h->v.plane;
  if (!h->best_f) {
    CU3(h->alloc(&h->best_f, fb));
    CU3(h->alloc(&h->best_mask, mb));
    CU3(h->alloc(&h->best_fields, vb));
  }
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (save) {
    CU3(cudaMemcpyAsync(h->best_f, h->v.f, fb, k, h->stream));
    CU3(cudaMemcpyAsync(h->best_mask, h->v.mask, mb, k, h->stream));
    CU3(cudaMemcpyAsync(h->best_fields, h->v.drho, vb, k, h->stream));
    CU3(cudaStreamSynchronize(h->stream));
    return LBM_OK;
  }
  CU3(cudaMemcpyAsync(h->v.f, h->best_f, fb, k, h->stream));
  CU3(cudaMemcpyAsync(h->v.mask, h->best_mask, mb, k, h->stream));
  CU3(cudaMemcpyAsync(h->v.drho, h->best_fields, vb, k, h->stream));
  return build_worklist(h);  // the restored mask has its own segments
}

}  // namespace

extern "C" {

lbm_status lbm3d_create(const lbm3d_params* params, const uint8_t* cell_types, void* cuda_stream,
                        lbm3d_handle* out) {
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || !cell_types) return fail(LBM_ERR_ARG, "params or cell_types is NULL");
  lbm3d_handle h = new lbm3d_handle_s();
  const lbm_status st = create3(*params, cell_types, cuda_stream, h);
  if (st != LBM_OK) {
    delete h;
    return st;
  }
  *out = h;
  return LBM_OK;
}

void lbm3d_destroy(lbm3d_handle h) { delete h; }

lbm_status lbm3d_solve(lbm3d_handle h, int64_t n_steps, lbm3d_solve_result* out) {
  if (!h || !out) return fail(LBM_ERR_ARG, "handle or out is NULL");
  return solve3(h, n_steps, out);
}

lbm_status lbm3d_optimize_step(lbm3d_handle h, int32_t n_swap, int64_t n_steps, lbm3d_opt_result* out) {
  if (!h || !out) return fail(LBM_ERR_ARG, "handle or out is NULL");
  if (!h->solved) return fail(LBM_ERR_ARG, "lbm3d_optimize_step needs a field: call lbm3d_solve first");
  if (n_steps < 2 || (n_steps & 1)) return fail(LBM_ERR_ARG, "n_steps must be even and >= 2");
  lbm_status st = select3(h, h->v.drho, h->v.ux, h->v.uy, h->v.uz, n_swap);
  if (st != LBM_OK) return st;
  const int n = h->h_small[1];
  CU3(launch_oc_apply3(h->p.precision, h->v, h->oc, h->stream));
  if (h->p.reinit == LBM_REINIT_COLD)
    CU3(cudaMemsetAsync(h->v.f, 0, (size_t)kQ3 * h->v.plane * h->elem, h->stream));
  if ((st = build_worklist(h)) != LBM_OK) return st;
  std::memset(out, 0, sizeof(*out));
  out->n_swapped = n;
  out->fluid_count = h->fluid;
  return solve3(h, n_steps, &out->solve);
}

lbm_status lbm3d_optimize(lbm3d_handle h, const lbm_opt_plan* plan, double* dp_history, lbm_opt_summary* out) {
  if (!h || !plan || !out) return fail(LBM_ERR_ARG, "handle, plan or out is NULL");
  const lbm_opt_plan& P = *plan;
  if (P.n_steps < 2 || (P.n_steps % 2) != 0 || P.max_iter < 0 || P.n_swap < 1 || P.patience < 1 ||
      (P.adapt != 0 && P.adapt != 1) || (P.keep_best != 0 && P.keep_best != 1) || P.reserved != 0 ||
      !std::isfinite(P.tol))
    return fail(LBM_ERR_ARG, "plan: n_steps even >= 2, max_iter >= 0, n_swap >= 1, patience >= 1, flags 0/1");
  std::memset(out, 0, sizeof(*out));
  lbm3d_solve_result r;
  lbm_status st = solve3(h, P.n_steps, &r);
  if (st != LBM_OK) return st;
  std::vector<double> hist{r.dp};
  if (dp_history) dp_history[0] = r.dp;
  int best = 0, calm = 0;
  int32_t n_swap = P.n_swap;
  if (P.keep_best && (st = keep_state(h, true)) != LBM_OK) return st;
  for (int k = 1; k <= P.max_iter; ++k) {
    out->iterations = k - 1;
    out->n_swap_final = n_swap;
    lbm3d_opt_result o;
    if ((st = lbm3d_optimize_step(h, n_swap, P.n_steps, &o)) != LBM_OK) return st;
    out->swapped += o.n_swapped;
    const double dp = o.solve.dp;
    hist.push_back(dp);
    if (dp_history) dp_history[k] = dp;
    if (dp < hist[best]) {
      best = k;
      if (P.keep_best && (st = keep_state(h, true)) != LBM_OK) return st;
    }
    if (P.adapt && dp > hist[k - 1]) n_swap = std::max(1, n_swap / 2);
    if (P.tol > 0.0) {
      calm = std::fabs(dp - hist[k - 1]) <= P.tol * std::fabs(dp) ? calm + 1 : 0;
      if (calm >= P.patience) {
        out->stopped = 1;
        break;
      }
    }
  }
  out->iterations = (int32_t)hist.size() - 1;
  out->n_swap_final = n_swap;
  out->best_iter = best;
  out->dp_first = hist.front();
  out->dp_best = hist[best];
  out->dp_last = hist.back();
  if (P.keep_best && best != out->iterations && (st = keep_state(h, false)) != LBM_OK) return st;
  return LBM_OK;
}

lbm_status lbm3d_read_fields(lbm3d_handle h, uint32_t which, void* dst, size_t dst_bytes, int dst_is_device) {
  if (!h || !dst) return fail(LBM_ERR_ARG, "handle or dst is NULL");
  const View3& v = h->v;
  const size_t rows = (size_t)v.nz * v.ny;
  const float* src = nullptr;
  switch (which) {
    case LBM3D_FIELD_DRHO: src = v.drho; break;
    case LBM3D_FIELD_UX: src = v.ux; break;
    case LBM3D_FIELD_UY: src = v.uy; break;
    case LBM3D_FIELD_UZ: src = v.uz; break;
    case LBM3D_FIELD_MASK: {
      if (dst_bytes < (size_t)h->ncells) return fail(LBM_ERR_ARG, "dst too small");
      if (!h->d_cells) CU3(h->alloc(&h->d_cells, (size_t)h->ncells));
      CU3(launch_unpack_mask3(v, h->d_cells, h->stream));
      return copy_field(h, h->d_cells, (size_t)v.nx, (size_t)v.nx, rows, dst, dst_is_device);
    }
    case LBM3D_FIELD_POPS: {
      if (dst_bytes < (size_t)kQ3 * h->ncells * h->elem) return fail(LBM_ERR_ARG, "dst too small");
      return copy_field(h, v.f, (size_t)v.nxp * h->elem, (size_t)v.nx * h->elem, (size_t)kQ3 * rows, dst,
                        dst_is_device);
    }
    default: return fail(LBM_ERR_ARG, "which must be one LBM3D_FIELD_* bit");
  }
  if (dst_bytes < sizeof(float) * h->ncells) return fail(LBM_ERR_ARG, "dst too small");
  return copy_field(h, src, sizeof(float) * v.nxp, sizeof(float) * v.nx, rows, dst, dst_is_device);
}

lbm_status lbm3d_load_state(lbm3d_handle h, const void* pops, size_t bytes, int src_is_device) {
  if (!h || !pops) return fail(LBM_ERR_ARG, "handle or pops is NULL");
  const View3& v = h->v;
  if (bytes != (size_t)kQ3 * h->ncells * h->elem) return fail(LBM_ERR_ARG, "pops has the wrong size");
  const size_t rows = (size_t)kQ3 * v.nz * v.ny;
  CU3(cudaMemcpy2DAsync(v.f, (size_t)v.nxp * h->elem, pops, (size_t)v.nx * h->elem, (size_t)v.nx * h->elem, rows,
                        src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  CU3(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm3d_select_swaps(lbm3d_handle h, const float* drho, const float* ux, const float* uy,
                              const float* uz, int32_t n_swap, int32_t* fluid_idx_out, int32_t* solid_idx_out,
                              int32_t* n_out) {
  if (!h || !drho || !ux || !uy || !uz || !n_out || (n_swap > 0 && (!fluid_idx_out || !solid_idx_out)))
    return fail(LBM_ERR_ARG, "NULL argument");
  const View3& v = h->v;
  if (!h->t_fields) CU3(h->alloc(&h->t_fields, sizeof(float) * 4 * v.plane));
  const float* src[4] = {drho, ux, uy, uz};
  const size_t rows = (size_t)v.nz * v.ny;
  for (int k = 0; k < 4; ++k)
    CU3(cudaMemcpy2DAsync(h->t_fields + k * v.plane, sizeof(float) * v.nxp, src[k], sizeof(float) * v.nx,
                          sizeof(float) * v.nx, rows, cudaMemcpyHostToDevice, h->stream));
  const lbm_status st = select3(h, h->t_fields, h->t_fields + v.plane, h->t_fields + 2 * v.plane,
                                h->t_fields + 3 * v.plane, n_swap);
  if (st != LBM_OK) return st;
  const int n = h->h_small[1];
  *n_out = n;
  if (n > 0) {
    CU3(cudaMemcpyAsync(fluid_idx_out, h->oc.sel_f, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream));
    CU3(cudaMemcpyAsync(solid_idx_out, h->oc.sel_s, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream));
    CU3(cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

lbm_status lbm3d_kernel_time(lbm3d_handle h, int reset, double* ms, int64_t* launches, int64_t* fluid_updates) {
  if (!h || !ms || !launches || !fluid_updates) return fail(LBM_ERR_ARG, "NULL argument");
  *ms = h->kt_ms;
  *launches = h->kt_launches;
  *fluid_updates = h->kt_updates;
  if (reset) {
    h->kt_ms = 0.0;
    h->kt_launches = 0;
    h->kt_updates = 0;
  }
  return LBM_OK;
}

lbm_status lbm3d_debug_task_counts(lbm3d_handle h, int32_t* segment_tasks, int32_t* packed_tasks) {
  if (!h || !segment_tasks || !packed_tasks) return fail(LBM_ERR_ARG, "NULL argument");
  *segment_tasks = h->nseg_rows;
  *packed_tasks = h->nseg - h->nseg_rows;
  return LBM_OK;
}

lbm_status lbm3d_set_block(lbm3d_handle h, int32_t warps_per_block) {
  if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
  if (warps_per_block != 4 && warps_per_block != 8 && warps_per_block != 16)
    return fail(LBM_ERR_ARG, "warps_per_block must be 4, 8 or 16");
  return set_shape(h, warps_per_block);
}

}  // extern "C"
