// Heuristic optimality criterion and the equal-count exchange of Sec. 2.2-2.3,
// for every lattice of a set in one launch per stage.
//
//   scores   interface fluid cells: dynamic pressure q = 1/2 rho |u|^2 (Eq. 6);
//            interface solid cells: sigma = sum over fluid 4-neighbours n (E, N,
//            W, S order) of mu |u_t(n)| / 0.5, u_t = u_y across a vertical face,
//            u_x across a horizontal one (Eq. 5).  FP64, every operation
//            rounded separately (no fused multiply-add), in the same order as
//            a plain sequential statement, so that a given FP32 field gives
//            bit-identical scores on any machine.
//   select   n = min(n_swap, #fluid candidates, #solid candidates); the n fluid
//            candidates of smallest (q, idx) and the n solid candidates of
//            largest sigma, ties to the smaller idx.  Exact 96-bit radix select
//            (64-bit order-preserving score key, 32-bit cell index), one block
//            per (class, lattice).
//   apply    flip the 2n mask bits at once; new fluid cells start from the
//            rest equilibrium of rho0 (shifted populations 0).
//
// Interface / movable cells: 4-neighbourhood; columns 0, 1, nx-2, nx-1 and
// rows 0, ny-1 never move.  Candidate enumeration works on whole mask words
// with bit operations; the words of all lattices are numbered consecutively,
// so candidates come out lattice by lattice in ascending cell index.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {
namespace {

struct WordMasks {
  uint32_t fluid_cand, solid_cand, e, w, n, s;
};

__device__ __forceinline__ uint32_t region_bits(int w, int nx) {
  // bits b with 2 <= 32w + b <= nx - 3
  uint32_t m = 0xffffffffu;
  const int x0 = w * 32;
  if (x0 < 2) m &= ~((1u << (2 - x0)) - 1u);
  const int hi = nx - 3 - x0;  // last allowed bit
  if (hi < 0) return 0u;
  if (hi < 31) m &= (2u << hi) - 1u;
  return m;
}

// Connectivity guard: bits of the cells whose 4-connectivity number is 1,
//   N4 = sum over k in {E, N, W, S} of f_k (1 - f_k+1 f_k+2),
// f the fluid flags of the eight neighbours counter-clockwise from E -- the
// fluid cells that may turn solid without separating their fluid
// 4-neighbours within the 3 x 3 block (the same rule as the oracle's).
__device__ __forceinline__ uint32_t simple_bits(const uint32_t* row, int ms, int w, uint32_t e, uint32_t wb,
                                                uint32_t n, uint32_t s) {
  const uint32_t* rn = row + ms;
  const uint32_t* rs = row - ms;
  const uint32_t ne = __funnelshift_r(rn[w], rn[w + 1], 1), nw = __funnelshift_l(rn[w - 1], rn[w], 1);
  const uint32_t se = __funnelshift_r(rs[w], rs[w + 1], 1), sw = __funnelshift_l(rs[w - 1], rs[w], 1);
  // fluid flags (mask bit set = solid)
  const uint32_t fE = ~e, fNE = ~ne, fN = ~n, fNW = ~nw, fW = ~wb, fSW = ~sw, fS = ~s, fSE = ~se;
  const uint32_t t1 = fE & ~(fNE & fN), t3 = fN & ~(fNW & fW), t5 = fW & ~(fSW & fS), t7 = fS & ~(fSE & fE);
  const uint32_t any = t1 | t3 | t5 | t7;
  const uint32_t two = (t1 & t3) | (t5 & t7) | ((t1 | t3) & (t5 | t7));
  return any & ~two;
}

__device__ __forceinline__ WordMasks word_masks(const uint32_t* __restrict__ mask, int nx, int ny,
                                                int wpr, int y, int w, int guard) {
  WordMasks r{0, 0, 0, 0, 0, 0};
  if (y < 1 || y > ny - 2) return r;
  const int ms = mask_stride(wpr);
  const uint32_t* row = mask + (long long)y * ms;
  const uint32_t mc = row[w];
  const uint32_t cw = row[w - 1], ce = row[w + 1];  // padding words read as wall
  r.e = __funnelshift_r(mc, ce, 1);
  r.w = __funnelshift_l(cw, mc, 1);
  r.n = row[w + ms];
  r.s = row[w - ms];
  const uint32_t reg = region_bits(w, nx);
  r.fluid_cand = ~mc & (r.e | r.w | r.n | r.s) & reg;
  if (guard) r.fluid_cand &= simple_bits(row, ms, w, r.e, r.w, r.n, r.s);
  r.solid_cand = mc & (~r.e | ~r.w | ~r.n | ~r.s) & reg;
  return r;
}

// word i of the concatenated word space -> lattice l, row y, word w
__device__ __forceinline__ void word_of(const LatticeView* __restrict__ views,
                                        const int* __restrict__ word_off, int n, int i, int& l,
                                        int& y, int& w) {
  l = find_lattice(word_off, n, i);
  const int wpr = views[l].wpr;
  const int local = i - word_off[l];
  y = local / wpr;
  w = local - y * wpr;
}

__global__ void k_oc_count(const LatticeView* __restrict__ views, const int* __restrict__ word_off, int n,
                           int total, int* __restrict__ cnt_f, int* __restrict__ cnt_s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int l, y, w;
  word_of(views, word_off, n, i, l, y, w);
  const LatticeView& L = views[l];
  const WordMasks m = word_masks(L.mask, L.nx, L.ny, L.wpr, y, w, L.guard);
  cnt_f[i] = __popc(m.fluid_cand);
  cnt_s[i] = __popc(m.solid_cand);
}

// order-preserving map of a double to an unsigned key (-0 folded onto +0)
__device__ __forceinline__ unsigned long long order_key(double v) {
  v = __dadd_rn(v, 0.0);
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_oc_emit(const LatticeView* __restrict__ views, const int* __restrict__ word_off, int n,
                          int total, const int* __restrict__ off_f, const int* __restrict__ off_s,
                          unsigned long long* __restrict__ key_f, int* __restrict__ idx_f,
                          unsigned long long* __restrict__ key_s, int* __restrict__ idx_s,
                          int* __restrict__ info) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int l, y, w;
  word_of(views, word_off, n, i, l, y, w);
  const LatticeView* L = views + l;
  const int nx = L->nx, pitch = L->pitch;
  const double rho0 = L->rho0d, mu = L->mu;
  const WordMasks m = word_masks(L->mask, nx, L->ny, L->wpr, y, w, L->guard);
  int of = off_f[i], os = off_s[i];
  bool bad = false;
  // a field value, its index checked in the bounds-checked build (0 when outside)
  const long long plane = L->plane;
  (void)plane;
  auto fld = [&](const float* a, long long c) { return LBM_OK_IDX(c, plane) ? (double)a[c] : 0.0; };
  uint32_t fc = m.fluid_cand;
  while (fc) {
    const int b = __ffs(fc) - 1;
    fc &= fc - 1;
    const int x = w * 32 + b;
    const long long c = (long long)y * pitch + x;
    const double ux = fld(L->ux, c), uy = fld(L->uy, c);
    const double rho = __dadd_rn(rho0, fld(L->drho, c));
    const double s = __dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy));
    const double q = __dmul_rn(__dmul_rn(0.5, rho), s);
    bad |= isnan(q);
    key_f[of] = order_key(q);
    idx_f[of] = y * nx + x;
    ++of;
  }
  uint32_t sc = m.solid_cand;
  while (sc) {
    const int b = __ffs(sc) - 1;
    sc &= sc - 1;
    const int x = w * 32 + b;
    const long long c = (long long)y * pitch + x;
    // fluid 4-neighbours in the order E, N, W, S
    const bool fe = !((m.e >> b) & 1u), fn = !((m.n >> b) & 1u), fw = !((m.w >> b) & 1u),
               fs = !((m.s >> b) & 1u);
    double sigma = 0.0;
    if (fe) sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, fabs(fld(L->uy, c + 1))), 0.5));
    if (fn) sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, fabs(fld(L->ux, c + pitch))), 0.5));
    if (fw) sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, fabs(fld(L->uy, c - 1))), 0.5));
    if (fs) sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, fabs(fld(L->ux, c - pitch))), 0.5));
    bad |= isnan(sigma);
    key_s[os] = ~order_key(sigma);  // ascending key = descending sigma
    idx_s[os] = y * nx + x;
    ++os;
  }
  if (bad) atomicOr(info + 8 * l + 3, 1);
}

constexpr int kSelThreads = 1024;

// Grid (2, lattices): block (0, l) selects among lattice l's fluid candidates,
// block (1, l) among its solid candidates: the n smallest (key, idx) pairs,
// written in candidate (= ascending idx) order to the lattice's pick range.
__global__ void __launch_bounds__(kSelThreads)
    k_oc_select(const LatticeView* __restrict__ views, const int* __restrict__ word_off,
                const unsigned long long* __restrict__ key_f, const int* __restrict__ idx_f,
                const unsigned long long* __restrict__ key_s, const int* __restrict__ idx_s,
                const int* __restrict__ off_f, const int* __restrict__ off_s,
                const int* __restrict__ n_swap, int* __restrict__ sel_f, int* __restrict__ sel_s,
                int* __restrict__ info) {
  __shared__ int hist[256];
  __shared__ unsigned long long s_key;
  __shared__ unsigned int s_idx;
  __shared__ int s_rem;
  __shared__ int scan[kSelThreads];
  const int tid = threadIdx.x;
  const int l = blockIdx.y;
  const LatticeView* L = views + l;
  const int w0 = word_off[l], w1 = word_off[l + 1];
  const int f0 = off_f[w0], nf = off_f[w1] - f0;
  const int s0 = off_s[w0], ns = off_s[w1] - s0;
  const bool fluid_class = blockIdx.x == 0;
  const unsigned long long* key = fluid_class ? key_f + f0 : key_s + s0;
  const int* idx = fluid_class ? idx_f + f0 : idx_s + s0;
  int* sel = (fluid_class ? sel_f : sel_s) + L->sel_off;
  const int ncand = fluid_class ? nf : ns;
  int n = n_swap[l];
  const int cap = sel_capacity(L->nx, L->ny);
  n = n < cap ? n : cap;
  n = n < nf ? n : nf;
  n = n < ns ? n : ns;
  if (n < 0) n = 0;
  if (fluid_class && tid == 0) {
    info[8 * l + 0] = n;
    info[8 * l + 1] = nf;
    info[8 * l + 2] = ns;
  }
  if (n == 0) return;
  if (tid == 0) {
    s_key = 0;
    s_idx = 0;
    s_rem = n;  // rank (1-based) of the threshold among matching candidates
  }
  __syncthreads();
  // 12 digits of 8 bits: 8 of the score key, then 4 of the index
  for (int d = 0; d < 12; ++d) {
    for (int k = tid; k < 256; k += kSelThreads) hist[k] = 0;
    __syncthreads();
    const unsigned long long pk = s_key;
    const unsigned int pi = s_idx;
    for (int k = tid; k < ncand; k += kSelThreads) {
      const unsigned long long kk = key[k];
      const unsigned int ii = (unsigned int)idx[k];
      int digit;
      bool match;
      if (d < 8) {
        match = d == 0 || (kk >> (64 - 8 * d)) == (pk >> (64 - 8 * d));
        digit = (int)((kk >> (56 - 8 * d)) & 0xffu);
      } else {
        const int dd = d - 8;
        match = kk == pk && (dd == 0 || (ii >> (32 - 8 * dd)) == (pi >> (32 - 8 * dd)));
        digit = (int)((ii >> (24 - 8 * dd)) & 0xffu);
      }
      if (match) atomicAdd(&hist[digit], 1);
    }
    __syncthreads();
    if (tid == 0) {
      int rem = s_rem, b = 0;
      while (b < 255 && hist[b] < rem) {
        rem -= hist[b];
        ++b;
      }
      s_rem = rem;
      if (d < 8)
        s_key = pk | ((unsigned long long)b << (56 - 8 * d));
      else
        s_idx = pi | ((unsigned int)b << (24 - 8 * (d - 8)));
    }
    __syncthreads();
  }
  const unsigned long long tk = s_key;
  const unsigned int ti = s_idx;
  // ordered compaction of all (key, idx) <= (tk, ti): exactly n of them
  const int per = (ncand + kSelThreads - 1) / kSelThreads;
  const int begin = min(ncand, tid * per), end = min(ncand, begin + per);
  int cnt = 0;
  for (int k = begin; k < end; ++k) {
    const unsigned long long kk = key[k];
    cnt += (kk < tk || (kk == tk && (unsigned int)idx[k] <= ti)) ? 1 : 0;
  }
  scan[tid] = cnt;
  __syncthreads();
  for (int off = 1; off < kSelThreads; off <<= 1) {
    const int v = tid >= off ? scan[tid - off] : 0;
    __syncthreads();
    scan[tid] += v;
    __syncthreads();
  }
  int pos = scan[tid] - cnt;
  for (int k = begin; k < end; ++k) {
    const unsigned long long kk = key[k];
    if (kk < tk || (kk == tk && (unsigned int)idx[k] <= ti)) sel[pos++] = idx[k];
  }
}

// grid (blocks, lattices): exchange lattice l's picks
template <class T>
__global__ void k_oc_apply(const LatticeView* __restrict__ views, const int* __restrict__ sel_f_all,
                           const int* __restrict__ sel_s_all, const int* __restrict__ info) {
  const int l = blockIdx.y;
  const LatticeView* L = views + l;
  const int n = info[8 * l];
  const int nx = L->nx, ms = mask_stride(L->wpr), pitch = L->pitch;
  const long long pl = L->plane;
  uint32_t* mask = const_cast<uint32_t*>(L->mask);
  T* F = static_cast<T*>(L->f);
  const int* sel_f = sel_f_all + L->sel_off;
  const int* sel_s = sel_s_all + L->sel_off;
  const long long cells = (long long)nx * L->ny;
  (void)cells;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    // the picks are cell indices of the lattice (checked in the bounds-checked build)
    if (!LBM_OK_IDX(sel_f[k], cells) || !LBM_OK_IDX(sel_s[k], cells)) continue;
    {  // fluid -> solid
      const int id = sel_f[k];
      const int y = id / nx, x = id - y * nx;
      atomicOr(mask + (long long)y * ms + (x >> 5), 1u << (x & 31));
      const long long c = (long long)y * pitch + x;
      L->drho[c] = 0.0f;
      L->ux[c] = 0.0f;
      L->uy[c] = 0.0f;
    }
    {  // solid -> fluid, at the rest equilibrium of rho0: g_i = 0
      const int id = sel_s[k];
      const int y = id / nx, x = id - y * nx;
      atomicAnd(mask + (long long)y * ms + (x >> 5), ~(1u << (x & 31)));
      const long long c = (long long)y * pitch + x;
#pragma unroll
      for (int i = 0; i < 9; ++i)
        if (LBM_OK_IDX(i * pl + c, L->f_elems)) F[i * pl + c] = T(0.0f);
      L->drho[c] = 0.0f;
      L->ux[c] = 0.0f;
      L->uy[c] = 0.0f;
    }
  }
}

inline int blocks_for(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_oc_select(const LatticeView* views, const int* word_off, int n_lattices, int total,
                             const int* n_swap, const OcScratch& s, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(s.info, 0, 8 * sizeof(int) * n_lattices, stream);
  if (e != cudaSuccess) return e;
  k_oc_count<<<blocks_for(total, 256), 256, 0, stream>>>(views, word_off, n_lattices, total, s.cnt_f,
                                                         s.cnt_s);
  count_launches(1);
  if ((e = launch_scan(s.cnt_f, s.off_f, total, s.scan_tmp, stream)) != cudaSuccess) return e;
  if ((e = launch_scan(s.cnt_s, s.off_s, total, s.scan_tmp, stream)) != cudaSuccess) return e;
  k_oc_emit<<<blocks_for(total, 256), 256, 0, stream>>>(views, word_off, n_lattices, total, s.off_f,
                                                        s.off_s, s.key_f, s.idx_f, s.key_s, s.idx_s,
                                                        s.info);
  k_oc_select<<<dim3(2, n_lattices), kSelThreads, 0, stream>>>(views, word_off, s.key_f, s.idx_f, s.key_s,
                                                               s.idx_s, s.off_f, s.off_s, n_swap, s.sel_f,
                                                               s.sel_s, s.info);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_oc_select_only(const LatticeView* views, const int* word_off, int n_lattices, const int* n_swap,
                                  const OcScratch& s, cudaStream_t stream) {
  k_oc_select<<<dim3(2, n_lattices), kSelThreads, 0, stream>>>(views, word_off, s.key_f, s.idx_f, s.key_s, s.idx_s,
                                                               s.off_f, s.off_s, n_swap, s.sel_f, s.sel_s, s.info);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_oc_apply(int precision, const LatticeView* views, int n_lattices, const OcScratch& s,
                            cudaStream_t stream) {
  const dim3 grid(4, n_lattices);
  switch (precision) {
    case LBM_F32:
      k_oc_apply<float><<<grid, 128, 0, stream>>>(views, s.sel_f, s.sel_s, s.info);
      break;
    case LBM_BF16_SHIFTED:
      k_oc_apply<__nv_bfloat16><<<grid, 128, 0, stream>>>(views, s.sel_f, s.sel_s, s.info);
      break;
    case LBM_F16_SHIFTED:
      k_oc_apply<__half><<<grid, 128, 0, stream>>>(views, s.sel_f, s.sel_s, s.info);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace lbm
