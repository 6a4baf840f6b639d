// FP64 reductions of a solved field: pressure drop, inlet and outlet flow
// rates (Sec. 2.3 step 5), the uniformity measures of Eq. 9-11 and the
// convergence residual -- for every lattice of a set in one launch.
//
// All sums are accumulated in double from the FP32 moments of the last step
// and are deterministic: every thread owns a fixed set of cells, warps sum
// by a fixed shuffle butterfly, block sums take the warp sums in ascending
// warp order, and partial sums are combined in ascending block order.  No
// floating-point atomics.
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kRedThreads = 256;

// Sum over a warp by shuffles: a fixed butterfly, so every lane gets the
// same bits for the same inputs in the same lanes.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of kRedThreads doubles: each warp by shuffles, then the warp sums
// by the first warp in ascending warp order.  Every thread gets the result.
__device__ double block_sum(double v, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  double r = lane < kRedThreads / 32 ? sm[lane] : 0.0;
  r = warp_sum(r);
  __syncthreads();  // sm is reused by the next call
  return r;
}

// Residual partials, grid (kResidualBlocks, lattices): block b of lattice l
// covers rows [b*ny/B, (b+1)*ny/B).  partials[l][2b] = sum |u - u_prev|_1,
// partials[l][2b+1] = sum |u|_1 (solid cells hold zeros in both fields).
__global__ void __launch_bounds__(kRedThreads)
    k_residual_partials(const LatticeView* __restrict__ views, double* __restrict__ partials) {
  __shared__ double sm[kRedThreads / 32];
  const LatticeView* L = views + blockIdx.y;
  const int nx = L->nx, ny = L->ny, pitch = L->pitch;
  const int b = blockIdx.x;
  const int y0 = (int)((long long)b * ny / kResidualBlocks);
  const int y1 = (int)((long long)(b + 1) * ny / kResidualBlocks);
  const long long n = (long long)(y1 - y0) * nx;
  double du = 0.0, u = 0.0;
  for (long long k = threadIdx.x; k < n; k += kRedThreads) {
    const int y = y0 + (int)(k / nx), x = (int)(k % nx);
    const long long c = (long long)y * pitch + x;
    if (!LBM_OK_IDX(c, L->plane)) continue;
    const double ux = L->ux[c], uy = L->uy[c];
    du += fabs(ux - (double)L->ux_prev[c]) + fabs(uy - (double)L->uy_prev[c]);
    u += fabs(ux) + fabs(uy);
  }
  du = block_sum(du, sm);
  u = block_sum(u, sm);
  if (threadIdx.x == 0) {
    double* p = partials + (size_t)blockIdx.y * 2 * kResidualBlocks;
    p[2 * b] = du;
    p[2 * b + 1] = u;
  }
}

// One block per lattice: port sums and the final combination.
__global__ void __launch_bounds__(kRedThreads)
    k_finalize(const LatticeView* __restrict__ views, const double* __restrict__ partials_all,
               int with_residual, double* __restrict__ result_all) {
  __shared__ double sm[kRedThreads / 32];
  const LatticeView* L = views + blockIdx.x;
  double* result = result_all + (size_t)blockIdx.x * kResultDoubles;
  const double* partials = partials_all + (size_t)blockIdx.x * 2 * kResidualBlocks;
  const int nx = L->nx, ny = L->ny, pitch = L->pitch, wpr = L->wpr;
  const int n_outlets = L->n_outlets;
  const double rho0 = L->rho0d;
  const int wl = (nx - 1) >> 5, bl = (nx - 1) & 31;
  double s_in = 0.0, s_out = 0.0, m_in = 0.0, n_in = 0.0, n_out = 0.0;
  for (int y = threadIdx.x; y < ny; y += kRedThreads) {
    const uint32_t* mr = L->mask + (long long)y * mask_stride(wpr);
    const long long c0 = (long long)y * pitch;
    if (!LBM_OK_IDX(c0 + nx - 1, L->plane)) continue;
    if (!(mr[0] & 1u)) {
      const double d = L->drho[c0];
      s_in += d;
      m_in += (rho0 + d) * (double)L->ux[c0];
      n_in += 1.0;
    }
    if (!((mr[wl] >> bl) & 1u)) {
      s_out += L->drho[c0 + nx - 1];
      n_out += 1.0;
    }
  }
  s_in = block_sum(s_in, sm);
  s_out = block_sum(s_out, sm);
  m_in = block_sum(m_in, sm);
  n_in = block_sum(n_in, sm);
  n_out = block_sum(n_out, sm);
  // each outlet run summed by one warp: lane l takes rows ya + l, ya + l + 32,
  // ... in ascending order, then the lanes' sums by shuffles
  {
    const int lane = threadIdx.x & 31;
    for (int j = threadIdx.x >> 5; j < n_outlets; j += kRedThreads / 32) {
      double m = 0.0;
      const int ya = L->out_start[j], yb = ya + L->out_len[j];
      for (int y = ya + lane; y < yb; y += 32) {
        const long long c = (long long)y * pitch + nx - 1;
        if (!LBM_OK_IDX(c, L->plane)) continue;
        m += (rho0 + (double)L->drho[c]) * (double)L->ux[c];
      }
      m = warp_sum(m);
      if (lane == 0) result[10 + j] = m;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Eq. 9-11: theta = m_max / m_min, D_g = sqrt(sum (m_j / m_ave - 1)^2 / (N - 1))
    const double* m = result + 10;
    double mx = m[0], mn = m[0], sum = 0.0;
    for (int j = 0; j < n_outlets; ++j) {
      mx = m[j] > mx ? m[j] : mx;
      mn = m[j] < mn ? m[j] : mn;
      sum += m[j];
    }
    const double ave = sum / n_outlets;
    double acc = 0.0;
    for (int j = 0; j < n_outlets; ++j) {
      const double d = m[j] / ave - 1.0;
      acc += d * d;
    }
    result[8] = mx / mn;
    result[9] = n_outlets > 1 ? sqrt(acc / (n_outlets - 1)) : 0.0;
    // p = rho c_s^2 = rho / 3 (Eq. 4); the rho0/3 parts cancel in the difference
    const double dp = (s_in / n_in - s_out / n_out) / 3.0;
    double res = -1.0, sdu = 0.0, su = 0.0;
    if (with_residual) {
      for (int b = 0; b < kResidualBlocks; ++b) {
        sdu += partials[2 * b];
        su += partials[2 * b + 1];
      }
      res = sdu / su;
    }
    result[0] = dp;
    result[1] = m_in;
    result[2] = res;
    result[3] = n_in;
    result[4] = n_out;
    result[5] = sdu;
    result[6] = su;
    const bool bad = !isfinite(dp) || !isfinite(m_in) || (with_residual && !isfinite(res));
    result[7] = bad ? 1.0 : 0.0;
  }
}

}  // namespace

cudaError_t launch_residual_partials(const LatticeView* views, int n_lattices, double* partials,
                                     cudaStream_t stream) {
  k_residual_partials<<<dim3(kResidualBlocks, n_lattices), kRedThreads, 0, stream>>>(views, partials);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const LatticeView* views, int n_lattices, const double* partials,
                            int with_residual, double* result, cudaStream_t stream) {
  k_finalize<<<n_lattices, kRedThreads, 0, stream>>>(views, partials, with_residual, result);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace lbm
