// Per-cell D2Q9 arithmetic shared by the step kernels (step.cu, resident.cu):
// storage conversion of the shifted populations, the moments of Eq. 2, the
// BGK relaxation of Eq. 1 towards the second-order equilibrium of Sec. 2.1
// (and the other collision models), and the port rules of Sec. 3.3.  Every
// step kernel calls these same functions, so all of them compute the same
// bits per cell.
#pragma once

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
  // the element held in a 4-byte word (hi: the upper of two 16-bit halves)
  static __device__ __forceinline__ float from_word(uint32_t w, int) { return __uint_as_float(w); }
};
template <>
struct Pop<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ float ldcg(const __nv_bfloat16* p) { return __bfloat162float(__ldcg(p)); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float from_word(uint32_t w, int hi) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)(w >> (hi ? 16 : 0))));
  }
};
template <>
struct Pop<__half> {
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ float ldcg(const __half* p) { return __half2float(__ldcg(p)); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ float from_word(uint32_t w, int hi) {
    return __half2float(__ushort_as_half((unsigned short)(w >> (hi ? 16 : 0))));
  }
};

// Two adjacent elements of a plane, the first at an even x (rows start on
// 128-byte boundaries, so the pair is aligned to its own size): one memory
// instruction for two cells.  The conversions are those of Pop, element by
// element (a 16-bit element widens exactly; both halves round to nearest
// even on the way back).
template <class T>
struct Pop2;
template <>
struct Pop2<float> {
  static __device__ __forceinline__ void ld(const float* p, float& lo, float& hi) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    lo = v.x;
    hi = v.y;
  }
  static __device__ __forceinline__ void st(float* p, float lo, float hi) {
    *reinterpret_cast<float2*>(p) = make_float2(lo, hi);
  }
};
template <>
struct Pop2<__nv_bfloat16> {
  static __device__ __forceinline__ void ld(const __nv_bfloat16* p, float& lo, float& hi) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
    lo = __uint_as_float(w << 16);  // a bfloat16 is the upper half of its float
    hi = __uint_as_float(w & 0xffff0000u);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float lo, float hi) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(lo, hi);
  }
};
template <>
struct Pop2<__half> {
  static __device__ __forceinline__ void ld(const __half* p, float& lo, float& hi) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    lo = v.x;
    hi = v.y;
  }
  static __device__ __forceinline__ void st(__half* p, float lo, float hi) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(lo, hi);
  }
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

// BGK conserves mass and momentum; rounded FP32 relaxation does not quite,
// and the drift dominates the FP32 error over thousands of steps.  Close
// both exactly: g1 and g2 carry the momentum balance, the rest population
// the mass balance (an identity in exact arithmetic; so for every collision
// model here, which all conserve both).
__device__ __forceinline__ void close_moments(float (&g)[9], float drho, float jx, float jy) {
  g[1] = jx + g[3] - ((g[5] - g[7]) + (g[8] - g[6]));
  g[2] = jy + g[4] - ((g[5] - g[7]) + (g[6] - g[8]));
  g[0] = drho - (((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
}

// Moments (Eq. 2) and BGK relaxation (Eq. 1) of one cell, in place.
__device__ __forceinline__ void bgk(float (&g)[9], float rho0, float omega, float& drho, float& ux,
                                    float& uy) {
  drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const float rho = rho0 + drho;
  const float jx = (g[1] - g[3]) + (g[5] - g[7]) + (g[8] - g[6]);
  const float jy = (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
  const float inv = __frcp_rn(rho);  // correctly rounded: the value of 1.0f / rho
  ux = jx * inv;
  uy = jy * inv;
  const float t0 = drho - 1.5f * rho * (ux * ux + uy * uy);
  relax_pair(g[1], g[3], ux, kW1, rho, t0, omega);
  relax_pair(g[2], g[4], uy, kW1, rho, t0, omega);
  relax_pair(g[5], g[7], ux + uy, kW5, rho, t0, omega);
  relax_pair(g[8], g[6], ux - uy, kW5, rho, t0, omega);
  close_moments(g, drho, jx, jy);
}

// The same update for two cells at once (a lane's pair of a paired task), in
// the packed FP32 instructions of sm_100-family parts (add/sub/mul/fma.rn
// .f32x2).  Each step is the rounding the compiler gives bgk()'s expressions:
// a product feeding a sum becomes one fused multiply-add (t0 + 3 rho cu,
// then + 4.5 rho cu^2; g + omega (e - g); drho - 1.5 rho (ux ux + uy uy)), so
// that the two forms give the same bits -- the paired kernel's GPU tests
// require it against the row-segment kernel at every storage type.
struct F2 {
  unsigned long long v;  // two FP32 values: the lower cell, the upper cell
};
__device__ __forceinline__ F2 f2(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_split(F2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ F2 f2_c(float c) { return f2(c, c); }

__device__ __forceinline__ void relax_pair2(F2& gi, F2& go, F2 cu, F2 w, F2 r3, F2 r3n, F2 r45, F2 t0, F2 omega) {
  const F2 b = f2_mul(r45, cu);
  const F2 ei = f2_mul(w, f2_fma(b, cu, f2_fma(r3, cu, t0)));
  const F2 eo = f2_mul(w, f2_fma(b, cu, f2_fma(r3n, cu, t0)));
  gi = f2_fma(omega, f2_sub(ei, gi), gi);
  go = f2_fma(omega, f2_sub(eo, go), go);
}

__device__ __forceinline__ void bgk2(float (&a)[9], float (&b)[9], float rho0_, float omega_, float& dra,
                                     float& uxa, float& uya, float& drb, float& uxb, float& uyb) {
  F2 g[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) g[i] = f2(a[i], b[i]);
  const F2 drho = f2_add(f2_add(f2_add(f2_add(g[0], g[1]), f2_add(g[2], g[3])),
                                f2_add(f2_add(g[4], g[5]), f2_add(g[6], g[7]))), g[8]);
  const F2 rho = f2_add(f2_c(rho0_), drho);
  const F2 jx = f2_add(f2_add(f2_sub(g[1], g[3]), f2_sub(g[5], g[7])), f2_sub(g[8], g[6]));
  const F2 jy = f2_add(f2_add(f2_sub(g[2], g[4]), f2_sub(g[5], g[7])), f2_sub(g[6], g[8]));
  float rl, rh;
  f2_split(rho, rl, rh);
  const F2 inv = f2(__frcp_rn(rl), __frcp_rn(rh));  // correctly rounded: the value of 1.0f / rho
  const F2 ux = f2_mul(jx, inv), uy = f2_mul(jy, inv);
  const F2 t0 = f2_fma(f2_mul(f2_c(-1.5f), rho), f2_fma(ux, ux, f2_mul(uy, uy)), drho);
  const F2 r3 = f2_mul(f2_c(3.0f), rho), r3n = f2_mul(f2_c(-3.0f), rho), r45 = f2_mul(f2_c(4.5f), rho);
  const F2 omega = f2_c(omega_);
  relax_pair2(g[1], g[3], ux, f2_c(kW1), r3, r3n, r45, t0, omega);
  relax_pair2(g[2], g[4], uy, f2_c(kW1), r3, r3n, r45, t0, omega);
  relax_pair2(g[5], g[7], f2_add(ux, uy), f2_c(kW5), r3, r3n, r45, t0, omega);
  relax_pair2(g[8], g[6], f2_sub(ux, uy), f2_c(kW5), r3, r3n, r45, t0, omega);
  g[1] = f2_sub(f2_add(jx, g[3]), f2_add(f2_sub(g[5], g[7]), f2_sub(g[8], g[6])));
  g[2] = f2_sub(f2_add(jy, g[4]), f2_add(f2_sub(g[5], g[7]), f2_sub(g[6], g[8])));
  g[0] = f2_sub(drho, f2_add(f2_add(f2_add(g[1], g[2]), f2_add(g[3], g[4])),
                             f2_add(f2_add(g[5], g[6]), f2_add(g[7], g[8]))));
#pragma unroll
  for (int i = 0; i < 9; ++i) f2_split(g[i], a[i], b[i]);
  f2_split(drho, dra, drb);
  f2_split(ux, uxa, uxb);
  f2_split(uy, uya, uyb);
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

// Collision beyond BGK, of one cell in place (moments as in bgk()):
//   regularised: g_i <- g^eq_i + (1 - omega) [w_i/(2 c_s^4) Q_i : Pi], the
//                non-equilibrium part projected on its second moment Pi before
//                relaxing (regularize() builds g^eq + that projection);
//   Smagorinsky: BGK with the local relaxation time
//                tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 |Pi| / rho)) / 2,
//                |Pi| = sqrt(Pi:Pi): the positive root of
//                tau_eff^2 - tau tau_eff = C^2 sqrt(2 Pi:Pi) / (2 rho c_s^4),
//                i.e. nu_t = C^2 |S| with the strain rate S = -Pi / (2 rho c_s^2 tau_eff).
__device__ __forceinline__ void collide_other(float (&g)[9], float rho0, float omega, int model, float c_smag,
                                           float& drho, float& ux, float& uy) {
  drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const float rho = rho0 + drho;
  const float jx = (g[1] - g[3]) + (g[5] - g[7]) + (g[8] - g[6]);
  const float jy = (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
  const float inv = 1.0f / rho;
  ux = jx * inv;
  uy = jy * inv;
  float e[9];
  shifted_equilibria(e, rho0, drho, ux, uy);
  if (model == LBM_COLLIDE_REGULARIZED) {
    regularize(g, e);
    const float keep = 1.0f - omega;
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = e[i] + keep * (g[i] - e[i]);
  } else {
    float n[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) n[i] = g[i] - e[i];
    const float dsum = (n[5] + n[6]) + (n[7] + n[8]);
    const float pxx = (n[1] + n[3]) + dsum;
    const float pyy = (n[2] + n[4]) + dsum;
    const float pxy = (n[5] + n[7]) - (n[6] + n[8]);
    const float pp = pxx * pxx + pyy * pyy + 2.0f * pxy * pxy;
    const float tau = 1.0f / omega;
    const float tau_eff = 0.5f * (tau + sqrtf(tau * tau + 18.0f * 1.41421356f * c_smag * c_smag * sqrtf(pp) / rho));
    const float w = 1.0f / tau_eff;
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] += w * (e[i] - g[i]);
  }
  close_moments(g, drho, jx, jy);
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

}  // namespace
}  // namespace lbm
