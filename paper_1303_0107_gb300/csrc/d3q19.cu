// D3Q19 form of the hot path: fused stream + collide on a single lattice
// (AA access pattern), the FP64 port reductions, and the exchange of Sec.
// 2.2-2.3 on the 6-neighbourhood.
//
// Storage.  Populations shifted, g_i = f_i - w_i rho0, in 19 planes
// F[i][z][y][x] (row pitch nxp = 32 nsx), FP32, BF16 or FP16; FP32
// arithmetic.  Between steps F[i][cell] is the post-collision g_i of the
// cell.  Steps come in pairs, as in 2D:
//   phase A  cell x takes g_i from F[i][x - c_i] (or, where x - c_i is
//            solid, the reversed F[opp(i)][x]), relaxes, and writes g_i to
//            F[opp(i)][x + c_i] -- the slot it read for direction opp(i) --
//            or, where x + c_i is solid, to F[i][x];
//   phase B  cell x finds its incoming g_i in F[opp(i)][x], relaxes, writes
//            F[i][x].
// Each slot is read and then written by one thread per phase: one lattice,
// no barrier, solid cells never read.
//
// Thread mapping.  A warp takes one task of a device-resident list.  A
// segment task is a row segment (32 cells of one mask word, row (y, z))
// holding at least pack_below fluid cells; lane l is cell 32 s + l, and each
// population access of the warp is one contiguous 32-element row piece,
// shifted by at most one element.  A packed task holds 32 fluid cells of
// the sparser segments (at branch walls), one a lane, in index order.  The
// neighbour flags of segments that are not open, and the flags of packed
// cells, are built with the list (lanes 0..26 of a warp load the 27 mask
// words around a segment and share them by shuffles).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm3d_internal.h"

namespace lbm {
namespace {

constexpr int kQ = 19;

// D3Q19 velocity set (the order of include/lbm3d.h); opposites are (1,2),
// (3,4), ..., (17,18).  Called with loop indices of unrolled loops, these
// fold to constants.
__host__ __device__ constexpr int cx3(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy3(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz3(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp3(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// the direction with c_y negated (reflection in a plane normal to y)
__host__ __device__ constexpr int mir3(int i) {
  return (i == 3 || i == 4) ? 7 - i : (i == 7) ? 9 : (i == 9) ? 7 : (i == 8) ? 10 : (i == 10) ? 8
         : (i == 15) ? 18 : (i == 18) ? 15 : (i == 16) ? 17 : (i == 17) ? 16 : i;
}
// the direction with c_z negated (reflection in a plane normal to z)
__host__ __device__ constexpr int mirz3(int i) {
  return (i == 5 || i == 6) ? 11 - i : (i == 11) ? 13 : (i == 13) ? 11 : (i == 12) ? 14 : (i == 14) ? 12
         : (i == 15) ? 17 : (i == 17) ? 15 : (i == 16) ? 18 : (i == 18) ? 16 : i;
}
__host__ __device__ constexpr float w3(int i) { return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f); }
// c * v for c in {-1, 0, 1} without a multiply (0 * v is not 0 for v = inf/NaN)
__device__ __forceinline__ float cmul(int c, float v) { return c == 0 ? 0.0f : (c > 0 ? v : -v); }

template <class T>
struct P3;
template <>
struct P3<float> {
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct P3<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct P3<__half> {
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};

// Shifted second-order equilibrium g^eq_i = f^eq_i(rho0 + drho, u) - w_i rho0
//   = w_i (t0 + 3 rho c.u + 4.5 rho (c.u)^2),  t0 = drho - 1.5 rho u.u.
__device__ __forceinline__ float geq3(int i, float rho, float t0, float ux, float uy, float uz) {
  const float cu = cmul(cx3(i), ux) + cmul(cy3(i), uy) + cmul(cz3(i), uz);
  return w3(i) * (t0 + 3.0f * rho * cu + 4.5f * rho * cu * cu);
}

// Relax a pair of opposite directions towards their equilibria (c_o = -c_i).
__device__ __forceinline__ void relax_pair3(float& gi, float& go, float cu, float w, float rho, float t0,
                                            float omega) {
  const float a = 3.0f * rho * cu;
  const float b = 4.5f * rho * cu * cu;
  gi += omega * (w * (t0 + a + b) - gi);
  go += omega * (w * (t0 - a + b) - go);
}

// Rounded FP32 relaxation drifts in mass and momentum over thousands of
// steps; BGK conserves both exactly, so restore them: g1, g3, g5 carry the
// three momentum balances, the rest population the mass balance.
__device__ __forceinline__ void close_moments3(float (&g)[kQ], float drho, float jx, float jy, float jz) {
  g[1] = jx + g[2] - (((g[7] - g[8]) + (g[9] - g[10])) + ((g[11] - g[12]) + (g[13] - g[14])));
  g[3] = jy + g[4] - (((g[7] - g[8]) + (g[10] - g[9])) + ((g[15] - g[16]) + (g[17] - g[18])));
  g[5] = jz + g[6] - (((g[11] - g[12]) + (g[14] - g[13])) + ((g[15] - g[16]) + (g[18] - g[17])));
  float s = 0.0f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) s += g[i];
  g[0] = drho - s;
}

__device__ __forceinline__ void moments3(const float (&g)[kQ], float& drho, float& jx, float& jy, float& jz) {
  float s = g[0];
#pragma unroll
  for (int i = 1; i < kQ; ++i) s += g[i];
  drho = s;
  jx = ((g[1] - g[2]) + (g[7] - g[8])) + ((g[9] - g[10]) + (g[11] - g[12])) + (g[13] - g[14]);
  jy = ((g[3] - g[4]) + (g[7] - g[8])) + ((g[10] - g[9]) + (g[15] - g[16])) + (g[17] - g[18]);
  jz = ((g[5] - g[6]) + (g[11] - g[12])) + ((g[14] - g[13]) + (g[15] - g[16])) + (g[18] - g[17]);
}

// Moments and BGK relaxation of one cell, in place.
__device__ __forceinline__ void bgk3(float (&g)[kQ], float rho0, float omega, float& drho, float& ux, float& uy,
                                     float& uz) {
  float jx, jy, jz;
  moments3(g, drho, jx, jy, jz);
  const float rho = rho0 + drho;
  const float inv = 1.0f / rho;
  ux = jx * inv;
  uy = jy * inv;
  uz = jz * inv;
  const float t0 = drho - 1.5f * rho * (ux * ux + uy * uy + uz * uz);
  g[0] += omega * (w3(0) * t0 - g[0]);
  constexpr float wf = 1.0f / 18.0f, we = 1.0f / 36.0f;
  relax_pair3(g[1], g[2], ux, wf, rho, t0, omega);
  relax_pair3(g[3], g[4], uy, wf, rho, t0, omega);
  relax_pair3(g[5], g[6], uz, wf, rho, t0, omega);
  relax_pair3(g[7], g[8], ux + uy, we, rho, t0, omega);
  relax_pair3(g[9], g[10], ux - uy, we, rho, t0, omega);
  relax_pair3(g[11], g[12], ux + uz, we, rho, t0, omega);
  relax_pair3(g[13], g[14], ux - uz, we, rho, t0, omega);
  relax_pair3(g[15], g[16], uy + uz, we, rho, t0, omega);
  relax_pair3(g[17], g[18], uy - uz, we, rho, t0, omega);
  close_moments3(g, drho, jx, jy, jz);
}

// The collision models beyond BGK (regularised, Smagorinsky), in place, in
// the shifted form: with e_i the shifted equilibria and Pi = sum c c (g - e),
//   regularised   g_i = e_i + (1 - omega) 4.5 w_i Q_i : Pi  (Q_i = c_i c_i - I/3);
//   Smagorinsky   g_i += omega_eff (e_i - g_i), omega_eff = 1 / tau_eff,
//                 tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 sqrt(Pi:Pi) / rho)) / 2,
// the positive root of the closure nu_t = C^2 |S| with S from Pi (c_s^4 = 1/9).
// Mass and momentum are then closed exactly, as for BGK.
__device__ __forceinline__ void collide_other3(float (&g)[kQ], float rho0, float omega, float tau, int model,
                                               float c_smag, float& drho, float& ux, float& uy, float& uz) {
  float jx, jy, jz;
  moments3(g, drho, jx, jy, jz);
  const float rho = rho0 + drho;
  const float inv = 1.0f / rho;
  ux = jx * inv;
  uy = jy * inv;
  uz = jz * inv;
  const float t0 = drho - 1.5f * rho * (ux * ux + uy * uy + uz * uz);
  float e[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) e[i] = geq3(i, rho, t0, ux, uy, uz);
  float pxx = 0.0f, pyy = 0.0f, pzz = 0.0f, pxy = 0.0f, pxz = 0.0f, pyz = 0.0f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float nq = g[i] - e[i];
    if (cx3(i) != 0) pxx += nq;
    if (cy3(i) != 0) pyy += nq;
    if (cz3(i) != 0) pzz += nq;
    pxy += cmul(cx3(i) * cy3(i), nq);
    pxz += cmul(cx3(i) * cz3(i), nq);
    pyz += cmul(cy3(i) * cz3(i), nq);
  }
  if (model == LBM_COLLIDE_REGULARIZED) {
    const float keep = 1.0f - omega;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float qxx = (float)(cx3(i) * cx3(i)) - 1.0f / 3.0f;
      const float qyy = (float)(cy3(i) * cy3(i)) - 1.0f / 3.0f;
      const float qzz = (float)(cz3(i) * cz3(i)) - 1.0f / 3.0f;
      const float q = qxx * pxx + qyy * pyy + qzz * pzz +
                      2.0f * (cmul(cx3(i) * cy3(i), pxy) + cmul(cx3(i) * cz3(i), pxz) + cmul(cy3(i) * cz3(i), pyz));
      g[i] = e[i] + keep * (4.5f * w3(i) * q);
    }
  } else {
    const float pp = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
    const float tau_eff = 0.5f * (tau + sqrtf(tau * tau + 18.0f * 1.41421356f * c_smag * c_smag * sqrtf(pp) / rho));
    const float om = 1.0f / tau_eff;
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] += om * (e[i] - g[i]);
  }
  close_moments3(g, drho, jx, jy, jz);
}

// Port cell (x = 0 inlet, x = nx-1 outlet).  Known sums: G0 over c_x = 0,
// Gk over the directions arriving from inside (c_x < 0 at the inlet, > 0 at
// the outlet).  With sum_{c_x=0} w = 2/3 and sum_{c_x<0} w = 1/6:
//   inlet   u = u_in,  rho - rho0 = (G0 + 2 Gk + rho0 u) / (1 - u);
//   outlet  rho = rho0, u = (G0 + 2 Gk) / rho0;
// unknown populations g_i = g^eq_i + (g_opp(i) - g^eq_opp(i)); then every
// population is regularised, g_i = g^eq_i + 4.5 w_i Q_i : Pi with
// Pi = sum c c (g - g^eq), Q_i = c_i c_i - I/3 (w_i / (2 c_s^4) = 4.5 w_i).
__device__ __forceinline__ void port3(float (&g)[kQ], bool inlet, float u_in, float rho0) {
  float G0 = g[0] + ((g[3] + g[4]) + (g[5] + g[6])) + ((g[15] + g[16]) + (g[17] + g[18]));
  float dr, u;
  if (inlet) {
    const float Gk = (g[2] + g[8]) + (g[10] + g[12]) + g[14];
    u = u_in;
    dr = (G0 + 2.0f * Gk + rho0 * u) / (1.0f - u);
  } else {
    const float Gk = (g[1] + g[7]) + (g[9] + g[11]) + g[13];
    u = (G0 + 2.0f * Gk) / rho0;
    dr = 0.0f;
  }
  const float rho = rho0 + dr;
  const float t0 = dr - 1.5f * rho * u * u;
  float e[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) e[i] = geq3(i, rho, t0, u, 0.0f, 0.0f);
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const bool unknown = inlet ? cx3(i) > 0 : cx3(i) < 0;
    if (unknown) g[i] = e[i] + (g[opp3(i)] - e[opp3(i)]);
  }
  float pxx = 0.0f, pyy = 0.0f, pzz = 0.0f, pxy = 0.0f, pxz = 0.0f, pyz = 0.0f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float nq = g[i] - e[i];
    if (cx3(i) != 0) pxx += nq;
    if (cy3(i) != 0) pyy += nq;
    if (cz3(i) != 0) pzz += nq;
    pxy += cmul(cx3(i) * cy3(i), nq);
    pxz += cmul(cx3(i) * cz3(i), nq);
    pyz += cmul(cy3(i) * cz3(i), nq);
  }
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float qxx = (float)(cx3(i) * cx3(i)) - 1.0f / 3.0f;
    const float qyy = (float)(cy3(i) * cy3(i)) - 1.0f / 3.0f;
    const float qzz = (float)(cz3(i) * cz3(i)) - 1.0f / 3.0f;
    const float q = qxx * pxx + qyy * pyy + qzz * pzz +
                    2.0f * (cmul(cx3(i) * cy3(i), pxy) + cmul(cx3(i) * cz3(i), pxz) + cmul(cy3(i) * cz3(i), pyz));
    g[i] = e[i] + 4.5f * w3(i) * q;
  }
}

constexpr unsigned kFull = 0xffffffffu;

// keep a value opaque to the optimiser at this point (no hoisting or reuse)
__device__ __forceinline__ void opaque(int& a) { asm volatile("" : "+r"(a)); }
__device__ __forceinline__ void opaque(long long& a) { asm volatile("" : "+l"(a)); }

// The populations of one fluid cell: load (pull or local), port rule,
// collision, store.  c: the cell's element index within a plane,
// (z ny + y) nxp + x.  NB0: no neighbour of this cell is solid (no
// bounce-back selects at all, no port).  nb: bit i set when x + c_i is solid.
// on_py / on_pz: the cell lies on the layer next to a symmetry plane below
// y = 0 / z = 0 (mirror build, phase A).  port: 0 none, 1 inlet (x = 0), 2
// outlet (x = nx - 1); urow() gives z ny + y, called only for a port cell.
// IX: element index type -- int when all 19 planes have fewer than 2^31
// elements (one IMAD per address), else long long.  FEAT: kernel build, bit
// kFeat3Models (collision models beyond BGK), bit kFeat3Mirror (symmetry
// planes)
constexpr int kFeat3Models = 1, kFeat3Mirror = 2;

template <class T, int PHASE, int MOM, bool NB0, class IX, int FEAT, class URow>
__device__ __forceinline__ void cell_core3(const View3& v, IX c, uint32_t nb, bool on_py, bool on_pz, int port,
                                           URow urow) {
  IX sy = (IX)v.nxp, sz = (IX)v.ny * (IX)v.nxp;
  IX pl = (IX)v.plane;
  // opaque per cell: keeps the compiler from hoisting 18 plane and neighbour
  // offsets out of the warp's loop into registers
  opaque(pl);
  opaque(sy);
  opaque(sz);
  T* F = static_cast<T*>(v.f);
  // every population access is checked against the 19 planes in the
  // bounds-checked build (a violation is printed and skipped)
  const long long fe = (long long)kQ * v.plane;
  (void)fe;
  auto ld3 = [&](IX i) { return LBM_OK_IDX(i, fe) ? P3<T>::ld(F + i) : 0.0f; };
  auto st3 = [&](IX i, float val) {
    if (LBM_OK_IDX(i, fe)) P3<T>::st(F + i, val);
  };
  // Symmetry planes below y = 0 and/or z = 0: a ghost layer is the image of
  // the layer next to it (its mask rows are copies, so nb tells whether an
  // image cell is solid).  A population arriving from a fluid image cell is
  // the one its original cell sent with the crossed components negated; one
  // sent towards a fluid image cell comes back into the plane's layer with
  // those components negated, into the slot the local phase reads for it.
  // Solid images reflect as walls (the nb path).
  const bool py = (FEAT & kFeat3Mirror) && PHASE == 0 && !NB0 && on_py;
  const bool pz = (FEAT & kFeat3Mirror) && PHASE == 0 && !NB0 && on_pz;
  float g[kQ];
  g[0] = ld3(c);
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const IX off = cx3(i) + cy3(i) * sy + cz3(i) * sz;
    const bool xy = cy3(i) > 0 && py, xz = cz3(i) > 0 && pz;  // the source lies past a plane
    if (PHASE == 1 || (!NB0 && ((nb >> opp3(i)) & 1u)))
      g[i] = ld3(opp3(i) * pl + c);
    else if (xy && xz)
      g[i] = ld3(mirz3(mir3(i)) * pl + c - cx3(i));
    else if (xy)
      g[i] = ld3(mir3(i) * pl + c - (cx3(i) + cz3(i) * sz));
    else if (xz)
      g[i] = ld3(mirz3(i) * pl + c - (cx3(i) + cy3(i) * sy));
    else
      g[i] = ld3(i * pl + c - off);
  }
  if (!NB0 && port != 0) port3(g, port == 1, v.u_in[urow()], v.rho0);
  float drho, ux, uy, uz;
  if ((FEAT & kFeat3Models) && v.collision != LBM_COLLIDE_BGK)  // the plain build has no branch here
    collide_other3(g, v.rho0, v.omega, v.tau, v.collision, v.c_smag, drho, ux, uy, uz);
  else
    bgk3(g, v.rho0, v.omega, drho, ux, uy, uz);
  // Recompute the store addresses from the cell index instead of keeping the
  // 18 load addresses alive across the collision (halves the registers).
  opaque(c);
  opaque(pl);
  st3(c, g[0]);
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const IX off = cx3(i) + cy3(i) * sy + cz3(i) * sz;
    const bool xy = cy3(i) < 0 && py, xz = cz3(i) < 0 && pz;  // the target lies past a plane
    if (PHASE == 1 || (!NB0 && ((nb >> i) & 1u)))
      st3(i * pl + c, g[i]);
    else if (xy && xz)
      st3(opp3(mirz3(mir3(i))) * pl + c + cx3(i), g[i]);
    else if (xy)
      st3(opp3(mir3(i)) * pl + c + (cx3(i) + cz3(i) * sz), g[i]);
    else if (xz)
      st3(opp3(mirz3(i)) * pl + c + (cx3(i) + cy3(i) * sy), g[i]);
    else
      st3(opp3(i) * pl + c + off, g[i]);
  }
  if (MOM && LBM_OK_IDX(c, v.plane)) {
    v.drho[c] = drho;
    v.ux[c] = ux;
    v.uy[c] = uy;
    v.uz[c] = uz;
    if (!(isfinite(drho) && isfinite(ux) && isfinite(uy) && isfinite(uz))) atomicOr(v.flag, 1);
  }
}

// cell_core3 for cell x of row (y, z)
template <class T, int PHASE, int MOM, bool NB0, class IX, int FEAT>
__device__ __forceinline__ void cell_update3(const View3& v, int x, int y, int z, uint32_t nb) {
  const IX c = ((IX)z * v.ny + y) * (IX)v.nxp + x;
  const int port = NB0 ? 0 : (x == 0 ? 1 : (x == v.nx - 1 ? 2 : 0));
  cell_core3<T, PHASE, MOM, NB0, IX, FEAT>(v, c, nb, (v.mirror & 1) && y == 0, (v.mirror & 2) && z == 0, port,
                                           [&] { return (long long)z * v.ny + y; });
}

// Bit l set when some D3Q19 neighbour of cell 32 s + l of row (y, z) is solid
// (bits past the row's end and the padding words count as solid).
__device__ __forceinline__ uint32_t solid_nb3(const View3& v, int y, int z, int s) {
  uint32_t solid_nb = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy) {
      const uint32_t* row = v.mask + mask3_row(v.ny, v.ms, y + dy, z + dz) + 1;
      const uint32_t m = row[s];
      solid_nb |= (dy == 0 && dz == 0) ? 0u : m;        // c_x = 0 (not the cell itself)
      if (dy != 0 && dz != 0) continue;                 // D3Q19 has no (+-1, +-1, +-1)
      solid_nb |= __funnelshift_r(m, row[s + 1], 1);    // c_x = +1
      solid_nb |= __funnelshift_l(row[s - 1], m, 1);    // c_x = -1
    }
  return solid_nb;
}

// Solid flags of the 18 neighbours of the lane's cell of segment `seg` (bit
// i: x + c_i is solid), from the mask: lanes 0..26 load the 27 words around
// the segment (rows y-1..y+1 x z-1..z+1, words s-1..s+1) in one instruction
// and the warp shares them by shuffles.
__device__ __forceinline__ uint32_t neighbour_flags3(const View3& v, int seg, int lane) {
  const int row = seg / v.nsx;
  const int s = seg - row * v.nsx;
  const int z = row / v.ny;
  const int y = row - z * v.ny;
  // lanes 0..8: word s of row r = (dz+1)*3 + (dy+1); 9..17: word s-1; 18..26: word s+1
  uint32_t wv = 0xffffffffu;
  if (lane < 27) {
    const int part = lane / 9, r = lane - 9 * part;
    const int dy = r % 3 - 1, dz = r / 3 - 1;
    const int dw = part == 0 ? 0 : (part == 1 ? -1 : 1);
    wv = v.mask[mask3_row(v.ny, v.ms, y + dy, z + dz) + 1 + s + dw];
  }
  uint32_t M[9], Lw[9], H[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    M[r] = __shfl_sync(kFull, wv, r);
    Lw[r] = __shfl_sync(kFull, wv, 9 + r);
    H[r] = __shfl_sync(kFull, wv, 18 + r);
  }
  uint32_t nb = 0;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int r = (cz3(i) + 1) * 3 + (cy3(i) + 1);
    const uint32_t word = cx3(i) == 0 ? M[r]
                          : cx3(i) > 0 ? __funnelshift_r(M[r], H[r], 1)
                                       : __funnelshift_l(Lw[r], M[r], 1);
    nb |= ((word >> lane) & 1u) << i;
  }
  return nb;
}

// One phase on task t of the list (one row segment).  The neighbour flags
// (built with the list) are read before waiting for the previous step, the
// populations after.  Phase A on a segment whose fluid cells have no solid
// neighbour (and hence no port cell: outside the row reads as solid) takes
// the select-free path.
template <class T, int PHASE, int MOM, class IX, int FEAT>
__device__ __forceinline__ void seg_task3(const View3& v, Seg3 sg, int t, int lane, bool& waited) {
  const int seg = sg.seg & kSegIndexMask;
  const bool open = PHASE == 0 && (sg.seg & kSegOpen);
  const int row = seg / v.nsx;
  const int s = seg - row * v.nsx;
  const int z = row / v.ny;
  const int y = row - z * v.ny;
  const uint32_t nb = (PHASE == 0 && !open) ? v.nbs[(long long)t * 32 + lane] : 0u;
  if (!waited) {  // warp-uniform: the previous step's populations are final from here on
    asm volatile("griddepcontrol.wait;" ::: "memory");
    waited = true;
  }
  if ((sg.word >> lane) & 1u) return;  // solid, or past the row's end
  const int x = 32 * s + lane;
  if (open)
    cell_update3<T, PHASE, MOM, true, IX, FEAT>(v, x, y, z, 0u);
  else
    cell_update3<T, PHASE, MOM, false, IX, FEAT>(v, x, y, z, nb);
}

constexpr uint32_t kCell3Pad = 0xffffffffu;  // cell index of a padding entry of the packed list

// One phase on packed task t (t >= n_seg): entries 32 (t - n_seg) .. + 31 of
// the packed-cell list, the fluid cells of sparse segments one a lane.  No
// packed cell is a port cell or lies next to a symmetry plane (those
// segments stay segment tasks), so phase A needs only the neighbour flags
// (the task's flag block) and phase B only the index.  They are read before
// waiting for the previous step, the populations after.
template <class T, int PHASE, int MOM, class IX, int FEAT>
__device__ __forceinline__ void packed_task3(const View3& v, int t, int n_seg, int lane, bool& waited) {
  const uint32_t c = v.cidx[(long long)(t - n_seg) * 32 + lane];
  const uint32_t nb = PHASE == 0 ? v.nbs[(long long)t * 32 + lane] : 0u;
  if (!waited) {  // warp-uniform: the previous step's populations are final from here on
    asm volatile("griddepcontrol.wait;" ::: "memory");
    waited = true;
  }
  if (c == kCell3Pad) return;
  cell_core3<T, PHASE, MOM, PHASE == 1, IX, FEAT>(v, (IX)c, nb, false, false, 0, [] { return 0ll; });
}

// One phase of one time step over the task list (warps stride over it):
// tasks 0 .. counts[0]-1 are row segments, the rest packed cells.  Launched
// as a programmatic dependent of the previous step.
template <class T, int PHASE, int MOM, class IX, int FEAT>
__global__ void __launch_bounds__(512) k_step3(const View3 v, const Seg3* __restrict__ segs,
                                               const int* __restrict__ counts) {
  // the next step may be scheduled now; it touches populations only after
  // waiting for this grid to complete
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int n_seg = counts[0], n_task = counts[1];
  const int wpb = blockDim.x >> 5;
  const int stride = gridDim.x * wpb;
  bool waited = false;
  for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < n_task; t += stride) {
    if (t < n_seg)  // warp-uniform
      seg_task3<T, PHASE, MOM, IX, FEAT>(v, segs[t], t, lane, waited);
    else
      packed_task3<T, PHASE, MOM, IX, FEAT>(v, t, n_seg, lane, waited);
  }
  // every thread waits once, so this grid completes only after the previous one
  if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
}

inline int blocks_for(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b > 0 ? b : 1);
}

// ---- work-list ---------------------------------------------------------------
// word i of the rows y in [y0, ny-2], z in [z0, nz-2] (y0 = z0 = 1, or 0
// next to a symmetry plane for the step work-list)
__device__ __forceinline__ void word3_of(const View3& v, int y0, int z0, int i, int& y, int& z, int& s) {
  const int per_z = (v.ny - 1 - y0) * v.nsx;
  const int zi = i / per_z;
  const int rest = i - zi * per_z;
  const int yi = rest / v.nsx;
  s = rest - yi * v.nsx;
  y = y0 + yi;
  z = z0 + zi;
}

// Word i: cnt[i] = its fluid cells when it goes to packed tasks (fewer than
// pack_below, and neither a word holding a port column -- the first or the
// last of its row -- nor one on a layer next to a symmetry plane), else 0;
// flags[i] = 1 for a segment task (any other word holding fluid).
__global__ void k_seg3_flags(const View3 v, int total, int pack_below, int* __restrict__ flags,
                             int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int y, z, s;
  word3_of(v, first_row3(v), first_layer3(v), i, y, z, s);
  const int fill = __popc(~v.mask[mask3_row(v.ny, v.ms, y, z) + 1 + s]);
  const bool packable = fill < pack_below && s != 0 && s != v.nsx - 1 && !((v.mirror & 1) && y == 0) &&
                        !((v.mirror & 2) && z == 0);
  cnt[i] = packable ? fill : 0;
  flags[i] = fill > 0 && !packable;
}

// Entry of a segment holding fluid: its index, its own mask word, and
// kSegOpen when none of its fluid cells has a solid cell among its 18
// neighbours (the bits past the row's end and the padding count as solid).
__global__ void k_seg3_scatter(const View3 v, int total, const int* __restrict__ flags,
                               const int* __restrict__ offs, Seg3* __restrict__ segs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total || !flags[i]) return;
  int y, z, s;
  word3_of(v, first_row3(v), first_layer3(v), i, y, z, s);
  const uint32_t own = v.mask[mask3_row(v.ny, v.ms, y, z) + 1 + s];
  const uint32_t solid_nb = solid_nb3(v, y, z, s);
  // the layers next to a symmetry plane pull across it: never the open path
  const bool open = (solid_nb & ~own) == 0u && y >= 1 && z >= 1;
  const int seg = (z * v.ny + y) * v.nsx + s;
  segs[offs[i]] = Seg3{seg | (open ? kSegOpen : 0), own};
}

// Packed cells: one warp per word; lane l places cell 32 s + l of a sparse
// segment at its offset in the packed list, with its neighbour flags in the
// flag block after the segment tasks'.  Block 0 also pads the packed list to
// whole tasks and writes counts {segment tasks, tasks}.
__global__ void k_pack3_scatter(const View3 v, int total, const int* __restrict__ cnt,
                                const int* __restrict__ offs, const int* __restrict__ coffs,
                                uint32_t* __restrict__ cidx, uint32_t* __restrict__ nbs, int* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int n_seg = offs[total], n_packed = coffs[total];
  const int packed_end = (n_packed + 31) & ~31;
  uint32_t* flags = nbs + (long long)n_seg * 32;
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    if (n_packed + lane < packed_end) {
      cidx[n_packed + lane] = kCell3Pad;
      flags[n_packed + lane] = 0u;
    }
    if (lane == 0) {
      counts[0] = n_seg;
      counts[1] = n_seg + (packed_end >> 5);
    }
  }
  const uint32_t bit = 1u << lane, below = bit - 1u;
  const int stride = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < total; i += stride) {
    if (cnt[i] == 0) continue;  // warp-uniform
    int y, z, s;
    word3_of(v, first_row3(v), first_layer3(v), i, y, z, s);
    const uint32_t fluid = ~v.mask[mask3_row(v.ny, v.ms, y, z) + 1 + s];
    const uint32_t nb = neighbour_flags3(v, (z * v.ny + y) * v.nsx + s, lane);  // the whole warp
    if (fluid & bit) {
      const int k = coffs[i] + __popc(fluid & below);
      cidx[k] = (uint32_t)(((long long)z * v.ny + y) * v.nxp + 32 * s + lane);
      flags[k] = nb;
    }
  }
}

// neighbour flags of every cell of the list's segment tasks that are not
// open (one warp per segment; open segments need none)
__global__ void k_nb3(const View3 v, const Seg3* __restrict__ segs, const int* __restrict__ counts,
                      uint32_t* __restrict__ nbs) {
  const int lane = threadIdx.x & 31;
  const int nseg = counts[0];
  const int stride = (gridDim.x * blockDim.x) >> 5;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nseg; t += stride) {
    const Seg3 sg = segs[t];
    if (sg.seg & kSegOpen) continue;  // warp-uniform
    nbs[(long long)t * 32 + lane] = neighbour_flags3(v, sg.seg & kSegIndexMask, lane);
  }
}

// ---- reductions ----------------------------------------------------------------
constexpr int kObsThreads = 256;

// fixed-order block sum (deterministic for a fixed block size)
__device__ double block_sum(double a, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = a;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;  // valid in thread 0
}

// block 0: dp and m_in; block 1 + r: m_out of region r.  Port lists hold row
// indices z * ny + y (the column is 0 at the inlet, nx-1 at the outlet).
__global__ void __launch_bounds__(kObsThreads) k_obs3(const View3 v, const int* __restrict__ in_rows, int n_in,
                                                      const int* __restrict__ out_rows,
                                                      const int* __restrict__ out_off, int n_regions,
                                                      double* __restrict__ result) {
  __shared__ double sh[kObsThreads / 32];
  const double rho0 = (double)v.rho0;
  if (blockIdx.x == 0) {
    double di = 0.0, mi = 0.0, dout = 0.0;
    for (int k = threadIdx.x; k < n_in; k += blockDim.x) {
      const long long c = (long long)in_rows[k] * v.nxp;
      const double d = (double)v.drho[c];
      di += d;
      mi += (rho0 + d) * (double)v.ux[c];
    }
    const int n_out = out_off[n_regions];
    for (int k = threadIdx.x; k < n_out; k += blockDim.x)
      dout += (double)v.drho[(long long)out_rows[k] * v.nxp + (v.nx - 1)];
    const double s_di = block_sum(di, sh);
    const double s_mi = block_sum(mi, sh);
    const double s_do = block_sum(dout, sh);
    if (threadIdx.x == 0) {
      result[0] = (s_di / (double)n_in - s_do / (double)n_out) / 3.0;
      result[1] = s_mi;
    }
  } else {
    const int r = blockIdx.x - 1;
    double m = 0.0;
    for (int k = out_off[r] + threadIdx.x; k < out_off[r + 1]; k += blockDim.x) {
      const long long c = (long long)out_rows[k] * v.nxp + (v.nx - 1);
      m += (rho0 + (double)v.drho[c]) * (double)v.ux[c];
    }
    const double t = block_sum(m, sh);
    if (threadIdx.x == 0) result[2 + r] = t;
  }
}

// ---- exchange ------------------------------------------------------------------
struct Words3 {
  uint32_t fluid_cand, solid_cand, e, w, n, s, u, d;  // neighbour words: bit set = solid
};

__device__ __forceinline__ uint32_t region3_bits(int s, int nx) {
  // bits b with 2 <= 32 s + b <= nx - 3
  uint32_t m = 0xffffffffu;
  const int x0 = s * 32;
  if (x0 < 2) m &= ~((1u << (2 - x0)) - 1u);
  const int hi = nx - 3 - x0;
  if (hi < 0) return 0u;
  if (hi < 31) m &= (2u << hi) - 1u;
  return m;
}

__device__ __forceinline__ Words3 words3(const View3& v, int y, int z, int s) {
  const uint32_t* row = v.mask + mask3_row(v.ny, v.ms, y, z) + 1;
  const long long ry = v.ms, rz = (long long)(v.ny + 2) * v.ms;
  Words3 r;
  const uint32_t mc = row[s];
  r.e = __funnelshift_r(mc, row[s + 1], 1);
  r.w = __funnelshift_l(row[s - 1], mc, 1);
  r.n = row[s + ry];
  r.s = row[s - ry];
  r.u = row[s + rz];
  r.d = row[s - rz];
  const uint32_t reg = region3_bits(s, v.nx);
  r.fluid_cand = ~mc & (r.e | r.w | r.n | r.s | r.u | r.d) & reg;
  r.solid_cand = mc & (~r.e | ~r.w | ~r.n | ~r.s | ~r.u | ~r.d) & reg;
  return r;
}

__global__ void k_oc3_count(const View3 v, int total, int* __restrict__ cnt_f, int* __restrict__ cnt_s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int y, z, s;
  word3_of(v, 1, 1, i, y, z, s);
  const Words3 m = words3(v, y, z, s);
  cnt_f[i] = __popc(m.fluid_cand);
  cnt_s[i] = __popc(m.solid_cand);
}

__device__ __forceinline__ unsigned long long order_key3(double x) {
  x = __dadd_rn(x, 0.0);  // -0 -> +0
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// |u_t| of a face neighbour: the magnitude of its two velocity components
// along the face, sqrt(a^2 + b^2), FP64 and correctly rounded
__device__ __forceinline__ double tangential(float a, float b) {
  const double da = (double)a, db = (double)b;
  return __dsqrt_rn(__dadd_rn(__dmul_rn(da, da), __dmul_rn(db, db)));
}

__global__ void k_oc3_emit(const View3 v, const float* __restrict__ drho, const float* __restrict__ ux,
                           const float* __restrict__ uy, const float* __restrict__ uz, double mu, int total,
                           const int* __restrict__ off_f, const int* __restrict__ off_s,
                           unsigned long long* __restrict__ key_f, int* __restrict__ idx_f,
                           unsigned long long* __restrict__ key_s, int* __restrict__ idx_s,
                           int* __restrict__ info) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int y, z, s;
  word3_of(v, 1, 1, i, y, z, s);
  const Words3 m = words3(v, y, z, s);
  const double rho0 = (double)v.rho0;
  const long long sy = v.nxp, sz = (long long)v.ny * v.nxp;
  const long long rowc = ((long long)z * v.ny + y) * v.nxp;
  const int rowd = (z * v.ny + y) * v.nx;
  int of = off_f[i], os = off_s[i];
  bool bad = false;
  uint32_t fc = m.fluid_cand;
  while (fc) {
    const int b = __ffs(fc) - 1;
    fc &= fc - 1;
    const int x = 32 * s + b;
    const long long c = rowc + x;
    const double a = (double)ux[c], bb = (double)uy[c], cc = (double)uz[c];
    const double rho = __dadd_rn(rho0, (double)drho[c]);
    const double sq = __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(bb, bb)), __dmul_rn(cc, cc));
    const double q = __dmul_rn(__dmul_rn(0.5, rho), sq);
    bad |= isnan(q);
    key_f[of] = order_key3(q);
    idx_f[of] = rowd + x;
    ++of;
  }
  uint32_t sc = m.solid_cand;
  while (sc) {
    const int b = __ffs(sc) - 1;
    sc &= sc - 1;
    const int x = 32 * s + b;
    const long long c = rowc + x;
    // fluid face neighbours in the order +x, +y, -x, -y, +z, -z
    double sigma = 0.0;
    if (!((m.e >> b) & 1u)) sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, tangential(uy[c + 1], uz[c + 1])), 0.5));
    if (!((m.n >> b) & 1u))
      sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, tangential(ux[c + sy], uz[c + sy])), 0.5));
    if (!((m.w >> b) & 1u)) sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, tangential(uy[c - 1], uz[c - 1])), 0.5));
    if (!((m.s >> b) & 1u))
      sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, tangential(ux[c - sy], uz[c - sy])), 0.5));
    if (!((m.u >> b) & 1u))
      sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, tangential(ux[c + sz], uy[c + sz])), 0.5));
    if (!((m.d >> b) & 1u))
      sigma = __dadd_rn(sigma, __ddiv_rn(__dmul_rn(mu, tangential(ux[c - sz], uy[c - sz])), 0.5));
    bad |= isnan(sigma);
    key_s[os] = ~order_key3(sigma);  // ascending key = descending sigma
    idx_s[os] = rowd + x;
    ++os;
  }
  if (bad) atomicOr(info + 3, 1);
}

template <class T>
__global__ void k_oc3_apply(const View3 v, const int* __restrict__ sel_f, const int* __restrict__ sel_s,
                            const int* __restrict__ info) {
  const int n = info[0];
  T* F = static_cast<T*>(v.f);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int id = side == 0 ? sel_f[k] : sel_s[k];
      const int row = id / v.nx, x = id - row * v.nx;
      const int z = row / v.ny, y = row - z * v.ny;
      uint32_t* w = v.mask + mask3_row(v.ny, v.ms, y, z) + 1 + (x >> 5);
      const long long c = (long long)row * v.nxp + x;
      if (side == 0) {  // fluid -> solid
        atomicOr(w, 1u << (x & 31));
      } else {          // solid -> fluid at the rest equilibrium of rho0: g_i = 0
        atomicAnd(w, ~(1u << (x & 31)));
#pragma unroll
        for (int i = 0; i < kQ; ++i) P3<T>::st(F + i * v.plane + c, 0.0f);
      }
      v.drho[c] = 0.0f;
      v.ux[c] = 0.0f;
      v.uy[c] = 0.0f;
      v.uz[c] = 0.0f;
    }
  }
}

__global__ void k_unpack3(const View3 v, uint8_t* __restrict__ cells) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)v.nx * v.ny * v.nz;
  if (i >= n) return;
  const long long row = i / v.nx;
  const int x = (int)(i - row * v.nx);
  const int z = (int)(row / v.ny), y = (int)(row - (long long)z * v.ny);
  cells[i] = (uint8_t)((v.mask[mask3_row(v.ny, v.ms, y, z) + 1 + (x >> 5)] >> (x & 31)) & 1u);
}

// FEAT: the build with the collision models beyond BGK and/or the symmetry
// plane (kept apart so that the plain build keeps its registers)
template <class T, class IX, int FEAT>
void* step3_kernel(int phase, int moments) {
  if (phase == 0) return (void*)k_step3<T, 0, 0, IX, FEAT>;
  return moments ? (void*)k_step3<T, 1, 1, IX, FEAT> : (void*)k_step3<T, 1, 0, IX, FEAT>;
}

template <class T, class IX>
void* step3_kernel(int phase, int moments, int feat) {
  switch (feat) {
    case 0: return step3_kernel<T, IX, 0>(phase, moments);
    case kFeat3Models: return step3_kernel<T, IX, kFeat3Models>(phase, moments);
    case kFeat3Mirror: return step3_kernel<T, IX, kFeat3Mirror>(phase, moments);
    default: return step3_kernel<T, IX, kFeat3Models | kFeat3Mirror>(phase, moments);
  }
}

template <class T>
void* step3_kernel(int phase, int moments, bool idx64, int feat) {
  return idx64 ? step3_kernel<T, long long>(phase, moments, feat) : step3_kernel<T, int>(phase, moments, feat);
}

void* step3_for(int precision, int phase, int moments, bool idx64, int feat) {
  switch (precision) {
    case LBM_F32: return step3_kernel<float>(phase, moments, idx64, feat);
    case LBM_BF16_SHIFTED: return step3_kernel<__nv_bfloat16>(phase, moments, idx64, feat);
    case LBM_F16_SHIFTED: return step3_kernel<__half>(phase, moments, idx64, feat);
    default: return nullptr;
  }
}

inline bool needs_idx64(const View3& v) { return v.idx64 != 0; }

inline int feat3(const View3& v) {
  return (v.collision != LBM_COLLIDE_BGK ? kFeat3Models : 0) | (v.mirror ? kFeat3Mirror : 0);
}

}  // namespace

size_t seg3_scratch_ints(long long total) { return 4 * (size_t)total + 2 + scan_tmp_ints(total); }

size_t packed3_capacity(long long fluid) { return (size_t)fluid + 32; }

cudaError_t launch_build_segments3(const View3& v, int pack_below, int* scratch, Seg3* segs, int* counts,
                                   cudaStream_t stream) {
  const int total = seg3_words(v);
  int* flags = scratch;
  int* offs = scratch + total;           // total + 1
  int* cnt = scratch + 2 * total + 1;
  int* coffs = scratch + 3 * total + 1;  // total + 1
  int* tmp = scratch + 4 * total + 2;
  k_seg3_flags<<<blocks_for(total, 256), 256, 0, stream>>>(v, total, pack_below, flags, cnt);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_scan(flags, offs, total, tmp, stream)) != cudaSuccess) return e;
  if ((e = launch_scan(cnt, coffs, total, tmp, stream)) != cudaSuccess) return e;
  k_seg3_scatter<<<blocks_for(total, 256), 256, 0, stream>>>(v, total, flags, offs, segs);
  count_launches(1);
  uint32_t* nbs = const_cast<uint32_t*>(v.nbs);
  k_pack3_scatter<<<blocks_for((long long)total * 32, 256), 256, 0, stream>>>(
      v, total, cnt, offs, coffs, const_cast<uint32_t*>(v.cidx), nbs, counts);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_nb3<<<blocks_for((long long)total * 32, 256), 256, 0, stream>>>(v, segs, counts, nbs);
  count_launches(1);
  return cudaGetLastError();
}

int step3_resident_blocks(int precision, int phase, int moments, int warps_per_block, const View3& v) {
  void* k = step3_for(precision, phase, moments, needs_idx64(v), feat3(v));
  int dev = 0, sms = 0, n = 0;
  if (!k || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps_per_block, 0) != cudaSuccess)
    return 0;
  return n * sms;
}

cudaError_t launch_step3(int precision, int phase, int moments, const View3& v, const Seg3* segs,
                         const int* counts, int blocks, int warps_per_block, cudaStream_t stream) {
  void* k = step3_for(precision, phase, moments, needs_idx64(v), feat3(v));
  if (!k || blocks < 1) return cudaErrorInvalidValue;
  void* args[] = {(void*)&v, (void*)&segs, (void*)&counts};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(32 * warps_per_block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

cudaError_t launch_observables3(const View3& v, const int* in_rows, int n_in, const int* out_rows,
                                const int* out_off, int n_regions, double* result, cudaStream_t stream) {
  k_obs3<<<1 + n_regions, kObsThreads, 0, stream>>>(v, in_rows, n_in, out_rows, out_off, n_regions, result);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_oc_select3(const View3& v, const float* drho, const float* ux, const float* uy,
                              const float* uz, double mu, const LatticeView* one, const int* word_off,
                              const int* n_swap, const OcScratch& s, cudaStream_t stream) {
  const int total = (v.ny - 2) * (v.nz - 2) * v.nsx;
  cudaError_t e = cudaMemsetAsync(s.info, 0, 8 * sizeof(int), stream);
  if (e != cudaSuccess) return e;
  k_oc3_count<<<blocks_for(total, 256), 256, 0, stream>>>(v, total, s.cnt_f, s.cnt_s);
  count_launches(1);
  if ((e = launch_scan(s.cnt_f, s.off_f, total, s.scan_tmp, stream)) != cudaSuccess) return e;
  if ((e = launch_scan(s.cnt_s, s.off_s, total, s.scan_tmp, stream)) != cudaSuccess) return e;
  k_oc3_emit<<<blocks_for(total, 256), 256, 0, stream>>>(v, drho, ux, uy, uz, mu, total, s.off_f, s.off_s, s.key_f,
                                                         s.idx_f, s.key_s, s.idx_s, s.info);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_oc_select_only(one, word_off, 1, n_swap, s, stream);
}

cudaError_t launch_oc_apply3(int precision, const View3& v, const OcScratch& s, cudaStream_t stream) {
  switch (precision) {
    case LBM_F32: k_oc3_apply<float><<<8, 128, 0, stream>>>(v, s.sel_f, s.sel_s, s.info); break;
    case LBM_BF16_SHIFTED: k_oc3_apply<__nv_bfloat16><<<8, 128, 0, stream>>>(v, s.sel_f, s.sel_s, s.info); break;
    case LBM_F16_SHIFTED: k_oc3_apply<__half><<<8, 128, 0, stream>>>(v, s.sel_f, s.sel_s, s.info); break;
    default: return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack_mask3(const View3& v, uint8_t* cells, cudaStream_t stream) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  k_unpack3<<<blocks_for(n, 256), 256, 0, stream>>>(v, cells);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace lbm
