/*
 * lbm3d_oracle.c -- plain FP64 CPU statement of the three-dimensional
 * extension of the method (D3Q19): the same loop of Sec. 2.3 -- lattice BGK
 * solve, pressure drop and outlet flow rates, optimality-criterion exchange
 * of fluid and solid cells -- on a 3D lattice.  The paper computes in 2D and
 * names 3D distributors (its references) as the next step; every 3D choice
 * below is a reading, stated where it is made.
 *
 * TEST INFRASTRUCTURE ONLY, like lbm_oracle.c: nothing on the product path
 * loads it, and it shares no code with the CUDA library.  Two lattices, pull
 * streaming, every cell visited, double precision, no fused multiply-add,
 * sums in ascending index order.
 *
 * Layout: populations f[i*N + (z*ny + y)*nx + x], i = 0..18, N = nx*ny*nz;
 * cell arrays (z*ny + y)*nx + x; solid[] = 1 for a solid cell.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* D3Q19: rest, the 6 face neighbours (weight 1/18), the 12 edge neighbours
 * (weight 1/36); c_s^2 = 1/3.  Opposite pairs are (1,2), (3,4), ..., (17,18). */
static const int C3X[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int C3Y[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int C3Z[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const int OPP3[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
/* reflection in a plane normal to y: the direction with c_y negated */
static const int MIR3[19] = {0, 1, 2, 4, 3, 5, 6, 9, 10, 7, 8, 11, 12, 13, 14, 18, 17, 16, 15};
/* reflection in a plane normal to z: the direction with c_z negated */
static const int MIRZ3[19] = {0, 1, 2, 3, 4, 6, 5, 7, 8, 9, 10, 13, 14, 11, 12, 17, 18, 15, 16};
static const double W3[19] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                              1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2_3 = 1.0 / 3.0;

enum { ORA3_OK = 0, ORA3_ERR_ARG = 1, ORA3_ERR_GEOMETRY = 2, ORA3_ERR_DIVERGED = 5 };
enum { ORA3_REINIT_WARM = 0, ORA3_REINIT_COLD = 1 };
enum { ORA3_COLLIDE_BGK = 0, ORA3_COLLIDE_REGULARIZED = 1, ORA3_COLLIDE_SMAGORINSKY = 2 };

typedef struct {
  int32_t nx, ny, nz;  /* x along the flow, y across, z through the depth   */
  int32_t periodic;    /* bit 0: wrap x, bit 1: wrap y, bit 2: wrap z; a
                          wrapped x axis has no ports (checks of the bulk
                          scheme only)                                       */
  double tau, rho0, u_max;
  int32_t collision;   /* ORA3_COLLIDE_*, as in 2D                           */
  int32_t mirror;      /* bit 0: a symmetry plane half a cell below y = 0, bit
                          1: one half a cell below z = 0 (the 2D rule of Sec.
                          3.3's half domain, per plane): the layer next to a
                          plane may be fluid, and what crosses a plane comes
                          back as the mirror image of what that layer sends
                          out (both components negated past the corner)      */
  double c_smag;       /* Smagorinsky constant                               */
} ora3_params;

void ora3_lattice(int32_t* cx, int32_t* cy, int32_t* cz, int32_t* opp, double* w, double* cs2) {
  for (int i = 0; i < 19; ++i) {
    cx[i] = C3X[i];
    cy[i] = C3Y[i];
    cz[i] = C3Z[i];
    opp[i] = OPP3[i];
    w[i] = W3[i];
  }
  *cs2 = CS2_3;
}

/* second-order equilibrium, as in 2D (Sec. 2.1) */
double ora3_feq(int32_t i, double rho, double ux, double uy, double uz) {
  double cu = C3X[i] * ux + C3Y[i] * uy + C3Z[i] * uz;
  double uu = ux * ux + uy * uy + uz * uz;
  return W3[i] * rho * (1.0 + cu / CS2_3 + (cu * cu) / (2.0 * CS2_3 * CS2_3) - uu / (2.0 * CS2_3));
}

static size_t cell3(const ora3_params* p, int x, int y, int z) {
  return ((size_t)z * p->ny + y) * p->nx + x;
}

/* Geometry rules: the faces y = 0, y = ny-1, z = 0, z = nz-1 solid (unless
 * wrapped); every inlet cell (x = 0) has a fluid cell behind it, every
 * outlet cell (x = nx-1) one before it; at least one inlet and one outlet. */
int32_t ora3_check_geometry(const ora3_params* p, const uint8_t* solid) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  if (nx < 4 || ny < 3 || nz < 3) return ORA3_ERR_ARG;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int edge_y = !(p->periodic & 2) && ((y == 0 && !(p->mirror & 1)) || y == ny - 1);
        int edge_z = !(p->periodic & 4) && ((z == 0 && !(p->mirror & 2)) || z == nz - 1);
        if ((edge_y || edge_z) && !solid[cell3(p, x, y, z)]) return ORA3_ERR_GEOMETRY;
      }
  if (p->periodic & 1) return ORA3_OK;
  int n_in = 0, n_out = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      if (!solid[cell3(p, 0, y, z)]) {
        if (solid[cell3(p, 1, y, z)]) return ORA3_ERR_GEOMETRY;
        ++n_in;
      }
      if (!solid[cell3(p, nx - 1, y, z)]) {
        if (solid[cell3(p, nx - 2, y, z)]) return ORA3_ERR_GEOMETRY;
        ++n_out;
      }
    }
  return (n_in && n_out) ? ORA3_OK : ORA3_ERR_GEOMETRY;
}

/* Inlet speeds (a reading: the parabolic profile of Sec. 3.3 taken along
 * each walled cross direction).  For inlet cell (0, y, z): its fluid run
 * along y at this z spans [y_lo, y_hi), its run along z at this y spans
 * [z_lo, z_hi); s_y = (y - y_lo + 1/2) / (y_hi - y_lo), likewise s_z;
 * a_y = 4 s_y (1 - s_y), or 1 when y wraps, likewise a_z; u_x = u_max a_y a_z.
 * So a duct gets 16 u_max s_y (1 - s_y) s_z (1 - s_z), and a slot wrapped in
 * y the plane-channel parabola of the 2D method.  u_in[z*ny + y].            */
void ora3_inlet_profile(const ora3_params* p, const uint8_t* solid, double* u_in) {
  int ny = p->ny, nz = p->nz;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      u_in[(size_t)z * ny + y] = 0.0;
      if (solid[cell3(p, 0, y, z)]) continue;
      double ay = 1.0, az = 1.0;
      if (!(p->periodic & 2)) {
        int lo = y, hi = y;
        while (lo > 0 && !solid[cell3(p, 0, lo - 1, z)]) --lo;
        while (hi < ny && !solid[cell3(p, 0, hi, z)]) ++hi;
        /* a run against the symmetry plane is half of a run twice as wide,
           centred on the plane */
        if ((p->mirror & 1) && lo == 0) lo = -hi;
        double s = ((double)(y - lo) + 0.5) / (double)(hi - lo);
        ay = 4.0 * s * (1.0 - s);
      }
      if (!(p->periodic & 4)) {
        int lo = z, hi = z;
        while (lo > 0 && !solid[cell3(p, 0, y, lo - 1)]) --lo;
        while (hi < nz && !solid[cell3(p, 0, y, hi)]) ++hi;
        if ((p->mirror & 2) && lo == 0) lo = -hi;
        double s = ((double)(z - lo) + 0.5) / (double)(hi - lo);
        az = 4.0 * s * (1.0 - s);
      }
      u_in[(size_t)z * ny + y] = p->u_max * ay * az;
    }
}

/* Outlet regions: the fluid cells of the face x = nx-1 grouped into
 * 4-connected components (in y, z; across a wrapped axis too); numbered in
 * the order of their first cell, z-major then y.  ids[z*ny + y] = region or -1.  Returns the count.  */
int32_t ora3_outlet_ids(const ora3_params* p, const uint8_t* solid, int32_t* ids) {
  int ny = p->ny, nz = p->nz, nx = p->nx, n = 0;
  size_t m = (size_t)ny * nz;
  for (size_t k = 0; k < m; ++k) ids[k] = -1;
  int* stack = (int*)malloc(sizeof(int) * (m ? m : 1));
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      size_t k = (size_t)z * ny + y;
      if (ids[k] >= 0 || solid[cell3(p, nx - 1, y, z)]) continue;
      int top = 0;
      stack[top++] = (int)k;
      ids[k] = n;
      while (top) {
        int q = stack[--top];
        int qy = q % ny, qz = q / ny;
        const int dy[4] = {1, -1, 0, 0}, dz[4] = {0, 0, 1, -1};
        for (int d = 0; d < 4; ++d) {
          int yy = qy + dy[d], zz = qz + dz[d];
          if (p->periodic & 2) yy = (yy + ny) % ny;
          if (p->periodic & 4) zz = (zz + nz) % nz;
          if (yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
          size_t kk = (size_t)zz * ny + yy;
          if (ids[kk] < 0 && !solid[cell3(p, nx - 1, yy, zz)]) {
            ids[kk] = n;
            stack[top++] = (int)kk;
          }
        }
      }
      ++n;
    }
  free(stack);
  return n;
}

void ora3_init(const ora3_params* p, const uint8_t* solid, double* f) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  for (int i = 0; i < 19; ++i)
    for (size_t c = 0; c < n; ++c) f[i * n + c] = solid[c] ? 0.0 : W3[i] * p->rho0;
}

/* f of every fluid cell at the equilibrium of the given (rho, u) */
void ora3_init_state(const ora3_params* p, const uint8_t* solid, const double* rho, const double* ux,
                     const double* uy, const double* uz, double* f) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  for (int i = 0; i < 19; ++i)
    for (size_t c = 0; c < n; ++c) f[i * n + c] = solid[c] ? 0.0 : ora3_feq(i, rho[c], ux[c], uy[c], uz[c]);
}

/* pull of direction i into cell (x, y, z); 0 if the source is outside the
 * lattice across a port face (the port rule supplies the population) */
static int pull3(const ora3_params* p, const uint8_t* solid, const double* fp, int i, int x, int y, int z,
                 double* out) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  int sx = x - C3X[i], sy = y - C3Y[i], sz = z - C3Z[i];
  if (p->periodic & 1) sx = (sx + p->nx) % p->nx;
  if (p->periodic & 2) sy = (sy + p->ny) % p->ny;
  if (p->periodic & 4) sz = (sz + p->nz) % p->nz;
  /* a ghost layer below a symmetry plane is the mirror image of the layer
     next to it: a solid image reflects as a wall (halfway bounce-back); a
     fluid one sends the population of its original cell with the crossed
     components negated */
  int ry = 0, rz = 0;
  if ((p->mirror & 1) && !(p->periodic & 2) && sy == -1) {
    ry = 1;
    sy = 0;
  }
  if ((p->mirror & 2) && !(p->periodic & 4) && sz == -1) {
    rz = 1;
    sz = 0;
  }
  if ((ry || rz) && sx >= 0 && sx < p->nx && sy < p->ny && sz < p->nz) {
    size_t img = cell3(p, sx, sy, sz), here = cell3(p, x, y, z);
    int j = i;
    if (ry) j = MIR3[j];
    if (rz) j = MIRZ3[j];
    *out = solid[img] ? fp[OPP3[i] * n + here] : fp[j * n + img];
    return 1;
  }
  if (sx < 0 || sx >= p->nx || sy < 0 || sy >= p->ny || sz < 0 || sz >= p->nz) return 0;
  size_t src = cell3(p, sx, sy, sz), here = cell3(p, x, y, z);
  *out = solid[src] ? fp[OPP3[i] * n + here] : fp[i * n + src];
  return 1;
}

/* Regularised populations: f_i = f_i^eq + w_i / (2 c_s^4) Q_i : Pi^neq,
 * Q_i = c_i c_i - c_s^2 I, Pi^neq = sum_i c_i c_i (f_i - f_i^eq).            */
static void regularize3(double* f, double rho, double ux, double uy, double uz) {
  double pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
  for (int i = 0; i < 19; ++i) {
    double nq = f[i] - ora3_feq(i, rho, ux, uy, uz);
    pxx += C3X[i] * C3X[i] * nq;
    pyy += C3Y[i] * C3Y[i] * nq;
    pzz += C3Z[i] * C3Z[i] * nq;
    pxy += C3X[i] * C3Y[i] * nq;
    pxz += C3X[i] * C3Z[i] * nq;
    pyz += C3Y[i] * C3Z[i] * nq;
  }
  for (int i = 0; i < 19; ++i) {
    double q = (C3X[i] * C3X[i] - CS2_3) * pxx + (C3Y[i] * C3Y[i] - CS2_3) * pyy + (C3Z[i] * C3Z[i] - CS2_3) * pzz +
               2.0 * (C3X[i] * C3Y[i] * pxy + C3X[i] * C3Z[i] * pxz + C3Y[i] * C3Z[i] * pyz);
    f[i] = ora3_feq(i, rho, ux, uy, uz) + W3[i] / (2.0 * CS2_3 * CS2_3) * q;
  }
}

void ora3_regularize(double* f, double rho, double ux, double uy, double uz) { regularize3(f, rho, ux, uy, uz); }

/* Relaxation time of the Smagorinsky closure (the 2D oracle's derivation
 * with the six components of the symmetric 3D stress): nu_t = C^2 |S|,
 * |S| = sqrt(2 S:S), S = -Pi / (2 rho c_s^2 tau_eff), tau_eff = tau + nu_t /
 * c_s^2, whose positive root is
 *   tau_eff = (tau + sqrt(tau^2 + 2 sqrt(2) C^2 sqrt(Pi:Pi) / (rho c_s^4))) / 2,
 * Pi:Pi = Pxx^2 + Pyy^2 + Pzz^2 + 2 (Pxy^2 + Pxz^2 + Pyz^2).                */
static double smagorinsky_tau3(double tau, double c, double rho, const double* f, double ux, double uy,
                               double uz) {
  double pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
  for (int i = 0; i < 19; ++i) {
    double nq = f[i] - ora3_feq(i, rho, ux, uy, uz);
    pxx += C3X[i] * C3X[i] * nq;
    pyy += C3Y[i] * C3Y[i] * nq;
    pzz += C3Z[i] * C3Z[i] * nq;
    pxy += C3X[i] * C3Y[i] * nq;
    pxz += C3X[i] * C3Z[i] * nq;
    pyz += C3Y[i] * C3Z[i] * nq;
  }
  double pp = pxx * pxx + pyy * pyy + pzz * pzz + 2.0 * (pxy * pxy + pxz * pxz + pyz * pyz);
  return 0.5 * (tau + sqrt(tau * tau + 2.0 * sqrt(2.0) * c * c * sqrt(pp) / (rho * CS2_3 * CS2_3)));
}

/* The collision of one cell with moments (rho, u), in place, as in 2D:
 *   BGK:          f_i <- f_i - (f_i - f_i^eq) / tau;
 *   regularised:  f_i <- f_i^eq + (1 - 1/tau) (second-order Hermite projection
 *                 of f - f^eq);
 *   Smagorinsky:  BGK with the local tau_eff above.                          */
static void collide3(const ora3_params* p, double* f, double rho, double ux, double uy, double uz) {
  if (p->collision == ORA3_COLLIDE_REGULARIZED) {
    double fr[19];
    for (int i = 0; i < 19; ++i) fr[i] = f[i];
    regularize3(fr, rho, ux, uy, uz);
    for (int i = 0; i < 19; ++i) {
      double eq = ora3_feq(i, rho, ux, uy, uz);
      f[i] = eq + (1.0 - 1.0 / p->tau) * (fr[i] - eq);
    }
    return;
  }
  double tau = p->tau;
  if (p->collision == ORA3_COLLIDE_SMAGORINSKY) tau = smagorinsky_tau3(p->tau, p->c_smag, rho, f, ux, uy, uz);
  for (int i = 0; i < 19; ++i) f[i] = f[i] - (f[i] - ora3_feq(i, rho, ux, uy, uz)) / tau;
}

/* The moments and collision of one cell (for the pins); returns tau_eff. */
double ora3_collide(const ora3_params* p, double* f) {
  double rho = 0, jx = 0, jy = 0, jz = 0;
  for (int i = 0; i < 19; ++i) {
    rho += f[i];
    jx += C3X[i] * f[i];
    jy += C3Y[i] * f[i];
    jz += C3Z[i] * f[i];
  }
  double ux = jx / rho, uy = jy / rho, uz = jz / rho;
  double tau = p->collision == ORA3_COLLIDE_SMAGORINSKY ? smagorinsky_tau3(p->tau, p->c_smag, rho, f, ux, uy, uz)
                                                         : p->tau;
  collide3(p, f, rho, ux, uy, uz);
  return tau;
}

/* One time step (stream with halfway bounce-back, ports, BGK collision).
 * Collision: BGK, regularised or Smagorinsky (collide3).
 * Ports (the 2D rules of Sec. 3.3 carried to 3D, regularised):
 *   inlet x = 0: velocity (u_in, 0, 0); rho from mass and x-momentum of the
 *     known populations, rho = (sum_{c_x=0} f + 2 sum_{c_x<0} f) / (1 - u);
 *     each unknown (c_x > 0) population takes the equilibrium plus the
 *     non-equilibrium part of its opposite; then the cell is regularised;
 *   outlet x = nx-1: density rho0, u = (-1 + (sum_{c_x=0} f + 2 sum_{c_x>0} f)
 *     / rho0, 0, 0); unknown (c_x < 0) populations likewise; regularised.   */
void ora3_step(const ora3_params* p, const uint8_t* solid, const double* u_in, const double* fp, double* fn,
               double* rho_out, double* ux_out, double* uy_out, double* uz_out) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  size_t n = (size_t)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t c = cell3(p, x, y, z);
        if (solid[c]) {
          for (int i = 0; i < 19; ++i) fn[i * n + c] = 0.0;
          if (rho_out) { rho_out[c] = 0; ux_out[c] = 0; uy_out[c] = 0; uz_out[c] = 0; }
          continue;
        }
        double f[19];
        for (int i = 0; i < 19; ++i)
          if (!pull3(p, solid, fp, i, x, y, z, &f[i])) f[i] = 0.0;
        int ports = !(p->periodic & 1);
        if (ports && (x == 0 || x == nx - 1)) {
          int inlet = x == 0;
          double s0 = 0.0, sk = 0.0;  /* sum over c_x = 0, and over the known side */
          for (int i = 0; i < 19; ++i) {
            if (C3X[i] == 0) s0 += f[i];
            else if ((inlet && C3X[i] < 0) || (!inlet && C3X[i] > 0)) sk += f[i];
          }
          double rho, ux;
          if (inlet) {
            ux = u_in[(size_t)z * ny + y];
            rho = (s0 + 2.0 * sk) / (1.0 - ux);
          } else {
            rho = p->rho0;
            ux = -1.0 + (s0 + 2.0 * sk) / rho;
          }
          for (int i = 0; i < 19; ++i) {
            int unknown = inlet ? C3X[i] > 0 : C3X[i] < 0;
            if (unknown)
              f[i] = ora3_feq(i, rho, ux, 0.0, 0.0) + (f[OPP3[i]] - ora3_feq(OPP3[i], rho, ux, 0.0, 0.0));
          }
          regularize3(f, rho, ux, 0.0, 0.0);
        }
        double rho = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < 19; ++i) {
          rho += f[i];
          jx += C3X[i] * f[i];
          jy += C3Y[i] * f[i];
          jz += C3Z[i] * f[i];
        }
        double ux = jx / rho, uy = jy / rho, uz = jz / rho;
        collide3(p, f, rho, ux, uy, uz);
        for (int i = 0; i < 19; ++i) fn[i * n + c] = f[i];
        if (rho_out) { rho_out[c] = rho; ux_out[c] = ux; uy_out[c] = uy; uz_out[c] = uz; }
      }
}

int32_t ora3_run(const ora3_params* p, const uint8_t* solid, const double* u_in, double* f, double* work,
                 int64_t n_steps, double* rho, double* ux, double* uy, double* uz) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  double* a = f;
  double* b = work;
  for (int64_t t = 0; t < n_steps; ++t) {
    ora3_step(p, solid, u_in, a, b, rho, ux, uy, uz);
    double* tmp = a;
    a = b;
    b = tmp;
  }
  if (a != f) memcpy(f, a, sizeof(double) * 19 * n);
  for (size_t c = 0; c < n; ++c)
    if (!solid[c] && !isfinite(rho[c])) return ORA3_ERR_DIVERGED;
  return ORA3_OK;
}

/* Pressure drop (mean rho/3 over the inlet face cells minus over the outlet
 * face cells), inlet mass flow (sum rho u_x), and the flow of every outlet
 * region (sum rho u_x over its cells in ascending cell order). */
void ora3_observables(const ora3_params* p, const uint8_t* solid, const double* rho, const double* ux,
                      const int32_t* ids, int32_t n_out, double* dp, double* m_in, double* m_out) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  double si = 0, so = 0, ni = 0, no = 0, mi = 0;
  for (int j = 0; j < n_out; ++j) m_out[j] = 0.0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      size_t a = cell3(p, 0, y, z), b = cell3(p, nx - 1, y, z);
      if (!solid[a]) {
        si += rho[a] / 3.0;
        ni += 1.0;
        mi += rho[a] * ux[a];
      }
      if (!solid[b]) {
        so += rho[b] / 3.0;
        no += 1.0;
        m_out[ids[(size_t)z * ny + y]] += rho[b] * ux[b];
      }
    }
  *dp = si / ni - so / no;
  *m_in = mi;
}

/* Scores of the exchange (Sec. 2.2), on the 6-neighbourhood.  Interior
 * movable cells only: x in [2, nx-3], y in [1, ny-2], z in [1, nz-2].
 *   fluid cell with a solid face neighbour: q = 1/2 rho |u|^2 (Eq. 6);
 *   solid cell with a fluid face neighbour: sigma = sum over its fluid face
 *     neighbours (order +x, +y, -x, -y, +z, -z) of mu |u_t| / 0.5, where u_t
 *     is the neighbour's velocity along the shared face -- the magnitude of
 *     its two components other than the face normal (Eq. 5 carried to 3D;
 *     with u_z = 0 it is the 2D rule).
 * cand: 1 fluid candidate, 2 solid candidate, 0 otherwise. */
void ora3_scores(const ora3_params* p, const uint8_t* solid, const double* rho, const double* ux,
                 const double* uy, const double* uz, double mu, uint8_t* cand, double* score) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  static const int DX[6] = {1, 0, -1, 0, 0, 0}, DY[6] = {0, 1, 0, -1, 0, 0}, DZ[6] = {0, 0, 0, 0, 1, -1};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t c = cell3(p, x, y, z);
        cand[c] = 0;
        score[c] = 0.0;
        if (x < 2 || x > nx - 3 || y < 1 || y > ny - 2 || z < 1 || z > nz - 2) continue;
        if (!solid[c]) {
          int wall = 0;
          for (int d = 0; d < 6; ++d) wall |= solid[cell3(p, x + DX[d], y + DY[d], z + DZ[d])];
          if (wall) {
            cand[c] = 1;
            double s = ux[c] * ux[c] + uy[c] * uy[c] + uz[c] * uz[c];
            score[c] = 0.5 * rho[c] * s;
          }
        } else {
          int touch = 0;
          double sigma = 0.0;
          for (int d = 0; d < 6; ++d) {
            size_t nb = cell3(p, x + DX[d], y + DY[d], z + DZ[d]);
            if (solid[nb]) continue;
            touch = 1;
            double a, b;
            if (DX[d]) { a = uy[nb]; b = uz[nb]; }
            else if (DY[d]) { a = ux[nb]; b = uz[nb]; }
            else { a = ux[nb]; b = uy[nb]; }
            double ut = sqrt(a * a + b * b);
            sigma += (mu * ut) / 0.5;
          }
          if (touch) {
            cand[c] = 2;
            score[c] = sigma;
          }
        }
      }
}

/* The exchange of Sec. 2.3 steps 3-4 in 3D (choice by the 2D ora_select on
 * flat arrays); WARM / COLD re-initialisation.  Returns the fluid count. */
int64_t ora3_apply(const ora3_params* p, uint8_t* solid, double* f, const int32_t* fluid_idx,
                   const int32_t* solid_idx, int32_t n, int32_t reinit) {
  size_t cells = (size_t)p->nx * p->ny * p->nz;
  for (int k = 0; k < n; ++k) {
    size_t c = (size_t)fluid_idx[k];
    solid[c] = 1;
    for (int i = 0; i < 19; ++i) f[i * cells + c] = 0.0;
  }
  for (int k = 0; k < n; ++k) {
    size_t c = (size_t)solid_idx[k];
    solid[c] = 0;
    for (int i = 0; i < 19; ++i) f[i * cells + c] = W3[i] * p->rho0;
  }
  if (reinit == ORA3_REINIT_COLD)
    for (size_t c = 0; c < cells; ++c)
      if (!solid[c])
        for (int i = 0; i < 19; ++i) f[i * cells + c] = W3[i] * p->rho0;
  int64_t fluid = 0;
  for (size_t c = 0; c < cells; ++c) fluid += !solid[c];
  return fluid;
}
