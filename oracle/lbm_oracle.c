/*
 * lbm_oracle.c -- plain FP64 CPU statement of the LBM shape-optimisation method
 * of Wang, Fan & Luo, "Lattice Boltzmann method for shape optimization of
 * fluid distributor" (arXiv:1303.0107).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  It shares no code, header, table or helper with the CUDA
 * path, and nothing on the product path may call it: only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it.
 *
 * It is deliberately slow and literal:
 *   - two lattices (post-collision state in, next post-collision state out),
 *     pull streaming, every cell visited, solid cells skipped;
 *   - double precision, built with -ffp-contract=off so that no multiply-add
 *     is fused and the results are the same on every host;
 *   - every sum runs in ascending index order.
 *
 * Method passages followed (section / equation of the paper):
 *   Sec. 2.1, Eq. 1 .......... D2Q9 velocity set, lattice BGK update
 *   Sec. 2.1, Eq. 2 (f^eq) ... second-order equilibrium, weights, c_s
 *   Sec. 2.1, Eq. 2 (moments)  density and momentum
 *   Sec. 2.1, Eq. 4 .......... p = rho c_s^2
 *   Sec. 2.2, Eq. 5, Eq. 6 ... viscous stress on solid cells, dynamic pressure
 *                              on fluid cells
 *   Sec. 2.2 / 2.3 step 3 .... equal-count fluid<->solid exchange
 *   Sec. 2.3 step 4 .......... re-initialisation for the new shape
 *   Sec. 3.3 ................. bounce-back walls, parabolic inlet, Neumann
 *                              outlet, equilibrium initial state
 *   Sec. 4.2, Eq. 9-11 ....... flow-rate ratio, maldistribution factor
 * Readings where the paper is silent or garbled are stated next to the code
 * they decide, and listed in the design notes of the repository.
 *
 * Layout: populations f[i*ny*nx + y*nx + x], i = 0..8; cell arrays y*nx + x;
 * solid[] holds 1 for a solid cell, 0 for a fluid cell.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- Sec. 2.1: the D2Q9 lattice ------------------------------------------
 * c_0 = 0; c_1..c_4 = (cos((i-1)pi/2), sin((i-1)pi/2)) = E, N, W, S.
 * The printed diagonal formula gives axis vectors of length sqrt(2); it is
 * read as the standard diagonals c_5..c_8 = NE, NW, SW, SE (angle
 * (i-5)pi/2 + pi/4, length sqrt(2)).                                          */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* index of the direction opposite to i: c_OPP[i] = -c_i */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* direction with the y component reversed (reflection in a plane y = const) */
static const int MIR[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
/* weights: 4/9 rest, 1/9 axis, 1/36 diagonal; c_s = sqrt(3)/3 */
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

enum { ORA_OUT_CONST_RHO = 0, ORA_OUT_NEUMANN = 1 };
enum { ORA_PORTS_REGULARIZED = 0, ORA_PORTS_ZOU_HE = 1 };
enum { ORA_REINIT_WARM = 0, ORA_REINIT_COLD = 1 };
enum { ORA_COLLIDE_BGK = 0, ORA_COLLIDE_REGULARIZED = 1, ORA_COLLIDE_SMAGORINSKY = 2 };
enum { ORA_OK = 0, ORA_ERR_ARG = 1, ORA_ERR_GEOMETRY = 2, ORA_ERR_DIVERGED = 5 };

typedef struct {
  int32_t nx, ny;      /* lattice size; x along the flow, y across            */
  double tau;          /* relaxation time of Eq. 1; nu = (tau - 1/2)/3         */
  double rho0;         /* reference density: initial state and outlet density */
  double u_max;        /* centre-line speed of the parabolic inlet profile    */
  int32_t outlet_rule; /* ORA_OUT_CONST_RHO or ORA_OUT_NEUMANN                */
  int32_t periodic;    /* 1: wrap streaming in x and y, no ports (a check of
                          the bulk scheme only; never used for distributors)  */
  int32_t port_scheme; /* ORA_PORTS_REGULARIZED or ORA_PORTS_ZOU_HE: how the
                          velocity inlet and the constant-density outlet are
                          imposed                                            */
  int32_t guard;       /* 1: a fluid cell may turn solid only if it is a
                          simple cell of the fluid region (see ora_simple)  */
  int32_t collision;   /* ORA_COLLIDE_*: how the collision of Eq. 1 relaxes */
  int32_t mirror;      /* 1: a symmetry plane lies half a cell below row 0
                          (Sec. 3.3 computes half of the domain): row 0 may
                          be fluid, and what streams in across the plane is
                          the mirror image of what row 0 sends out          */
  double c_smag;       /* Smagorinsky constant (ORA_COLLIDE_SMAGORINSKY)     */
} ora_params;

/* Host threads of the time steps (OpenMP over rows; 0 or less: the
 * default).  Returns the number in force.  The results do not depend on it:
 * every cell is computed by one thread from the previous lattice. */
int32_t ora_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Export the lattice tables so that tests can check them against the
 * closed forms of Sec. 2.1. */
void ora_lattice(int32_t* cx, int32_t* cy, int32_t* opp, double* w, double* cs2) {
  for (int i = 0; i < 9; ++i) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    opp[i] = OPP[i];
    w[i] = W[i];
  }
  *cs2 = CS2;
}

/* Second-order equilibrium (the unnumbered equation after Eq. 1, rendered as
 * Eq. 2).  Its printed second-order term has a misplaced bracket; it is read as
 * the standard (c_i.u)^2 / (2 c_s^4).                                        */
double ora_feq(int32_t i, double rho, double ux, double uy) {
  double cu = CX[i] * ux + CY[i] * uy;
  double uu = ux * ux + uy * uy;
  return W[i] * rho * (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* ---- Sec. 3.3: ports --------------------------------------------------------
 * Inlet cells are the fluid cells of column x = 0, outlet cells the fluid cells
 * of column x = nx-1.  Each maximal run of consecutive fluid rows on a port
 * column is one inlet or one outlet.                                          */

/* Parabolic velocity profile imposed at every inlet run (Sec. 3.3): across a
 * run of W rows starting at y_lo, u_x = 4 u_max s (1 - s) with the cell centre
 * s = (y - y_lo + 1/2) / W; zero on rows that are not inlet cells.
 * Returns the number of inlet runs.                                            */
int32_t ora_inlet_profile(const ora_params* p, const uint8_t* solid, double* u_in) {
  int nx = p->nx, ny = p->ny, runs = 0;
  for (int y = 0; y < ny; ++y) u_in[y] = 0.0;
  int y = 0;
  while (y < ny) {
    if (solid[y * nx + 0]) { ++y; continue; }
    int y_lo = y;
    while (y < ny && !solid[y * nx + 0]) ++y;
    int width = y - y_lo;
    /* a run that touches the symmetry plane is half of a run twice as wide,
       centred on the plane: rows -width .. width-1 of the whole domain */
    int lo = y_lo, w = width;
    if (p->mirror && y_lo == 0) {
      lo = -width;
      w = 2 * width;
    }
    for (int yy = y_lo; yy < y; ++yy) {
      double s = ((double)(yy - lo) + 0.5) / (double)w;
      u_in[yy] = 4.0 * p->u_max * s * (1.0 - s);
    }
    ++runs;
  }
  return runs;
}

/* Outlet number of every row of column nx-1 (-1 where the cell is solid);
 * runs are numbered from y = 0 upward.  Returns the number of outlets.       */
int32_t ora_outlet_ids(const ora_params* p, const uint8_t* solid, int32_t* ids) {
  int nx = p->nx, ny = p->ny, n = 0;
  for (int y = 0; y < ny; ++y) {
    if (solid[y * nx + nx - 1]) { ids[y] = -1; continue; }
    if (y == 0 || solid[(y - 1) * nx + nx - 1]) ++n;
    ids[y] = n - 1;
  }
  return n;
}

/* Geometry accepted by the method as built here: rows 0 and ny-1 solid (the
 * frame), every inlet cell (0,y) backed by a fluid (1,y), every outlet cell
 * (nx-1,y) backed by a fluid (nx-2,y).                                       */
int32_t ora_check_geometry(const ora_params* p, const uint8_t* solid) {
  int nx = p->nx, ny = p->ny;
  if (nx < 4 || ny < 3) return ORA_ERR_ARG;
  if (p->periodic) return ORA_OK;
  for (int x = 0; x < nx; ++x)
    if ((!p->mirror && !solid[x]) || !solid[(ny - 1) * nx + x]) return ORA_ERR_GEOMETRY;
  for (int y = 0; y < ny; ++y) {
    if (!solid[y * nx] && solid[y * nx + 1]) return ORA_ERR_GEOMETRY;
    if (!solid[y * nx + nx - 1] && solid[y * nx + nx - 2]) return ORA_ERR_GEOMETRY;
  }
  return ORA_OK;
}

/* Initial condition (Sec. 3.3): the equilibrium of rho0 at rest on every fluid
 * cell, i.e. f_i = w_i rho0.  Solid cells hold no state (zeros).  The array
 * is the post-collision state that the first step streams.                   */
void ora_init(const ora_params* p, const uint8_t* solid, double* f) {
  size_t n = (size_t)p->nx * p->ny;
  for (int i = 0; i < 9; ++i)
    for (size_t c = 0; c < n; ++c) f[i * n + c] = solid[c] ? 0.0 : ora_feq(i, p->rho0, 0.0, 0.0);
}

/* Initial condition with a given macroscopic state on fluid cells (used by the
 * mass-conservation and shear-wave checks): f_i = f_i^eq(rho, u).           */
void ora_init_state(const ora_params* p, const uint8_t* solid, const double* rho,
                    const double* ux, const double* uy, double* f) {
  size_t n = (size_t)p->nx * p->ny;
  for (int i = 0; i < 9; ++i)
    for (size_t c = 0; c < n; ++c)
      f[i * n + c] = solid[c] ? 0.0 : ora_feq(i, rho[c], ux[c], uy[c]);
}

/* Streaming of direction i into fluid cell (x, y) from the post-collision
 * state: the population leaving the upstream cell x - c_i (pull form of the
 * left-hand side of Eq. 1).  Where the upstream cell is solid, the population
 * this cell sent towards that wall returns reversed: halfway bounce-back, the
 * wall half a cell away (Sec. 3.3; the same half-cell distance as Eq. 5).
 * Returns 0 when the upstream position lies outside the lattice (a port: the
 * population is unknown and the port rule supplies it).                      */
static int pull(const ora_params* p, const uint8_t* solid, const double* fp, int i, int x, int y,
                double* out) {
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
  int sx = x - CX[i], sy = y - CY[i];
  if (p->periodic) {
    sx = (sx + nx) % nx;
    sy = (sy + ny) % ny;
  } else if (p->mirror && sy == -1 && sx >= 0 && sx < nx) {
    /* the ghost row below the symmetry plane is the mirror image of row 0:
       a solid image reflects as a wall (halfway bounce-back), a fluid one
       sends the reflected population of its original cell */
    size_t src = (size_t)sx, here = (size_t)y * nx + x;
    if (solid[src])
      *out = fp[OPP[i] * n + here];
    else
      *out = fp[MIR[i] * n + src];
    return 1;
  } else if (sx < 0 || sx >= nx || sy < 0 || sy >= ny) {
    return 0;
  }
  size_t src = (size_t)sy * nx + sx, here = (size_t)y * nx + x;
  if (solid[src])
    *out = fp[OPP[i] * n + here];
  else
    *out = fp[i * n + src];
  return 1;
}

/* Regularised populations of a port cell with moments (rho, ux, uy):
 * f_i = f_i^eq + w_i / (2 c_s^4) * (Q_i,xx Pi_xx + Q_i,yy Pi_yy + 2 Q_i,xy Pi_xy),
 * Pi^neq = sum_i c_i c_i (f_i - f_i^eq), Q_i = c_i c_i - c_s^2 I.           */
static void regularize(double* f, double rho, double ux, double uy) {
  double pxx = 0.0, pyy = 0.0, pxy = 0.0;
  for (int i = 0; i < 9; ++i) {
    double fneq = f[i] - ora_feq(i, rho, ux, uy);
    pxx += CX[i] * CX[i] * fneq;
    pyy += CY[i] * CY[i] * fneq;
    pxy += CX[i] * CY[i] * fneq;
  }
  for (int i = 0; i < 9; ++i) {
    double qxx = CX[i] * CX[i] - CS2, qyy = CY[i] * CY[i] - CS2, qxy = CX[i] * CY[i];
    f[i] = ora_feq(i, rho, ux, uy) + W[i] / (2.0 * CS2 * CS2) * (qxx * pxx + qyy * pyy + 2.0 * qxy * pxy);
  }
}

/* Second moment of the non-equilibrium populations, Pi = sum_i c_i c_i (f_i - f_i^eq). */
static void pi_neq(const double* f, double rho, double ux, double uy, double* pxx, double* pyy, double* pxy) {
  *pxx = *pyy = *pxy = 0.0;
  for (int i = 0; i < 9; ++i) {
    double fneq = f[i] - ora_feq(i, rho, ux, uy);
    *pxx += CX[i] * CX[i] * fneq;
    *pyy += CY[i] * CY[i] * fneq;
    *pxy += CX[i] * CY[i] * fneq;
  }
}

/* Relaxation time of the Smagorinsky model (large-eddy closure; the paper
 * names LES as a way to higher Reynolds numbers).  The eddy viscosity is
 * nu_t = (C delta)^2 |S| with delta = 1 and |S| = sqrt(2 S:S); in the lattice
 * the strain rate follows from the non-equilibrium stress,
 * S = -Pi / (2 rho c_s^2 tau_eff).  With tau_eff = tau + nu_t / c_s^2 this is a
 * quadratic in tau_eff:
 *   tau_eff^2 - tau tau_eff - C^2 sqrt(2 Pi:Pi) / (2 rho c_s^4) = 0,
 * whose positive root is
 *   tau_eff = (tau + sqrt(tau^2 + 2 sqrt(2) C^2 sqrt(Pi:Pi) / (rho c_s^4))) / 2. */
static double smagorinsky_tau(double tau, double c, double rho, double pxx, double pyy, double pxy) {
  double pp = pxx * pxx + pyy * pyy + 2.0 * pxy * pxy;
  return 0.5 * (tau + sqrt(tau * tau + 2.0 * sqrt(2.0) * c * c * sqrt(pp) / (rho * CS2 * CS2)));
}

/* The collision of one cell with moments (rho, ux, uy), in place:
 *   BGK (Eq. 1):        f_i <- f_i - (f_i - f_i^eq) / tau;
 *   regularised:        f_i <- f_i^eq + (1 - 1/tau) f_i^(1), where f^(1) is the
 *                       non-equilibrium part projected on the second-order
 *                       Hermite tensor, w_i / (2 c_s^4) Q_i : Pi (Latt & Chopard);
 *   Smagorinsky:        BGK with the local tau_eff of smagorinsky_tau.      */
static void collide(const ora_params* p, double* f, double rho, double ux, double uy) {
  if (p->collision == ORA_COLLIDE_REGULARIZED) {
    double fr[9];
    for (int i = 0; i < 9; ++i) fr[i] = f[i];
    regularize(fr, rho, ux, uy);
    for (int i = 0; i < 9; ++i) {
      double eq = ora_feq(i, rho, ux, uy);
      f[i] = eq + (1.0 - 1.0 / p->tau) * (fr[i] - eq);
    }
    return;
  }
  double tau = p->tau;
  if (p->collision == ORA_COLLIDE_SMAGORINSKY) {
    double pxx, pyy, pxy;
    pi_neq(f, rho, ux, uy, &pxx, &pyy, &pxy);
    tau = smagorinsky_tau(p->tau, p->c_smag, rho, pxx, pyy, pxy);
  }
  for (int i = 0; i < 9; ++i) f[i] = f[i] - (f[i] - ora_feq(i, rho, ux, uy)) / tau;
}

double ora_smagorinsky_tau(double tau, double c, double rho, double pxx, double pyy, double pxy) {
  return smagorinsky_tau(tau, c, rho, pxx, pyy, pxy);
}

/* One time step of Eq. 1 over columns [x_begin, x_end) (the whole lattice when
 * x_begin = 0, x_end = nx): stream (pull, bounce-back), apply the port rules,
 * take the moments (Eq. 2), relax towards f^eq with 1/tau.  fp is the
 * post-collision state of the previous step, fn receives the new one.  rho, ux,
 * uy (optional, may be NULL) receive the moments used in this collision; solid
 * cells get zeros there.
 *
 * Port rules (Sec. 3.3 imposes a parabolic velocity at the inlet and a Neumann
 * condition at the outlet without naming the schemes):
 *   inlet (x = 0): velocity (u_in(y), 0).  Zou-He: the density follows from
 *                   mass and x-momentum of the known populations,
 *                   rho = (f0 + f2 + f4 + 2 (f3 + f6 + f7)) / (1 - u), and the
 *                   unknown f1, f5, f8 are rebuilt so that the cell carries
 *                   exactly (rho, rho u);
 *   outlet (x = nx-1), constant density: rho0 imposed, the velocity
 *                   u = -1 + (f0 + f2 + f4 + 2 (f1 + f5 + f8)) / rho0, u_y = 0,
 *                   and f3, f6, f7 rebuilt the same way;
 *   port scheme "regularized" (default): after that, every population of the
 *                   port cell is replaced by f^eq(rho, u) plus the projection
 *                   of its non-equilibrium part onto the second-order Hermite
 *                   tensor: f_i = f_i^eq + w_i/(2 c_s^4) Q_i : Pi^neq,
 *                   Q_i = c_i c_i - c_s^2 I, Pi^neq = sum_i c_i c_i (f_i - f_i^eq),
 *                   with the unknown non-equilibrium parts first taken from the
 *                   opposite directions (Latt & Chopard 2008).  Same (rho, u);
 *                   stable down to tau close to 1/2, where plain Zou-He on wide
 *                   ports is not;
 *   port scheme "Zou-He": the Zou-He populations as they are (Zou & He 1997);
 *   outlet, Neumann (zero gradient, the paper's rule): the unknown f3, f6, f7
 *                   are the streamed f3, f6, f7 of the cell (nx-2, y).
 * A population of a port cell whose upstream cell is a wall was already set by
 * bounce-back and is used as it is.                                          */
void ora_step_columns(const ora_params* p, const uint8_t* solid, const double* u_in,
                      const double* fp, double* fn, double* rho_out, double* ux_out,
                      double* uy_out, int32_t x_begin, int32_t x_end) {
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = x_begin; x < x_end; ++x) {
      size_t c = (size_t)y * nx + x;
      if (solid[c]) {
        for (int i = 0; i < 9; ++i) fn[i * n + c] = 0.0;
        if (rho_out) { rho_out[c] = 0.0; ux_out[c] = 0.0; uy_out[c] = 0.0; }
        continue;
      }
      double f[9];
      for (int i = 0; i < 9; ++i)
        if (!pull(p, solid, fp, i, x, y, &f[i])) f[i] = 0.0; /* set by a port rule below */

      if (!p->periodic && x == 0) {
        double ux = u_in[y];
        double rho = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 - ux);
        if (p->port_scheme == ORA_PORTS_ZOU_HE) {
          f[1] = f[3] + (2.0 / 3.0) * rho * ux;
          f[5] = f[7] - 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * ux;
          f[8] = f[6] + 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * ux;
        } else {
          for (int k = 0; k < 3; ++k) {
            static const int UNK[3] = {1, 5, 8};
            int i = UNK[k];
            f[i] = ora_feq(i, rho, ux, 0.0) + (f[OPP[i]] - ora_feq(OPP[i], rho, ux, 0.0));
          }
          regularize(f, rho, ux, 0.0);
        }
      } else if (!p->periodic && x == nx - 1) {
        if (p->outlet_rule == ORA_OUT_NEUMANN) {
          double g;
          pull(p, solid, fp, 3, nx - 2, y, &g); f[3] = g;
          pull(p, solid, fp, 6, nx - 2, y, &g); f[6] = g;
          pull(p, solid, fp, 7, nx - 2, y, &g); f[7] = g;
        } else {
          double rho = p->rho0;
          double ux = -1.0 + (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / rho;
          if (p->port_scheme == ORA_PORTS_ZOU_HE) {
            f[3] = f[1] - (2.0 / 3.0) * rho * ux;
            f[7] = f[5] + 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * ux;
            f[6] = f[8] - 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * ux;
          } else {
            for (int k = 0; k < 3; ++k) {
              static const int UNK[3] = {3, 6, 7};
              int i = UNK[k];
              f[i] = ora_feq(i, rho, ux, 0.0) + (f[OPP[i]] - ora_feq(OPP[i], rho, ux, 0.0));
            }
            regularize(f, rho, ux, 0.0);
          }
        }
      }

      /* Eq. 2: rho = sum_i f_i, rho u = sum_i c_i f_i */
      double rho = 0.0, jx = 0.0, jy = 0.0;
      for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
      }
      double ux = jx / rho, uy = jy / rho;
      collide(p, f, rho, ux, uy);
      for (int i = 0; i < 9; ++i) fn[i * n + c] = f[i];
      if (rho_out) { rho_out[c] = rho; ux_out[c] = ux; uy_out[c] = uy; }
    }
  }
}

void ora_step(const ora_params* p, const uint8_t* solid, const double* u_in, const double* fp,
              double* fn, double* rho, double* ux, double* uy) {
  ora_step_columns(p, solid, u_in, fp, fn, rho, ux, uy, 0, p->nx);
}

/* n_steps steps starting from the post-collision state f (updated in place;
 * work is a second lattice of the same size).  rho/ux/uy receive the moments
 * of the last step.  Returns ORA_ERR_DIVERGED if a non-finite density shows up. */
int32_t ora_run(const ora_params* p, const uint8_t* solid, const double* u_in, double* f,
                double* work, int64_t n_steps, double* rho, double* ux, double* uy) {
  size_t n = (size_t)p->nx * p->ny;
  double* a = f;
  double* b = work;
  for (int64_t t = 0; t < n_steps; ++t) {
    ora_step(p, solid, u_in, a, b, rho, ux, uy);
    double* tmp = a; a = b; b = tmp;
  }
  if (a != f) memcpy(f, a, sizeof(double) * 9 * n);
  for (size_t c = 0; c < n; ++c)
    if (!solid[c] && !isfinite(rho[c])) return ORA_ERR_DIVERGED;
  return ORA_OK;
}

/* ---- Observables ------------------------------------------------------------
 * Pressure drop (Sec. 2.3 step 5): the mean of p = rho c_s^2 (Eq. 4) over the
 * inlet cells minus its mean over all outlet cells.
 * Flow rates (Sec. 4.2, Eq. 9-11, per unit depth): m_in = sum of rho u_x over
 * the inlet cells, m_out[j] = sum of rho u_x over the cells of outlet j.     */
int32_t ora_observables(const ora_params* p, const uint8_t* solid, const double* rho,
                        const double* ux, const int32_t* outlet_ids, int32_t n_outlets,
                        double* dp, double* m_in, double* m_out) {
  int nx = p->nx, ny = p->ny;
  double sum_in = 0.0, sum_out = 0.0, min_ = 0.0;
  int cnt_in = 0, cnt_out = 0;
  for (int j = 0; j < n_outlets; ++j) m_out[j] = 0.0;
  for (int y = 0; y < ny; ++y) {
    size_t ci = (size_t)y * nx + 0, co = (size_t)y * nx + nx - 1;
    if (!solid[ci]) {
      sum_in += rho[ci] * CS2;
      min_ += rho[ci] * ux[ci];
      ++cnt_in;
    }
    if (!solid[co]) {
      sum_out += rho[co] * CS2;
      m_out[outlet_ids[y]] += rho[co] * ux[co];
      ++cnt_out;
    }
  }
  if (cnt_in == 0 || cnt_out == 0) return ORA_ERR_GEOMETRY;
  *dp = sum_in / cnt_in - sum_out / cnt_out;
  *m_in = min_;
  return isfinite(*dp) ? ORA_OK : ORA_ERR_DIVERGED;
}

/* Eq. 9-11: theta = m_max / m_min; D_g = sqrt(sum_i (m_i/m_ave - 1)^2 / (N-1))
 * with m_ave = (1/N) sum_i m_i.                                               */
void ora_uniformity(const double* m, int32_t n, double* theta, double* dg) {
  double mx = m[0], mn = m[0], sum = 0.0;
  for (int i = 0; i < n; ++i) {
    if (m[i] > mx) mx = m[i];
    if (m[i] < mn) mn = m[i];
    sum += m[i];
  }
  double ave = sum / n;
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    double d = m[i] / ave - 1.0;
    acc += d * d;
  }
  *theta = mx / mn;
  *dg = n > 1 ? sqrt(acc / (n - 1)) : 0.0;
}

/* Convergence residual: sum over fluid cells of |u - u_prev|_1 divided by the
 * sum of |u|_1 (both in ascending cell order).                               */
double ora_residual(const ora_params* p, const uint8_t* solid, const double* ux, const double* uy,
                    const double* ux_prev, const double* uy_prev) {
  size_t n = (size_t)p->nx * p->ny;
  double num = 0.0, den = 0.0;
  for (size_t c = 0; c < n; ++c) {
    if (solid[c]) continue;
    num += fabs(ux[c] - ux_prev[c]) + fabs(uy[c] - uy_prev[c]);
    den += fabs(ux[c]) + fabs(uy[c]);
  }
  return num / den;
}

/* ---- Sec. 2.2: the optimality criteria --------------------------------------
 * Interface and movable cells (the paper does not define them): 4-neighbours
 * E, N, W, S; a fluid cell with at least one solid 4-neighbour and a solid
 * cell with at least one fluid 4-neighbour are interface cells; columns
 * x < 2 and x > nx-3 and rows 0 and ny-1 never move, so the ports and the
 * frame keep their shape.
 *
 * Fluid cell (Eq. 6): q = 1/2 rho |u|^2, with its own rho and u.
 * Solid cell (Eq. 5): the wall shear of each fluid 4-neighbour n, across a half
 * cell: mu u_x(n) / 0.5 through a horizontal face (n above or below) and
 * mu u_y(n) / 0.5 through a vertical face (n left or right); the score sigma is
 * the sum of their magnitudes in the order E, N, W, S, with mu = rho0 nu and
 * nu = (tau - 1/2)/3.
 * cand[c] = 1 for an interface fluid cell, 2 for an interface solid cell,
 * 0 otherwise; score[c] holds q or sigma there and 0 elsewhere.              */
/* Connectivity guard (a reading of Sec. 2.3 step 3, which does not say
 * whether an exchange may cut the fluid region apart).  Fluid cells connect
 * through faces (4-neighbourhood), solid cells through faces and corners.
 * Interior cell (x, y) is "simple" when removing it from the fluid changes
 * neither count locally: its 4-connectivity number
 *   N4 = sum over k in {E, N, W, S} of  f_k (1 - f_k+1 f_k+2),
 * with f the fluid indicators of the eight neighbours taken counter-
 * clockwise E, NE, N, NW, W, SW, S, SE (and around again), equals 1.
 * N4 counts the fluid 4-neighbours that stay separated from each other
 * inside the 3 x 3 block once the cell is gone. */
int32_t ora_simple(const ora_params* p, const uint8_t* solid, int32_t x, int32_t y) {
  static const int DX[8] = {1, 1, 0, -1, -1, -1, 0, 1};
  static const int DY[8] = {0, 1, 1, 1, 0, -1, -1, -1};
  int f[10];
  for (int k = 0; k < 8; ++k) f[k] = !solid[(size_t)(y + DY[k]) * p->nx + (x + DX[k])];
  f[8] = f[0];
  f[9] = f[1];
  int n4 = 0;
  for (int k = 0; k < 8; k += 2) n4 += f[k] * (1 - f[k + 1] * f[k + 2]);
  return n4 == 1;
}

void ora_scores(const ora_params* p, const uint8_t* solid, const double* rho, const double* ux,
                const double* uy, double mu, uint8_t* cand, double* score) {
  int nx = p->nx, ny = p->ny;
  static const int NB[4] = {1, 2, 3, 4}; /* E, N, W, S */
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      cand[c] = 0;
      score[c] = 0.0;
      if (x < 2 || x > nx - 3 || y < 1 || y > ny - 2) continue;
      if (!solid[c]) {
        int touches_wall = 0;
        for (int k = 0; k < 4; ++k) {
          int i = NB[k];
          if (solid[(size_t)(y + CY[i]) * nx + (x + CX[i])]) touches_wall = 1;
        }
        if (touches_wall && (!p->guard || ora_simple(p, solid, x, y))) {
          cand[c] = 1;
          double s = ux[c] * ux[c] + uy[c] * uy[c];
          score[c] = 0.5 * rho[c] * s;
        }
      } else {
        int touches_fluid = 0;
        double sigma = 0.0;
        for (int k = 0; k < 4; ++k) {
          int i = NB[k];
          size_t nb = (size_t)(y + CY[i]) * nx + (x + CX[i]);
          if (solid[nb]) continue;
          touches_fluid = 1;
          /* E/W neighbours share a vertical face: tangential velocity u_y;
             N/S neighbours share a horizontal face: tangential velocity u_x */
          double ut = (CX[i] != 0) ? uy[nb] : ux[nb];
          sigma += (mu * fabs(ut)) / 0.5;
        }
        if (touches_fluid) {
          cand[c] = 2;
          score[c] = sigma;
        }
      }
    }
  }
}

typedef struct {
  double key;
  int32_t idx;
} ora_cand;

/* fluid candidates: lowest q first, ties to the smaller index */
static int cmp_fluid(const void* a, const void* b) {
  const ora_cand* u = (const ora_cand*)a;
  const ora_cand* v = (const ora_cand*)b;
  if (u->key < v->key) return -1;
  if (u->key > v->key) return 1;
  return (u->idx > v->idx) - (u->idx < v->idx);
}
/* solid candidates: largest sigma first, ties to the smaller index */
static int cmp_solid(const void* a, const void* b) {
  const ora_cand* u = (const ora_cand*)a;
  const ora_cand* v = (const ora_cand*)b;
  if (u->key > v->key) return -1;
  if (u->key < v->key) return 1;
  return (u->idx > v->idx) - (u->idx < v->idx);
}
static int cmp_int(const void* a, const void* b) {
  int32_t u = *(const int32_t*)a, v = *(const int32_t*)b;
  return (u > v) - (u < v);
}

/* Sec. 2.3 step 3: among the interface cells pick the n fluid cells with the
 * lowest dynamic pressure and the n solid cells with the largest viscous
 * stress, n = min(n_swap, #fluid candidates, #solid candidates).  All picks
 * come from the same field.  The chosen indices are returned sorted
 * ascending.  Returns ORA_ERR_DIVERGED if a score is not a number.          */
int32_t ora_select(const ora_params* p, const uint8_t* cand, const double* score, int32_t n_swap,
                   int32_t* fluid_idx, int32_t* solid_idx, int32_t* n_out) {
  size_t n = (size_t)p->nx * p->ny;
  size_t nf = 0, ns = 0;
  for (size_t c = 0; c < n; ++c) {
    if (cand[c] && isnan(score[c])) return ORA_ERR_DIVERGED;
    if (cand[c] == 1) ++nf;
    if (cand[c] == 2) ++ns;
  }
  ora_cand* F = (ora_cand*)malloc(sizeof(ora_cand) * (nf ? nf : 1));
  ora_cand* S = (ora_cand*)malloc(sizeof(ora_cand) * (ns ? ns : 1));
  size_t a = 0, b = 0;
  for (size_t c = 0; c < n; ++c) {
    if (cand[c] == 1) { F[a].key = score[c]; F[a].idx = (int32_t)c; ++a; }
    if (cand[c] == 2) { S[b].key = score[c]; S[b].idx = (int32_t)c; ++b; }
  }
  qsort(F, nf, sizeof(ora_cand), cmp_fluid);
  qsort(S, ns, sizeof(ora_cand), cmp_solid);
  size_t m = (size_t)(n_swap > 0 ? n_swap : 0);
  if (m > nf) m = nf;
  if (m > ns) m = ns;
  for (size_t k = 0; k < m; ++k) {
    fluid_idx[k] = F[k].idx;
    solid_idx[k] = S[k].idx;
  }
  qsort(fluid_idx, m, sizeof(int32_t), cmp_int);
  qsort(solid_idx, m, sizeof(int32_t), cmp_int);
  *n_out = (int32_t)m;
  free(F);
  free(S);
  return ORA_OK;
}

/* Sec. 2.3 steps 3-4: exchange the chosen cells (fluid -> solid, solid ->
 * fluid) at once, then re-initialise.  WARM keeps the state of every fluid
 * cell that stays fluid and puts the new fluid cells at the equilibrium of
 * rho0 at rest; COLD puts every fluid cell there (the initial state of
 * Sec. 3.3).  Returns the fluid-cell count after the exchange.               */
int64_t ora_apply(const ora_params* p, uint8_t* solid, double* f, const int32_t* fluid_idx,
                  const int32_t* solid_idx, int32_t n, int32_t reinit) {
  size_t cells = (size_t)p->nx * p->ny;
  for (int k = 0; k < n; ++k) {
    size_t c = (size_t)fluid_idx[k];
    solid[c] = 1;
    for (int i = 0; i < 9; ++i) f[i * cells + c] = 0.0;
  }
  for (int k = 0; k < n; ++k) {
    size_t c = (size_t)solid_idx[k];
    solid[c] = 0;
    for (int i = 0; i < 9; ++i) f[i * cells + c] = ora_feq(i, p->rho0, 0.0, 0.0);
  }
  if (reinit == ORA_REINIT_COLD) ora_init(p, solid, f);
  int64_t fluid = 0;
  for (size_t c = 0; c < cells; ++c) fluid += solid[c] ? 0 : 1;
  return fluid;
}
