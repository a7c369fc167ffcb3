/*
 * fv_oracle.c -- plain FP64 CPU oracle for the first-order finite-volume
 * time step of Essadki, Jung, Larat, Pelletier, Perrier, "A task-driven
 * implementation of a simple numerical solver for hyperbolic conservation
 * laws" (arXiv:1701.05431).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; it is used by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * It follows the paper's steps in the paper's order, in FP64, with no
 * blocking, fusion or reordering:
 *   Sec. 2.2.1, Eq. (CFL_cond)   checkTimeStep: largest |eigenvalue|, dt
 *   Sec. 4.1.2, Sec. 4.2         copyOverlaps into ovlpE/N/W/S
 *   Sec. 2.2.1, Eq. (VF_scheme)  Lax-Friedrichs face fluxes, residuals
 *   Sec. 4.1.1, Eq. (update)     u += RHS
 *   Sec. 2.2.2, Eq. (SourceTerm) split forward-Euler source step
 *   Sec. 6.1-6.2                 evaporating-spray moments, source terms and
 *                                maximum-entropy reconstruction of n(S)
 *
 * Two modes compute the same numbers:
 *   literal: the paper's tasks per subdomain with uLoc, RHS and the four
 *            overlap strips of Sec. 4.1.2 (balanced NPartX x NPartY split of
 *            Sec. 3.2);
 *   plain:   one global array with a ghost layer and one flux per face.
 * Each cell's residual is the same expression of its four face fluxes in
 * both modes, so the two agree bit for bit.
 *
 * Readings taken where the paper is silent or garbled:
 *   - residual sign follows Eq. (VF_scheme): RHS = -dt/dx (Fe - Fw)
 *     - dt/dy (Fn - Fs) (Eq. (RHSFilling) prints the opposite sign);
 *   - the flux is the local Lax-Friedrichs (Rusanov) flux, sigma evaluated
 *     per face from W_L and W_R along that face's normal;
 *   - the largest eigenvalue in Eq. (CFL_cond) is taken over the two axis
 *     normals n=(1,0) and n=(0,1);
 *   - adaptive mode (cfl > 0, fixed_dt <= 0): dt_n = cfl*min(dx,dy)/lmax(W^n);
 *     paper mode (fixed_dt > 0): dt is fixed and only checked against
 *     Eq. (CFL_cond) at the start of every step;
 *   - boundaries: periodic = wrapped neighbour, transmissive = copy of the
 *     cell's own border value, Dirichlet = prescribed state; corners unused;
 *   - the spray source uses the maximum-entropy density
 *     n(S) = exp(-sum_k lam_k S^(k/2)), k = 0..3, found by damped Newton on
 *     the convex dual with Q-point Gauss-Legendre quadrature in x = sqrt(S).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OFV_ADVECTION = 0, OFV_EULER = 1, OFV_SPRAY = 2 };
enum { OFV_PERIODIC = 0, OFV_TRANSMISSIVE = 1, OFV_DIRICHLET = 2 };
enum { OFV_E = 0, OFV_N = 1, OFV_W = 2, OFV_S = 3 };
enum {
  OFV_OK = 0,
  OFV_ERR_ARG = 1,
  OFV_ERR_CFL = 4,
  OFV_ERR_NONPHYSICAL = 5
};
#define OFV_MAXVAR 8
#define OFV_MAXQ 128

/* Problem statement of Sec. 2.1-2.2: domain [xmin,xmax]x[ymin,ymax], Nx x Ny
 * cells, NPartX x NPartY subdomains, the system (nVar, flux, source),
 * boundary conditions (E, N, W, S) and the time-step policy.
 *   advection: params[0] = a_x, params[1] = a_y   (F = a u)
 *   euler:     params[0] = gamma                  (Eq. (Euler), Sec. 5)
 *   spray:     params[0] = K (evaporation rate), params[1] = theta (drag time,
 *              <= 0 disables drag), params[2] = gas field (0: u_g = 0,
 *              1: Taylor-Green), params[3] = Q quadrature nodes (0 -> 32),
 *              params[4] = Newton tolerance (0 -> 1e-13)  (Eq. (Essadki))   */
typedef struct {
  int nx, ny, npart_x, npart_y;
  double xmin, xmax, ymin, ymax;
  int system;
  int bc[4];
  double bc_state[4][OFV_MAXVAR];
  double cfl, fixed_dt;
  double params[8];
} ofv_problem;

int ofv_nvar(int system) {
  switch (system) {
    case OFV_ADVECTION: return 1;
    case OFV_EULER: return 4;
    case OFV_SPRAY: return 6;
    default: return 0;
  }
}

/* ------------------------------------------------------------------------ */
/* Physical flux F(W).n and the largest |eigenvalue| along n.               */
/* ------------------------------------------------------------------------ */

/* Euler, Eq. (Euler): W = (rho, rho u, rho v, rho E),
 * F.n = (rho un, rho u un + p nx, rho v un + p ny, rho un H),
 * p = (gamma-1) rho (E - (u^2+v^2)/2), H = E + p/rho, c^2 = gamma p / rho,
 * eigenvalues un - c, un, un, un + c. */
static void euler_flux(double gamma, const double *W, double nx_, double ny_,
                       double *F, double *s) {
  double rho = W[0];
  double u = W[1] / rho;
  double v = W[2] / rho;
  double E = W[3] / rho;
  double p = (gamma - 1.0) * rho * (E - (u * u + v * v) / 2.0);
  double H = E + p / rho;
  double un = u * nx_ + v * ny_;
  double c = sqrt(gamma * p / rho);
  F[0] = rho * un;
  F[1] = rho * u * un + p * nx_;
  F[2] = rho * v * un + p * ny_;
  F[3] = rho * un * H;
  *s = fabs(un) + c;
}

/* Scalar linear advection: F.n = (a.n) u, one eigenvalue a.n. */
static void advection_flux(const double *a, const double *W, double nx_,
                           double ny_, double *F, double *s) {
  double an = a[0] * nx_ + a[1] * ny_;
  F[0] = an * W[0];
  *s = fabs(an);
}

/* Spray moments, Eq. (Essadki): W = (m0, m1/2, m1, m3/2, m1 u, m1 v), all
 * transported by u = (m1 u)/m1: F.n = W (u.n), every eigenvalue equals u.n. */
static void spray_flux(const double *W, double nx_, double ny_, double *F,
                       double *s) {
  double u = W[4] / W[2];
  double v = W[5] / W[2];
  double un = u * nx_ + v * ny_;
  for (int k = 0; k < 6; ++k) F[k] = W[k] * un;
  *s = fabs(un);
}

static void phys_flux(const ofv_problem *P, const double *W, double nx_,
                      double ny_, double *F, double *s) {
  switch (P->system) {
    case OFV_ADVECTION: advection_flux(P->params, W, nx_, ny_, F, s); break;
    case OFV_EULER: euler_flux(P->params[0], W, nx_, ny_, F, s); break;
    default: spray_flux(W, nx_, ny_, F, s); break;
  }
}

/* Largest |eigenvalue| of one cell over the two axis normals, the quantity
 * maximised in Eq. (CFL_cond) and by the checkTimeStep task (Sec. 4.2). */
static double cell_lambda(const ofv_problem *P, const double *W) {
  double F[OFV_MAXVAR], sx, sy;
  phys_flux(P, W, 1.0, 0.0, F, &sx);
  phys_flux(P, W, 0.0, 1.0, F, &sy);
  return sx > sy ? sx : sy;
}

/* Local Lax-Friedrichs flux of Sec. 2.2.1:
 * F~(WL, WR, n) = (F(WL).n + F(WR).n)/2 - sigma/2 (WR - WL),
 * sigma = max_p max(|lambda_p(WL)|, |lambda_p(WR)|). */
static void lf_flux(const ofv_problem *P, int nvar, const double *WL,
                    const double *WR, double nx_, double ny_, double *Ft) {
  double FL[OFV_MAXVAR], FR[OFV_MAXVAR], sL, sR;
  phys_flux(P, WL, nx_, ny_, FL, &sL);
  phys_flux(P, WR, nx_, ny_, FR, &sR);
  double sigma = sL > sR ? sL : sR;
  for (int v = 0; v < nvar; ++v)
    Ft[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * sigma * (WR[v] - WL[v]);
}

/* Residual of one cell from its four face fluxes, Eq. (VF_scheme):
 * RHS = -(dt/dx)(Fe - Fw) - (dt/dy)(Fn - Fs).  Both modes call this. */
static void cell_rhs(int nvar, double lx, double ly, const double *Fe,
                     const double *Fw, const double *Fn, const double *Fs,
                     double *R) {
  for (int v = 0; v < nvar; ++v)
    R[v] = -(lx * (Fe[v] - Fw[v])) - (ly * (Fn[v] - Fs[v]));
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre quadrature on [0,1] and the maximum-entropy reconstruction */
/* (Sec. 6.2).                                                              */
/* ------------------------------------------------------------------------ */

/* Nodes and weights of the Q-point Gauss-Legendre rule on [0,1].  The nodes
 * are the roots of the Legendre polynomial P_Q, found by Newton's method on
 * the three-term recurrence (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}; the
 * weights are 2 / ((1 - t^2) P_Q'(t)^2) on [-1,1], halved for [0,1]. */
int ofv_gauss_legendre(int Q, double *x, double *w) {
  if (Q < 1 || Q > OFV_MAXQ) return OFV_ERR_ARG;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < Q; ++i) {
    double t = cos(pi * (i + 0.75) / (Q + 0.5));
    double dP = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < Q; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      /* P_Q = p1, P_{Q-1} = p0; P_Q' = Q (t P_Q - P_{Q-1}) / (t^2 - 1) */
      if (Q == 1) { p0 = 1.0; }
      dP = Q * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < Q; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (Q == 1) { p0 = 1.0; }
      dP = Q * (t * p1 - p0) / (t * t - 1.0);
    }
    double wt = 2.0 / ((1.0 - t * t) * dP * dP);
    /* map t in [-1,1] to [0,1], ascending order */
    x[Q - 1 - i] = 0.5 * (t + 1.0);
    w[Q - 1 - i] = 0.5 * wt;
  }
  return OFV_OK;
}

/* Moments M_k = int_0^1 S^(k/2) n(S) dS, k = 0..6, of
 * n(S) = exp(-(lam0 + lam1 S^(1/2) + lam2 S + lam3 S^(3/2))), computed in
 * x = sqrt(S) (dS = 2x dx) with the quadrature rule (xq, wq). */
static void maxent_moments(int Q, const double *xq, const double *wq,
                           const double *lam, double *M) {
  for (int k = 0; k < 7; ++k) M[k] = 0.0;
  for (int q = 0; q < Q; ++q) {
    double x = xq[q];
    double n = exp(-(lam[0] + lam[1] * x + lam[2] * x * x +
                     lam[3] * x * x * x));
    double f = wq[q] * 2.0 * x * n;
    double xk = 1.0;
    for (int k = 0; k < 7; ++k) {
      M[k] += f * xk;
      xk *= x;
    }
  }
}

/* Dual objective Phi(lam) = int n dS + sum_k lam_k m_k; convex, and its
 * minimiser matches the moments m_k. */
static double maxent_dual(int Q, const double *xq, const double *wq,
                          const double *lam, const double *m) {
  double M[7];
  maxent_moments(Q, xq, wq, lam, M);
  return M[0] + lam[0] * m[0] + lam[1] * m[1] + lam[2] * m[2] + lam[3] * m[3];
}

/* Solve the 4x4 symmetric positive definite system H d = r by Cholesky. */
static int spd_solve4(const double H[4][4], const double *r, double *d) {
  double L[4][4] = {{0}};
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = H[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0.0)) return OFV_ERR_NONPHYSICAL;
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  }
  double y[4];
  for (int i = 0; i < 4; ++i) {
    double s = r[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = 3; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 4; ++k) s -= L[k][i] * d[k];
    d[i] = s / L[i][i];
  }
  return OFV_OK;
}

/* Maximum-entropy reconstruction of Sec. 6.2: find lam such that
 * int S^(k/2) exp(-sum_j lam_j S^(j/2)) dS = m_k for k = 0..3, then return
 * n(S=0) = exp(-lam0) and m_{-1/2} = int S^(-1/2) n dS = 2 int_0^1 n(x^2) dx.
 * Damped Newton on the convex dual from lam = (-ln m0, 0, 0, 0) (the
 * constant density with the right m0); Hessian H_ij = M_{i+j}.  Stops when
 * every moment residual |M_k - m_k| <= tol * m_k. */
int ofv_maxent(const double *m, int Q, const double *xq, const double *wq,
               double tol, double *lam, double *n0, double *m_mhalf,
               int *iters) {
  if (!(m[0] > 0.0)) return OFV_ERR_NONPHYSICAL;
  lam[0] = -log(m[0]);
  lam[1] = lam[2] = lam[3] = 0.0;
  int it = 0, ok = 0;
  for (it = 0; it < 100; ++it) {
    double M[7];
    maxent_moments(Q, xq, wq, lam, M);
    double r[4], worst = 0.0;
    for (int k = 0; k < 4; ++k) {
      r[k] = M[k] - m[k];
      double rel = fabs(r[k]) / m[k];
      if (rel > worst) worst = rel;
    }
    if (worst <= tol) { ok = 1; break; }
    double H[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) H[i][j] = M[i + j];
    double d[4];
    if (spd_solve4(H, r, d) != OFV_OK) return OFV_ERR_NONPHYSICAL;
    /* Newton direction lam + d; gradient of Phi is m - M = -r. */
    double phi0 = M[0] + lam[0] * m[0] + lam[1] * m[1] + lam[2] * m[2] +
                  lam[3] * m[3];
    double slope = -(r[0] * d[0] + r[1] * d[1] + r[2] * d[2] + r[3] * d[3]);
    double alpha = 1.0;
    double trial[4];
    for (int k = 0; k < 4; ++k) trial[k] = lam[k] + d[k];
    /* Near the solution (every relative residual below 1e-3) Newton is in
     * its quadratic region and takes full steps: the dual's decrease is
     * then below its round-off and cannot steer a line search.  Farther
     * out, halve the step until the Armijo condition holds (with an
     * allowance of a few ulps of Phi). */
    if (worst >= 1e-3) {
      for (int ls = 0; ls < 60; ++ls) {
        for (int k = 0; k < 4; ++k) trial[k] = lam[k] + alpha * d[k];
        double phi = maxent_dual(Q, xq, wq, trial, m);
        if (phi <= phi0 + 1e-4 * alpha * slope + 4e-16 * fabs(phi0)) break;
        alpha *= 0.5;
      }
    }
    for (int k = 0; k < 4; ++k) lam[k] = trial[k];
  }
  if (iters) *iters = it;
  if (!ok) {
    /* accept a result that stalled at round-off level */
    double M[7];
    maxent_moments(Q, xq, wq, lam, M);
    for (int k = 0; k < 4; ++k)
      if (fabs(M[k] - m[k]) > 1e-10 * m[k]) return OFV_ERR_NONPHYSICAL;
  }
  *n0 = exp(-lam[0]);
  double s = 0.0;
  for (int q = 0; q < Q; ++q) {
    double x = xq[q];
    s += wq[q] * 2.0 *
         exp(-(lam[0] + lam[1] * x + lam[2] * x * x + lam[3] * x * x * x));
  }
  *m_mhalf = s;
  return OFV_OK;
}

/* Interior of the moment space of measures on [0,1] for (c0, c1, c2, c3):
 * the Hankel determinants of the measure and of its products with x and
 * 1 - x are positive. */
int ofv_realizable(const double *c) {
  if (!(c[0] > 0.0)) return 0;
  if (!(c[1] > 0.0)) return 0;
  if (!(c[0] - c[1] > 0.0)) return 0;
  if (!(c[0] * c[2] - c[1] * c[1] > 0.0)) return 0;
  if (!(c[1] - c[2] > 0.0)) return 0;
  if (!(c[1] * c[3] - c[2] * c[2] > 0.0)) return 0;
  if (!((c[0] - c[1]) * (c[2] - c[3]) - (c[1] - c[2]) * (c[1] - c[2]) > 0.0))
    return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Source step, Eq. (SourceTerm) with the spray sources of Eq. (Essadki).   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int Q;
  double xq[OFV_MAXQ], wq[OFV_MAXQ];
  double tol;
} maxent_rule;

/* Gas velocity of the drag term at (x, y). */
static void gas_velocity(const ofv_problem *P, double x, double y, double *ug,
                         double *vg) {
  const double pi = 3.14159265358979323846;
  if ((int)P->params[2] == 1) {
    *ug = sin(2.0 * pi * x) * cos(2.0 * pi * y);
    *vg = -cos(2.0 * pi * x) * sin(2.0 * pi * y);
  } else {
    *ug = 0.0;
    *vg = 0.0;
  }
}

/* W <- W + dt S(W) for one spray cell centred at (x, y):
 *   d m0   = -K n(S=0)
 *   d m1/2 = -K/2 m_{-1/2}
 *   d m1   = -K m0
 *   d m3/2 = -3K/2 m1/2
 *   d m1 u = -K m0 u + m0 (u_g - u)/theta      (same for v). */
static int spray_source(const ofv_problem *P, const maxent_rule *R, double dt,
                        double x, double y, double *W) {
  double K = P->params[0], theta = P->params[1];
  double m[4] = {W[0], W[1], W[2], W[3]};
  if (!ofv_realizable(m)) return OFV_ERR_NONPHYSICAL;
  double lam[4], n0, mmh;
  int it;
  int st = ofv_maxent(m, R->Q, R->xq, R->wq, R->tol, lam, &n0, &mmh, &it);
  if (st != OFV_OK) return st;
  double u = W[4] / W[2], v = W[5] / W[2];
  double S[6];
  S[0] = -K * n0;
  S[1] = -K / 2.0 * mmh;
  S[2] = -K * m[0];
  S[3] = -3.0 * K / 2.0 * m[1];
  S[4] = -K * m[0] * u;
  S[5] = -K * m[0] * v;
  if (theta > 0.0) {
    double ug, vg;
    gas_velocity(P, x, y, &ug, &vg);
    S[4] += m[0] * (ug - u) / theta;
    S[5] += m[0] * (vg - v) / theta;
  }
  for (int k = 0; k < 6; ++k) W[k] = W[k] + dt * S[k];
  double c[4] = {W[0], W[1], W[2], W[3]};
  if (!ofv_realizable(c)) return OFV_ERR_NONPHYSICAL;
  return OFV_OK;
}

/* ------------------------------------------------------------------------ */
/* Boundary ghosts (corners are never needed by the 5-point stencil).       */
/* ------------------------------------------------------------------------ */

/* Ghost value beyond side `side` given the cell just inside (own) and the
 * cell that wraps around (wrap). */
static void ghost_value(const ofv_problem *P, int nvar, int side,
                        const double *own, const double *wrap, double *g) {
  switch (P->bc[side]) {
    case OFV_PERIODIC:
      for (int v = 0; v < nvar; ++v) g[v] = wrap[v];
      break;
    case OFV_TRANSMISSIVE:
      for (int v = 0; v < nvar; ++v) g[v] = own[v];
      break;
    default:
      for (int v = 0; v < nvar; ++v) g[v] = P->bc_state[side][v];
      break;
  }
}

/* ------------------------------------------------------------------------ */
/* Plain mode: one global SoA array W[v][j][i] with a ghost layer.         */
/* ------------------------------------------------------------------------ */

typedef struct {
  const ofv_problem *P;
  int nvar, nx, ny;
  double dx, dy;
  maxent_rule rule;
} ctx_t;

#define AT(W, v, i, j, nx, ny) ((W)[((size_t)(v) * (ny) + (j)) * (nx) + (i)])

static void get_cell(const double *W, int nvar, int nx, int ny, int i, int j,
                     double *c) {
  for (int v = 0; v < nvar; ++v) c[v] = AT(W, v, i, j, nx, ny);
}

/* Largest cell eigenvalue over the whole state: the global form of the
 * checkTimeStep task. */
double ofv_lambda_max(const ofv_problem *P, const double *W) {
  int nvar = ofv_nvar(P->system), nx = P->nx, ny = P->ny;
  double lmax = 0.0;
  int bad = 0;
#pragma omp parallel for reduction(max : lmax) reduction(| : bad) schedule(static)
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double c[OFV_MAXVAR];
      get_cell(W, nvar, nx, ny, i, j, c);
      double l = cell_lambda(P, c);
      if (!(l == l) || isinf(l)) bad = 1;
      else if (l > lmax) lmax = l;
    }
  }
  return bad ? NAN : lmax;
}

static void plain_fv_update(const ctx_t *C, double dt, const double *W,
                            double *Wout) {
  const ofv_problem *P = C->P;
  int nvar = C->nvar, nx = C->nx, ny = C->ny;
  int gx = nx + 2, gy = ny + 2;
  double *G = (double *)malloc(sizeof(double) * nvar * gx * gy);
  double *Fx = (double *)malloc(sizeof(double) * nvar * (nx + 1) * ny);
  double *Fy = (double *)malloc(sizeof(double) * nvar * nx * (ny + 1));
  /* interior */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int v = 0; v < nvar; ++v)
        AT(G, v, i + 1, j + 1, gx, gy) = AT(W, v, i, j, nx, ny);
  /* ghost columns (W side at gi = 0, E side at gi = nx + 1) */
  for (int j = 0; j < ny; ++j) {
    double own[OFV_MAXVAR], wrap[OFV_MAXVAR], g[OFV_MAXVAR];
    get_cell(W, nvar, nx, ny, 0, j, own);
    get_cell(W, nvar, nx, ny, nx - 1, j, wrap);
    ghost_value(P, nvar, OFV_W, own, wrap, g);
    for (int v = 0; v < nvar; ++v) AT(G, v, 0, j + 1, gx, gy) = g[v];
    get_cell(W, nvar, nx, ny, nx - 1, j, own);
    get_cell(W, nvar, nx, ny, 0, j, wrap);
    ghost_value(P, nvar, OFV_E, own, wrap, g);
    for (int v = 0; v < nvar; ++v) AT(G, v, nx + 1, j + 1, gx, gy) = g[v];
  }
  /* ghost rows (S side at gj = 0, N side at gj = ny + 1) */
  for (int i = 0; i < nx; ++i) {
    double own[OFV_MAXVAR], wrap[OFV_MAXVAR], g[OFV_MAXVAR];
    get_cell(W, nvar, nx, ny, i, 0, own);
    get_cell(W, nvar, nx, ny, i, ny - 1, wrap);
    ghost_value(P, nvar, OFV_S, own, wrap, g);
    for (int v = 0; v < nvar; ++v) AT(G, v, i + 1, 0, gx, gy) = g[v];
    get_cell(W, nvar, nx, ny, i, ny - 1, own);
    get_cell(W, nvar, nx, ny, i, 0, wrap);
    ghost_value(P, nvar, OFV_N, own, wrap, g);
    for (int v = 0; v < nvar; ++v) AT(G, v, i + 1, ny + 1, gx, gy) = g[v];
  }
  /* one flux per x-face: face i sits between cells i-1 and i */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i <= nx; ++i) {
      double L[OFV_MAXVAR], R[OFV_MAXVAR], F[OFV_MAXVAR];
      get_cell(G, nvar, gx, gy, i, j + 1, L);
      get_cell(G, nvar, gx, gy, i + 1, j + 1, R);
      lf_flux(P, nvar, L, R, 1.0, 0.0, F);
      for (int v = 0; v < nvar; ++v) AT(Fx, v, i, j, nx + 1, ny) = F[v];
    }
  }
  /* one flux per y-face: face j sits between cells j-1 and j */
#pragma omp parallel for schedule(static)
  for (int j = 0; j <= ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double L[OFV_MAXVAR], R[OFV_MAXVAR], F[OFV_MAXVAR];
      get_cell(G, nvar, gx, gy, i + 1, j, L);
      get_cell(G, nvar, gx, gy, i + 1, j + 1, R);
      lf_flux(P, nvar, L, R, 0.0, 1.0, F);
      for (int v = 0; v < nvar; ++v) AT(Fy, v, i, j, nx, ny + 1) = F[v];
    }
  }
  double lx = dt / C->dx, ly = dt / C->dy;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double Fe[OFV_MAXVAR], Fw[OFV_MAXVAR], Fn[OFV_MAXVAR], Fs[OFV_MAXVAR];
      double R[OFV_MAXVAR];
      for (int v = 0; v < nvar; ++v) {
        Fw[v] = AT(Fx, v, i, j, nx + 1, ny);
        Fe[v] = AT(Fx, v, i + 1, j, nx + 1, ny);
        Fs[v] = AT(Fy, v, i, j, nx, ny + 1);
        Fn[v] = AT(Fy, v, i, j + 1, nx, ny + 1);
      }
      cell_rhs(nvar, lx, ly, Fe, Fw, Fn, Fs, R);
      for (int v = 0; v < nvar; ++v)
        AT(Wout, v, i, j, nx, ny) = AT(W, v, i, j, nx, ny) + R[v];
    }
  }
  free(G);
  free(Fx);
  free(Fy);
}

/* ------------------------------------------------------------------------ */
/* Literal mode: the paper's per-subdomain data and tasks (Sec. 4).         */
/* ------------------------------------------------------------------------ */

typedef struct {
  int x0, y0, nxl, nyl;
  double *uLoc, *RHS;               /* nvar x nyl x nxl, x fastest */
  double *ovlp[4];                  /* E, N, W, S; nvar x (nyl or nxl) */
} subdomain_t;

/* Balanced split of n cells into np parts: the first (n mod np) parts get
 * one extra cell (Sec. 3.2). */
static void balanced_split(int n, int np, int *start, int *len) {
  int base = n / np, extra = n % np, s = 0;
  for (int p = 0; p < np; ++p) {
    start[p] = s;
    len[p] = base + (p < extra ? 1 : 0);
    s += len[p];
  }
}

#define LOC(D, v, i, j) ((D)->uLoc[((size_t)(v) * (D)->nyl + (j)) * (D)->nxl + (i)])
#define RHSL(D, v, i, j) ((D)->RHS[((size_t)(v) * (D)->nyl + (j)) * (D)->nxl + (i)])
#define OVL(D, side, v, k)                                                  \
  ((D)->ovlp[side][(size_t)(v) *                                            \
                       (((side) == OFV_E || (side) == OFV_W) ? (D)->nyl     \
                                                             : (D)->nxl) +  \
                   (k)])

typedef struct {
  int npx, npy;
  subdomain_t *sd; /* npx * npy, index q * npx + p */
} partition_t;

static subdomain_t *SD(partition_t *T, int p, int q) {
  return &T->sd[q * T->npx + p];
}

/* initialCondition task: fill every uLoc from the global state. */
static void literal_scatter(partition_t *T, int nvar, int nx, int ny,
                            const double *W) {
  for (int q = 0; q < T->npy; ++q)
    for (int p = 0; p < T->npx; ++p) {
      subdomain_t *D = SD(T, p, q);
      for (int v = 0; v < nvar; ++v)
        for (int j = 0; j < D->nyl; ++j)
          for (int i = 0; i < D->nxl; ++i)
            LOC(D, v, i, j) = AT(W, v, D->x0 + i, D->y0 + j, nx, ny);
    }
}

/* gatherForOutput task: copy every uLoc back into the global array. */
static void literal_gather(partition_t *T, int nvar, int nx, int ny,
                           double *W) {
  for (int q = 0; q < T->npy; ++q)
    for (int p = 0; p < T->npx; ++p) {
      subdomain_t *D = SD(T, p, q);
      for (int v = 0; v < nvar; ++v)
        for (int j = 0; j < D->nyl; ++j)
          for (int i = 0; i < D->nxl; ++i)
            AT(W, v, D->x0 + i, D->y0 + j, nx, ny) = LOC(D, v, i, j);
    }
}

static int literal_alloc(partition_t *T, const ofv_problem *P, int nvar) {
  int npx = P->npart_x, npy = P->npart_y;
  int *xs = (int *)malloc(sizeof(int) * npx), *xl = (int *)malloc(sizeof(int) * npx);
  int *ys = (int *)malloc(sizeof(int) * npy), *yl = (int *)malloc(sizeof(int) * npy);
  balanced_split(P->nx, npx, xs, xl);
  balanced_split(P->ny, npy, ys, yl);
  T->npx = npx;
  T->npy = npy;
  T->sd = (subdomain_t *)calloc((size_t)npx * npy, sizeof(subdomain_t));
  for (int q = 0; q < npy; ++q)
    for (int p = 0; p < npx; ++p) {
      subdomain_t *D = SD(T, p, q);
      D->x0 = xs[p];
      D->nxl = xl[p];
      D->y0 = ys[q];
      D->nyl = yl[q];
      size_t n = (size_t)nvar * D->nxl * D->nyl;
      D->uLoc = (double *)malloc(sizeof(double) * n);
      D->RHS = (double *)malloc(sizeof(double) * n);
      /* the four overlap strips are always allocated (Sec. 4.1.2) */
      D->ovlp[OFV_E] = (double *)malloc(sizeof(double) * nvar * D->nyl);
      D->ovlp[OFV_W] = (double *)malloc(sizeof(double) * nvar * D->nyl);
      D->ovlp[OFV_N] = (double *)malloc(sizeof(double) * nvar * D->nxl);
      D->ovlp[OFV_S] = (double *)malloc(sizeof(double) * nvar * D->nxl);
    }
  free(xs);
  free(xl);
  free(ys);
  free(yl);
  return OFV_OK;
}

static void literal_free(partition_t *T) {
  for (int k = 0; k < T->npx * T->npy; ++k) {
    subdomain_t *D = &T->sd[k];
    free(D->uLoc);
    free(D->RHS);
    for (int s = 0; s < 4; ++s) free(D->ovlp[s]);
  }
  free(T->sd);
}

/* checkTimeStep task on one subdomain: its largest cell eigenvalue. */
static double task_check_time_step(const ofv_problem *P, int nvar,
                                   subdomain_t *D) {
  double lmax = 0.0;
  for (int j = 0; j < D->nyl; ++j)
    for (int i = 0; i < D->nxl; ++i) {
      double c[OFV_MAXVAR];
      for (int v = 0; v < nvar; ++v) c[v] = LOC(D, v, i, j);
      double l = cell_lambda(P, c);
      if (!(l == l) || isinf(l)) return NAN;
      if (l > lmax) lmax = l;
    }
  return lmax;
}

/* copyOverlaps task of subdomain (p,q), Sec. 4.2: its north row goes to the
 * northern neighbour's ovlpS, its south row to the southern neighbour's
 * ovlpN, its east column to the eastern neighbour's ovlpW and its west column
 * to the western neighbour's ovlpE.  Across a periodic side the neighbour is
 * the wrapped subdomain; on another physical side the subdomain fills its own
 * strip with the boundary ghost instead. */
static void task_copy_overlaps(const ofv_problem *P, int nvar, partition_t *T,
                               int p, int q) {
  subdomain_t *D = SD(T, p, q);
  int npx = T->npx, npy = T->npy;
  /* east column -> ovlpW of the eastern neighbour */
  if (p + 1 < npx || P->bc[OFV_E] == OFV_PERIODIC) {
    subdomain_t *Nb = SD(T, (p + 1) % npx, q);
    for (int v = 0; v < nvar; ++v)
      for (int j = 0; j < D->nyl; ++j)
        OVL(Nb, OFV_W, v, j) = LOC(D, v, D->nxl - 1, j);
  } else {
    for (int j = 0; j < D->nyl; ++j) {
      double own[OFV_MAXVAR], g[OFV_MAXVAR];
      for (int v = 0; v < nvar; ++v) own[v] = LOC(D, v, D->nxl - 1, j);
      ghost_value(P, nvar, OFV_E, own, own, g);
      for (int v = 0; v < nvar; ++v) OVL(D, OFV_E, v, j) = g[v];
    }
  }
  /* west column -> ovlpE of the western neighbour */
  if (p > 0 || P->bc[OFV_W] == OFV_PERIODIC) {
    subdomain_t *Nb = SD(T, (p + npx - 1) % npx, q);
    for (int v = 0; v < nvar; ++v)
      for (int j = 0; j < D->nyl; ++j)
        OVL(Nb, OFV_E, v, j) = LOC(D, v, 0, j);
  } else {
    for (int j = 0; j < D->nyl; ++j) {
      double own[OFV_MAXVAR], g[OFV_MAXVAR];
      for (int v = 0; v < nvar; ++v) own[v] = LOC(D, v, 0, j);
      ghost_value(P, nvar, OFV_W, own, own, g);
      for (int v = 0; v < nvar; ++v) OVL(D, OFV_W, v, j) = g[v];
    }
  }
  /* north row -> ovlpS of the northern neighbour */
  if (q + 1 < npy || P->bc[OFV_N] == OFV_PERIODIC) {
    subdomain_t *Nb = SD(T, p, (q + 1) % npy);
    for (int v = 0; v < nvar; ++v)
      for (int i = 0; i < D->nxl; ++i)
        OVL(Nb, OFV_S, v, i) = LOC(D, v, i, D->nyl - 1);
  } else {
    for (int i = 0; i < D->nxl; ++i) {
      double own[OFV_MAXVAR], g[OFV_MAXVAR];
      for (int v = 0; v < nvar; ++v) own[v] = LOC(D, v, i, D->nyl - 1);
      ghost_value(P, nvar, OFV_N, own, own, g);
      for (int v = 0; v < nvar; ++v) OVL(D, OFV_N, v, i) = g[v];
    }
  }
  /* south row -> ovlpN of the southern neighbour */
  if (q > 0 || P->bc[OFV_S] == OFV_PERIODIC) {
    subdomain_t *Nb = SD(T, p, (q + npy - 1) % npy);
    for (int v = 0; v < nvar; ++v)
      for (int i = 0; i < D->nxl; ++i)
        OVL(Nb, OFV_N, v, i) = LOC(D, v, i, 0);
  } else {
    for (int i = 0; i < D->nxl; ++i) {
      double own[OFV_MAXVAR], g[OFV_MAXVAR];
      for (int v = 0; v < nvar; ++v) own[v] = LOC(D, v, i, 0);
      ghost_value(P, nvar, OFV_S, own, own, g);
      for (int v = 0; v < nvar; ++v) OVL(D, OFV_S, v, i) = g[v];
    }
  }
}

/* Neighbour value of cell (i,j) of subdomain D across side `side`: a cell
 * of uLoc, or the overlap strip at the subdomain border. */
static void neighbour(const subdomain_t *D, int nvar, int i, int j, int side,
                      double *c) {
  int ii = i, jj = j;
  switch (side) {
    case OFV_E: ii = i + 1; break;
    case OFV_W: ii = i - 1; break;
    case OFV_N: jj = j + 1; break;
    default: jj = j - 1; break;
  }
  if (ii < 0 || ii >= D->nxl || jj < 0 || jj >= D->nyl) {
    int k = (side == OFV_E || side == OFV_W) ? j : i;
    for (int v = 0; v < nvar; ++v) c[v] = OVL(D, side, v, k);
  } else {
    for (int v = 0; v < nvar; ++v) c[v] = LOC(D, v, ii, jj);
  }
}

static void literal_cell_rhs(const ofv_problem *P, int nvar, subdomain_t *D,
                             int i, int j, double lx, double ly) {
  double c[OFV_MAXVAR], e[OFV_MAXVAR], w[OFV_MAXVAR], n[OFV_MAXVAR],
      s[OFV_MAXVAR];
  double Fe[OFV_MAXVAR], Fw[OFV_MAXVAR], Fn[OFV_MAXVAR], Fs[OFV_MAXVAR],
      R[OFV_MAXVAR];
  for (int v = 0; v < nvar; ++v) c[v] = LOC(D, v, i, j);
  neighbour(D, nvar, i, j, OFV_E, e);
  neighbour(D, nvar, i, j, OFV_W, w);
  neighbour(D, nvar, i, j, OFV_N, n);
  neighbour(D, nvar, i, j, OFV_S, s);
  lf_flux(P, nvar, c, e, 1.0, 0.0, Fe);
  lf_flux(P, nvar, w, c, 1.0, 0.0, Fw);
  lf_flux(P, nvar, c, n, 0.0, 1.0, Fn);
  lf_flux(P, nvar, s, c, 0.0, 1.0, Fs);
  cell_rhs(nvar, lx, ly, Fe, Fw, Fn, Fs, R);
  for (int v = 0; v < nvar; ++v) RHSL(D, v, i, j) = R[v];
}

static int is_border(const subdomain_t *D, int i, int j) {
  return i == 0 || j == 0 || i == D->nxl - 1 || j == D->nyl - 1;
}

/* internalResiduals task: residuals of the cells whose four faces lie
 * inside the subdomain (no overlap strip needed). */
static void task_internal_residuals(const ofv_problem *P, int nvar,
                                    subdomain_t *D, double lx, double ly) {
  for (int j = 0; j < D->nyl; ++j)
    for (int i = 0; i < D->nxl; ++i)
      if (!is_border(D, i, j)) literal_cell_rhs(P, nvar, D, i, j, lx, ly);
}

/* borderResiduals task: residuals of the border cells, whose outer faces
 * use the subdomain's own overlap strips.  Each cell's residual is written
 * once, from its four faces, so literal and plain modes agree bit for bit;
 * the inner faces of border cells are evaluated again here, as the paper's
 * GPU kernels evaluate every face twice (Sec. 5.3.1). */
static void task_border_residuals(const ofv_problem *P, int nvar,
                                  subdomain_t *D, double lx, double ly) {
  for (int j = 0; j < D->nyl; ++j)
    for (int i = 0; i < D->nxl; ++i)
      if (is_border(D, i, j)) literal_cell_rhs(P, nvar, D, i, j, lx, ly);
}

/* update task, Eq. (update): u += RHS. */
static void task_update(int nvar, subdomain_t *D) {
  size_t n = (size_t)nvar * D->nxl * D->nyl;
  for (size_t k = 0; k < n; ++k) D->uLoc[k] = D->uLoc[k] + D->RHS[k];
}

/* ------------------------------------------------------------------------ */
/* Driver.                                                                  */
/* ------------------------------------------------------------------------ */

static int validate(const ofv_problem *P) {
  if (ofv_nvar(P->system) == 0) return OFV_ERR_ARG;
  if (P->nx < 1 || P->ny < 1) return OFV_ERR_ARG;
  if (P->npart_x < 1 || P->npart_y < 1) return OFV_ERR_ARG;
  if (P->npart_x > P->nx || P->npart_y > P->ny) return OFV_ERR_ARG;
  if (!(P->xmax > P->xmin) || !(P->ymax > P->ymin)) return OFV_ERR_ARG;
  for (int s = 0; s < 4; ++s)
    if (P->bc[s] < 0 || P->bc[s] > 2) return OFV_ERR_ARG;
  if ((P->bc[OFV_E] == OFV_PERIODIC) != (P->bc[OFV_W] == OFV_PERIODIC))
    return OFV_ERR_ARG;
  if ((P->bc[OFV_N] == OFV_PERIODIC) != (P->bc[OFV_S] == OFV_PERIODIC))
    return OFV_ERR_ARG;
  if (!(P->fixed_dt > 0.0) && !(P->cfl > 0.0)) return OFV_ERR_ARG;
  return OFV_OK;
}

static void setup_ctx(ctx_t *C, const ofv_problem *P) {
  C->P = P;
  C->nvar = ofv_nvar(P->system);
  C->nx = P->nx;
  C->ny = P->ny;
  C->dx = (P->xmax - P->xmin) / P->nx;
  C->dy = (P->ymax - P->ymin) / P->ny;
  C->rule.Q = 0;
  if (P->system == OFV_SPRAY) {
    int Q = (int)P->params[3];
    if (Q <= 0) Q = 32;
    C->rule.Q = Q;
    ofv_gauss_legendre(Q, C->rule.xq, C->rule.wq);
    C->rule.tol = P->params[4] > 0.0 ? P->params[4] : 1e-13;
  }
}

/* Time step of step n from lmax(W^n): Eq. (CFL_cond).  Returns OFV_ERR_CFL
 * when a fixed dt violates it, OFV_ERR_ARG when lmax = 0 leaves the adaptive
 * step unbounded. */
static int choose_dt(const ofv_problem *P, const ctx_t *C, double lmax,
                     double t, double t_end, double *dt) {
  double h = C->dx < C->dy ? C->dx : C->dy;
  if (!(lmax == lmax) || isinf(lmax)) return OFV_ERR_NONPHYSICAL;
  double d;
  if (P->fixed_dt > 0.0) {
    if (P->fixed_dt * lmax > h) return OFV_ERR_CFL;
    d = P->fixed_dt;
  } else {
    double cap = INFINITY;
    if (P->system == OFV_SPRAY && P->params[1] > 0.0) cap = 0.5 * P->params[1];
    if (lmax > 0.0) d = P->cfl * h / lmax;
    else d = INFINITY;
    if (cap < d) d = cap;
    if (isinf(d)) return OFV_ERR_ARG;
  }
  if (t_end > 0.0 && t + d > t_end) d = t_end - t;
  *dt = d;
  return OFV_OK;
}

static int apply_source_global(const ctx_t *C, double dt, double *W) {
  const ofv_problem *P = C->P;
  int nx = C->nx, ny = C->ny;
  int err = OFV_OK;
#pragma omp parallel for schedule(dynamic, 4) reduction(max : err)
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double c[OFV_MAXVAR];
      for (int v = 0; v < 6; ++v) c[v] = AT(W, v, i, j, nx, ny);
      double x = P->xmin + (i + 0.5) * C->dx;
      double y = P->ymin + (j + 0.5) * C->dy;
      int st = spray_source(P, &C->rule, dt, x, y, c);
      if (st != OFV_OK && st > err) err = st;
      for (int v = 0; v < 6; ++v) AT(W, v, i, j, nx, ny) = c[v];
    }
  }
  return err;
}

static int apply_source_literal(const ctx_t *C, double dt, partition_t *T) {
  const ofv_problem *P = C->P;
  int err = OFV_OK;
  int nsd = T->npx * T->npy;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : err)
  for (int k = 0; k < nsd; ++k) {
    subdomain_t *D = &T->sd[k];
    for (int j = 0; j < D->nyl; ++j)
      for (int i = 0; i < D->nxl; ++i) {
        double c[OFV_MAXVAR];
        for (int v = 0; v < 6; ++v) c[v] = LOC(D, v, i, j);
        double x = P->xmin + (D->x0 + i + 0.5) * C->dx;
        double y = P->ymin + (D->y0 + j + 0.5) * C->dy;
        int st = spray_source(P, &C->rule, dt, x, y, c);
        if (st != OFV_OK && st > err) err = st;
        for (int v = 0; v < 6; ++v) LOC(D, v, i, j) = c[v];
      }
  }
  return err;
}

/* Advance W (conserved variables, nvar planes of ny rows of nx values, x
 * fastest) by up to nsteps steps, stopping early at t_end (> 0).
 *   mode 0: plain, mode 1: literal per-subdomain tasks.
 *   t_io: in = start time, out = end time.  dt_hist (nullable) receives the
 *   dt of every completed step; *steps_done the number completed.
 * Returns OFV_OK, or the first error with W at the last good step. */
int ofv_run(const ofv_problem *P, double *W, int nsteps, double t_end,
            int mode, int nthreads, double *t_io, double *dt_hist,
            int *steps_done) {
  int st = validate(P);
  if (st != OFV_OK) return st;
#ifdef _OPENMP
  int saved = omp_get_max_threads();
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  ctx_t C;
  setup_ctx(&C, P);
  int nvar = C.nvar, nx = P->nx, ny = P->ny;
  size_t N = (size_t)nvar * nx * ny;
  double t = t_io ? *t_io : 0.0;
  int done = 0;
  if (mode == 0) {
    double *Wn = (double *)malloc(sizeof(double) * N);
    for (int n = 0; n < nsteps; ++n) {
      if (t_end > 0.0 && t >= t_end) break;
      double lmax = ofv_lambda_max(P, W); /* checkTimeStep */
      double dt;
      st = choose_dt(P, &C, lmax, t, t_end, &dt);
      if (st != OFV_OK) break;
      plain_fv_update(&C, dt, W, Wn);
      if (P->system == OFV_SPRAY) {
        st = apply_source_global(&C, dt, Wn);
        if (st != OFV_OK) break;
      }
      memcpy(W, Wn, sizeof(double) * N);
      t += dt;
      if (dt_hist) dt_hist[done] = dt;
      ++done;
    }
    free(Wn);
  } else {
    partition_t T;
    literal_alloc(&T, P, nvar);
    literal_scatter(&T, nvar, nx, ny, W); /* initialCondition */
    int nsd = T.npx * T.npy;
    double h = C.dx < C.dy ? C.dx : C.dy;
    (void)h;
    for (int n = 0; n < nsteps; ++n) {
      if (t_end > 0.0 && t >= t_end) break;
      /* checkTimeStep on every subdomain, then the global maximum */
      double lmax = 0.0;
      int bad = 0;
      for (int k = 0; k < nsd; ++k) {
        double l = task_check_time_step(P, nvar, &T.sd[k]);
        if (!(l == l)) bad = 1;
        else if (l > lmax) lmax = l;
      }
      double dt;
      st = choose_dt(P, &C, bad ? NAN : lmax, t, t_end, &dt);
      if (st != OFV_OK) break;
      double lx = dt / C.dx, ly = dt / C.dy;
      for (int q = 0; q < T.npy; ++q)
        for (int p = 0; p < T.npx; ++p) task_copy_overlaps(P, nvar, &T, p, q);
#pragma omp parallel for schedule(dynamic, 1)
      for (int k = 0; k < nsd; ++k) {
        task_internal_residuals(P, nvar, &T.sd[k], lx, ly);
        task_border_residuals(P, nvar, &T.sd[k], lx, ly);
        task_update(nvar, &T.sd[k]);
      }
      if (P->system == OFV_SPRAY) {
        st = apply_source_literal(&C, dt, &T);
        if (st != OFV_OK) {
          /* the failing step's state is discarded: restore uLoc from W */
          literal_scatter(&T, nvar, nx, ny, W);
          break;
        }
      }
      literal_gather(&T, nvar, nx, ny, W);
      t += dt;
      if (dt_hist) dt_hist[done] = dt;
      ++done;
    }
    literal_free(&T);
  }
#ifdef _OPENMP
  omp_set_num_threads(saved);
#endif
  if (t_io) *t_io = t;
  if (steps_done) *steps_done = done;
  return st;
}

/* Primitive -> conserved variables of the initial condition, Eq.
 * (initial_condition):
 *   advection (u) -> (u)
 *   euler (rho, u, v, p) -> (rho, rho u, rho v, rho E) with
 *         rho E = p/(gamma-1) + rho (u^2+v^2)/2
 *   spray (m0, m1/2, m1, m3/2, u, v) -> (m0, m1/2, m1, m3/2, m1 u, m1 v). */
int ofv_prim_to_cons(const ofv_problem *P, const double *prim, double *W) {
  int nvar = ofv_nvar(P->system);
  if (!nvar) return OFV_ERR_ARG;
  size_t n = (size_t)P->nx * P->ny;
  for (size_t k = 0; k < n; ++k) {
    if (P->system == OFV_ADVECTION) {
      W[k] = prim[k];
    } else if (P->system == OFV_EULER) {
      double g = P->params[0];
      double rho = prim[k], u = prim[n + k], v = prim[2 * n + k],
             p = prim[3 * n + k];
      W[k] = rho;
      W[n + k] = rho * u;
      W[2 * n + k] = rho * v;
      W[3 * n + k] = p / (g - 1.0) + rho * (u * u + v * v) / 2.0;
    } else {
      for (int v = 0; v < 4; ++v) W[v * n + k] = prim[v * n + k];
      W[4 * n + k] = prim[2 * n + k] * prim[4 * n + k];
      W[5 * n + k] = prim[2 * n + k] * prim[5 * n + k];
    }
  }
  return OFV_OK;
}

/* Per-variable totals sum_ij W_v dx dy with Neumaier compensated summation,
 * row by row and then over rows. */
int ofv_totals(const ofv_problem *P, const double *W, double *tot) {
  int nvar = ofv_nvar(P->system), nx = P->nx, ny = P->ny;
  double dx = (P->xmax - P->xmin) / nx, dy = (P->ymax - P->ymin) / ny;
  for (int v = 0; v < nvar; ++v) {
    double s = 0.0, c = 0.0;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double x = AT(W, v, i, j, nx, ny);
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
      }
    tot[v] = (s + c) * dx * dy;
  }
  return OFV_OK;
}

/* Single-cell helpers exported for the tests. */
double ofv_cell_lambda(const ofv_problem *P, const double *W) {
  return cell_lambda(P, W);
}
void ofv_lf_flux(const ofv_problem *P, const double *WL, const double *WR,
                 double nx_, double ny_, double *F) {
  lf_flux(P, ofv_nvar(P->system), WL, WR, nx_, ny_, F);
}
void ofv_phys_flux(const ofv_problem *P, const double *W, double nx_,
                   double ny_, double *F, double *s) {
  phys_flux(P, W, nx_, ny_, F, s);
}
int ofv_spray_source_cell(const ofv_problem *P, double dt, double x, double y,
                          double *W) {
  ctx_t C;
  setup_ctx(&C, P);
  return spray_source(P, &C.rule, dt, x, y, W);
}
int ofv_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
