/*
 * Plain FP64 CPU oracle: one time step of the 2D-2V micro-macro KFVS scheme for the
 * Boltzmann-ES-BGK equation (Rossmanith & Sar, arXiv 2509.21832, Section 5 and Section 6.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Slow on purpose: every quantity is evaluated straight from the
 * paper's formulas at every phase-space point (one exp per Maxwellian value, velocity sums in
 * sequential k-fastest order).  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code with the CUDA path.
 *
 * OpenMP parallelises over spatial cells only; every cell's arithmetic is sequential, so the
 * result is bitwise identical at any thread count.
 *
 * Readings of passages that are ambiguous or garbled in the paper (all documented in the design
 * notes of the repository):
 *  - KFVS flux (Eq. flux-2D-1/2): the integral form is taken (right-going half from the left
 *    cell, left-going half from the right cell); the printed closed form has the cell indices of
 *    the two halves swapped.
 *  - The KFVS Gaussian is the one whose covariance is the temperature tensor P/rho.
 *  - Eq. (5-99) is evaluated with the cell value u^n_ij.
 *  - 1D-2V problems are the 2D scheme with ny = 1 and periodic y.
 *  - Specular walls (the paper names reflecting walls but prints only the diffuse form): mirror
 *    ghost cells, g_ghost(v) = g(mirrored v), macro ghost with negated normal momentum and
 *    negated off-diagonal energy, heat-flux ghost with the components odd in the normal velocity
 *    negated, Ghat with ghost velocity (-u_n, u_t) and ghost temperature T.
 *  - Diffuse walls: Ghat in wall-adjacent cells is -(1/tau)(I-Pi)[upwind v.grad M] and keeps the
 *    (G-M)/eps term unless wall_keep_es_term is 0; sides of such a cell that are not diffuse use
 *    their own ghost rule for M (extrapolation: M of the cell itself).
 *  - Extrapolation macro boundary flux is the full-range Gaussian flux without the heat flux,
 *    the heat flux at that face being the cell value.
 */
#include "mm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
/* Hard-sphere constant of the 2D Chapman viscosity, remark before Eq. (tau-for-2d-es-bgk). */
#define ORC_C25 0.436

typedef struct {
  double rho, u1, u2, T;
  double P11, P12, P22;
  double tau;
  double Ti11, Ti12, Ti22; /* inverse of the ES tensor (Eq. 2-19) */
  double detT;             /* det of the ES tensor */
} prim_t;

/* ------------------------------------------------------------------------------------------ */
/* Primitive variables (Section 2: u = rho u / rho, P = E - rho u (x) u, T = tr P / (2 rho);     */
/* Eq. 2-19 for the ES tensor; Eq. tau-for-2d-es-bgk and Section 4 for tau).                  */
/* ------------------------------------------------------------------------------------------ */
static int prim_of(const orc_params* p, const double q[6], prim_t* o) {
  double rho = q[0];
  if (!(rho > 0.0) || !isfinite(rho)) return 4;
  double u1 = q[1] / rho;
  double u2 = q[2] / rho;
  double P11 = q[3] - rho * u1 * u1;
  double P12 = q[4] - rho * u1 * u2;
  double P22 = q[5] - rho * u2 * u2;
  double T = (P11 + P22) / (2.0 * rho);
  double t11 = P11 / rho, t12 = P12 / rho, t22 = P22 / rho;
  double nu = p->nu;
  double s11 = (1.0 - nu) * T + nu * t11;
  double s12 = nu * t12;
  double s22 = (1.0 - nu) * T + nu * t22;
  double det = s11 * s22 - s12 * s12;
  if (!(P11 > 0.0) || !(P22 > 0.0) || !(T > 0.0) || !(t11 * t22 - t12 * t12 > 0.0) ||
      !(det > 0.0) || !isfinite(T) || !isfinite(u1) || !isfinite(u2) || !isfinite(P12))
    return 4;
  double tau;
  switch (p->tau_model) {
    case ORC_TAU_RHO: tau = p->tau0 * rho; break;
    case ORC_TAU_HARDSPHERE2D: tau = 3.0 * ORC_PI * ORC_C25 * rho / (sqrt(2.0) * (1.0 - nu)); break;
    case ORC_TAU_PRESSURE: tau = p->tau0 * rho * T; break;
    default: tau = p->tau0; break;
  }
  o->rho = rho; o->u1 = u1; o->u2 = u2; o->T = T;
  o->P11 = P11; o->P12 = P12; o->P22 = P22;
  o->tau = tau;
  o->Ti11 = s22 / det; o->Ti12 = -s12 / det; o->Ti22 = s11 / det;
  o->detT = det;
  return 0;
}

/* Energy tensor E = rho (u (x) u + T I) (Section 2, ES-BGK operator), evaluated in that order
 * and bracketing: E11 = rho (u1 u1 + T), E12 = rho (u1 u2), E22 = rho (u2 u2 + T). */
int orc_q_from_prim(int ncell, const double* rho, const double* u1, const double* u2,
                    const double* T, double* Q) {
  for (int c = 0; c < ncell; ++c)
    if (!(rho[c] > 0.0) || !(T[c] > 0.0) || !isfinite(rho[c]) || !isfinite(T[c]) ||
        !isfinite(u1[c]) || !isfinite(u2[c]))
      return -1;
  for (int c = 0; c < ncell; ++c) {
    Q[0 * ncell + c] = rho[c];
    Q[1 * ncell + c] = rho[c] * u1[c];
    Q[2 * ncell + c] = rho[c] * u2[c];
    Q[3 * ncell + c] = rho[c] * (u1[c] * u1[c] + T[c]);
    Q[4 * ncell + c] = rho[c] * (u1[c] * u2[c]);
    Q[5 * ncell + c] = rho[c] * (u2[c] * u2[c] + T[c]);
  }
  return 0;
}

int orc_prims(const orc_params* p, const double q[6], double out[8]) {
  prim_t o;
  int rc = prim_of(p, q, &o);
  if (rc) return rc;
  out[0] = o.rho; out[1] = o.u1; out[2] = o.u2; out[3] = o.T;
  out[4] = o.P11; out[5] = o.P12; out[6] = o.P22; out[7] = o.tau;
  return 0;
}

/* Eq. (5-31) */
static double maxwell(const prim_t* c, double v1, double v2) {
  double c1 = v1 - c->u1, c2 = v2 - c->u2;
  return c->rho / (2.0 * ORC_PI * c->T) * exp(-(c1 * c1 + c2 * c2) / (2.0 * c->T));
}

/* Eq. (5-28): rho / sqrt(det(2 pi Tcal)) exp(-1/2 c . Tcal^{-1} c) */
static double gauss_es(const prim_t* c, double v1, double v2) {
  double c1 = v1 - c->u1, c2 = v2 - c->u2;
  double quad = c->Ti11 * c1 * c1 + 2.0 * c->Ti12 * c1 * c2 + c->Ti22 * c2 * c2;
  return c->rho / sqrt(4.0 * ORC_PI * ORC_PI * c->detT) * exp(-0.5 * quad);
}

void orc_maxwellian_gauss(const orc_params* p, const double q[6], double v1, double v2,
                          double* M, double* Gs) {
  prim_t c;
  if (prim_of(p, q, &c)) { *M = NAN; *Gs = NAN; return; }
  *M = maxwell(&c, v1, v2);
  *Gs = gauss_es(&c, v1, v2);
}

/* ------------------------------------------------------------------------------------------ */
/* grid helpers                                                                                 */
/* ------------------------------------------------------------------------------------------ */
static double vel1(const orc_grid* g, int k) {
  double dv = (g->v1max - g->v1min) / g->nv1;
  return g->v1min + (k + 0.5) * dv;
}
static double vel2(const orc_grid* g, int l) {
  double dv = (g->v2max - g->v2min) / g->nv2;
  return g->v2min + (l + 0.5) * dv;
}
static size_t cell_of(const orc_grid* g, int i, int j) { return (size_t)j * g->nx + i; }
static size_t gidx(const orc_grid* g, int i, int j, int k, int l) {
  return (cell_of(g, i, j) * g->nv2 + l) * g->nv1 + k;
}

/* ------------------------------------------------------------------------------------------ */
/* Projection Pi_M (Eqs. 5-33, 5-33-plus; midpoint quadrature of Section 5.3)                  */
/* ------------------------------------------------------------------------------------------ */
static void project(const orc_grid* g, const prim_t* c, const double* F, double* out) {
  double dv1 = (g->v1max - g->v1min) / g->nv1;
  double dv2 = (g->v2max - g->v2min) / g->nv2;
  double sqT = sqrt(c->T);
  double A1 = 0, A2 = 0, A3 = 0, A4 = 0;
  for (int l = 0; l < g->nv2; ++l)
    for (int k = 0; k < g->nv1; ++k) {
      double c1 = vel1(g, k) - c->u1, c2 = vel2(g, l) - c->u2;
      double f = F[l * g->nv1 + k];
      A1 += f;
      A2 += c1 / sqT * f;
      A3 += c2 / sqT * f;
      A4 += ((c1 * c1 + c2 * c2) / (2.0 * c->T) - 1.0) * f;
    }
  double w = dv1 * dv2 / c->rho;
  A1 *= w; A2 *= w; A3 *= w; A4 *= w;
  for (int l = 0; l < g->nv2; ++l)
    for (int k = 0; k < g->nv1; ++k) {
      double v1 = vel1(g, k), v2 = vel2(g, l);
      double c1 = v1 - c->u1, c2 = v2 - c->u2;
      out[l * g->nv1 + k] =
          (A1 + A2 * c1 / sqT + A3 * c2 / sqT + A4 * ((c1 * c1 + c2 * c2) / (2.0 * c->T) - 1.0)) *
          maxwell(c, v1, v2);
    }
}

void orc_project(const orc_grid* g, double rho, double u1, double u2, double T, const double* F,
                 double* out) {
  prim_t c;
  memset(&c, 0, sizeof c);
  c.rho = rho; c.u1 = u1; c.u2 = u2; c.T = T;
  project(g, &c, F, out);
}

/* ------------------------------------------------------------------------------------------ */
/* KFVS half-range fluxes (Eq. flux-2D-1 / flux-2D-2 with a, b, J, K)                           */
/* ------------------------------------------------------------------------------------------ */
static void kfvs_abJK(const double q[6], int dir, double* a, double* b, double J[6], double K[6]) {
  double rho = q[0];
  double u1 = q[1] / rho, u2 = q[2] / rho;
  double P11 = q[3] - rho * u1 * u1;
  double P12 = q[4] - rho * u1 * u2;
  double P22 = q[5] - rho * u2 * u2;
  if (dir == 1) {
    *a = sqrt(2.0 * P11 / (ORC_PI * rho)) * exp(-rho * u1 * u1 / (2.0 * P11));
    *b = erf(u1 * sqrt(rho / (2.0 * P11)));
    J[0] = rho;
    J[1] = rho * u1;
    J[2] = rho * u2;
    J[3] = rho * u1 * u1 + 2.0 * P11;
    J[4] = rho * u1 * u2 + 2.0 * P12;
    J[5] = rho * u2 * u2 + P22 + P12 * P12 / P11;
    K[0] = rho * u1;
    K[1] = rho * u1 * u1 + P11;
    K[2] = rho * u1 * u2 + P12;
    K[3] = rho * u1 * u1 * u1 + 3.0 * u1 * P11;
    K[4] = rho * u1 * u1 * u2 + u2 * P11 + 2.0 * u1 * P12;
    K[5] = rho * u1 * u2 * u2 + u1 * P22 + 2.0 * u2 * P12;
  } else {
    *a = sqrt(2.0 * P22 / (ORC_PI * rho)) * exp(-rho * u2 * u2 / (2.0 * P22));
    *b = erf(u2 * sqrt(rho / (2.0 * P22)));
    J[0] = rho;
    J[1] = rho * u1;
    J[2] = rho * u2;
    J[3] = rho * u1 * u1 + P11 + P12 * P12 / P22;
    J[4] = rho * u1 * u2 + 2.0 * P12;
    J[5] = rho * u2 * u2 + 2.0 * P22;
    K[0] = rho * u2;
    K[1] = rho * u1 * u2 + P12;
    K[2] = rho * u2 * u2 + P22;
    K[3] = rho * u1 * u1 * u2 + u2 * P11 + 2.0 * u1 * P12;
    K[4] = rho * u1 * u2 * u2 + u1 * P22 + 2.0 * u2 * P12;
    K[5] = rho * u2 * u2 * u2 + 3.0 * u2 * P22;
  }
}

void orc_kfvs_half(const double q[6], int dir, double Fp[6], double Fm[6]) {
  double a, b, J[6], K[6];
  kfvs_abJK(q, dir, &a, &b, J, K);
  for (int m = 0; m < 6; ++m) {
    Fp[m] = 0.5 * (a * J[m] + (1.0 + b) * K[m]);
    Fm[m] = 0.5 * (-a * J[m] + (1.0 - b) * K[m]);
  }
}

static void kfvs_full(const double q[6], int dir, double F[6]) {
  double a, b, J[6], K[6];
  kfvs_abJK(q, dir, &a, &b, J, K);
  for (int m = 0; m < 6; ++m) F[m] = K[m];
}

/* Eq. (twodim_wall_densities_1) */
double orc_wall_R(double ua, double Taa, double Tw, int sign) {
  return sqrt(Taa / Tw) * exp(-ua * ua / (2.0 * Taa)) +
         ua * sqrt(ORC_PI / (2.0 * Tw)) * (erf(ua / sqrt(2.0 * Taa)) + (sign > 0 ? 1.0 : -1.0));
}

/* TR-BDF2 factor of the macro collision half step (Section 5.4) */
double orc_trbdf2_W(double tau, double nu, double eps, double dt) {
  double a = tau * (1.0 - nu);
  return (48.0 * eps * eps - 10.0 * a * eps * dt) /
         (48.0 * eps * eps + 14.0 * a * eps * dt + (a * dt) * (a * dt));
}

/* ------------------------------------------------------------------------------------------ */
/* time step rule                                                                               */
/* ------------------------------------------------------------------------------------------ */
double orc_dt_for_cfl(const orc_grid* g, double cfl, double t_final, int form, int* nsteps_out) {
  double dx = (g->x1 - g->x0) / g->nx;
  double dy = (g->y1 - g->y0) / g->ny;
  double V1 = fmax(fabs(g->v1min), fabs(g->v1max));
  double V2 = fmax(fabs(g->v2min), fabs(g->v2max));
  double dt;
  if (g->ny == 1)
    dt = cfl * dx / V1; /* 1D rule of Section 3.2 */
  else if (form == ORC_CFL_MIN)
    dt = cfl * fmin(dx / V1, dy / V2);
  else
    dt = cfl / (V1 / dx + V2 / dy);
  int n = 0;
  if (t_final > 0.0) {
    n = (int)ceil(t_final / dt * (1.0 - 1e-12));
    if (n < 1) n = 1;
    dt = t_final / n;
  }
  if (nsteps_out) *nsteps_out = n;
  return dt;
}

/* ------------------------------------------------------------------------------------------ */
/* micro sweeps                                                                                 */
/* ------------------------------------------------------------------------------------------ */

/* Value of G on the x-neighbour of (i, j) on side s (0: i-1, 1: i+1), ghost rules at walls. */
static double gx_nb(const orc_grid* g, const orc_params* p, const double* G, int i, int j, int k,
                    int l, int s) {
  int nb = s == 0 ? i - 1 : i + 1;
  if (nb >= 0 && nb < g->nx) return G[gidx(g, nb, j, k, l)];
  switch (p->bc[s]) {
    case ORC_BC_PERIODIC: return G[gidx(g, s == 0 ? g->nx - 1 : 0, j, k, l)];
    case ORC_BC_EXTRAP: return G[gidx(g, i, j, k, l)];
    case ORC_BC_SPECULAR: return G[gidx(g, i, j, g->nv1 - 1 - k, l)];
    default: return 0.0; /* diffuse: inflow of g set to zero */
  }
}
static double gy_nb(const orc_grid* g, const orc_params* p, const double* G, int i, int j, int k,
                    int l, int s) {
  int nb = s == 0 ? j - 1 : j + 1;
  if (nb >= 0 && nb < g->ny) return G[gidx(g, i, nb, k, l)];
  switch (p->bc[2 + s]) {
    case ORC_BC_PERIODIC: return G[gidx(g, i, s == 0 ? g->ny - 1 : 0, k, l)];
    case ORC_BC_EXTRAP: return G[gidx(g, i, j, k, l)];
    case ORC_BC_SPECULAR: return G[gidx(g, i, j, k, g->nv2 - 1 - l)];
    default: return 0.0;
  }
}

/* One split micro transport step, Eqs. (zmicrox)-(update-micro-2D-xdir) for dir = 1 and
 * Eqs. (zmicroy)-(update-micro-2D-ydir) for dir = 2.  Gin -> Gout, with M^n, u^n, T^n, rho^n. */
static void micro_sweep(const orc_grid* g, const orc_params* p, const prim_t* P, const double* Mc,
                        const double* Gin, double* Gout, double dt, int dir) {
  const int nx = g->nx, ny = g->ny, nv1 = g->nv1, nv2 = g->nv2, nv = nv1 * nv2;
  const double dx = (g->x1 - g->x0) / nx, dy = (g->y1 - g->y0) / ny;
  const double dv1 = (g->v1max - g->v1min) / nv1, dv2 = (g->v2max - g->v2min) / nv2;
#pragma omp parallel
  {
    double* Z = (double*)malloc(sizeof(double) * nv);
#pragma omp for schedule(static)
    for (int c = 0; c < nx * ny; ++c) {
      int i = c % nx, j = c / nx;
      const prim_t* pc = &P[c];
      for (int l = 0; l < nv2; ++l)
        for (int k = 0; k < nv1; ++k) {
          double g0 = Gin[gidx(g, i, j, k, l)];
          double v = dir == 1 ? vel1(g, k) : vel2(g, l);
          double h = dir == 1 ? dx : dy;
          double gm = dir == 1 ? gx_nb(g, p, Gin, i, j, k, l, 0) : gy_nb(g, p, Gin, i, j, k, l, 0);
          double gp = dir == 1 ? gx_nb(g, p, Gin, i, j, k, l, 1) : gy_nb(g, p, Gin, i, j, k, l, 1);
          double vm = v < 0.0 ? v : 0.0, vp = v > 0.0 ? v : 0.0;
          Z[l * nv1 + k] = vm * ((gp - g0) / h) + vp * ((g0 - gm) / h);
        }
      /* coefficients A1..A4, Eq. (coeffs-2D-xdir) / (coeffs-2D-ydir) */
      double sqT = sqrt(pc->T);
      double A1 = 0, A2 = 0, A3 = 0, A4 = 0;
      for (int l = 0; l < nv2; ++l)
        for (int k = 0; k < nv1; ++k) {
          double c1 = vel1(g, k) - pc->u1, c2 = vel2(g, l) - pc->u2;
          double z = Z[l * nv1 + k];
          A1 += z;
          A2 += c1 / sqT * z;
          A3 += c2 / sqT * z;
          A4 += ((c1 * c1 + c2 * c2) / (2.0 * pc->T) - 1.0) * z;
        }
      double w = dv1 * dv2 / pc->rho;
      A1 *= w; A2 *= w; A3 *= w; A4 *= w;
      const double* M = Mc + (size_t)c * nv;
      for (int l = 0; l < nv2; ++l)
        for (int k = 0; k < nv1; ++k) {
          double c1 = vel1(g, k) - pc->u1, c2 = vel2(g, l) - pc->u2;
          double zhat = (A1 + A2 * c1 / sqT + A3 * c2 / sqT +
                         A4 * ((c1 * c1 + c2 * c2) / (2.0 * pc->T) - 1.0)) * M[l * nv1 + k];
          size_t id = gidx(g, i, j, k, l);
          Gout[id] = Gin[id] + dt * (zhat - Z[l * nv1 + k]);
        }
    }
    free(Z);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Ghat (Eq. 5-97, 5-97more; wall form of Section 6.3)                                          */
/* ------------------------------------------------------------------------------------------ */

static int is_diffuse_wall_cell(const orc_grid* g, const orc_params* p, int i, int j) {
  return (i == 0 && p->bc[0] == ORC_BC_DIFFUSE) || (i == g->nx - 1 && p->bc[1] == ORC_BC_DIFFUSE) ||
         (j == 0 && p->bc[2] == ORC_BC_DIFFUSE) || (j == g->ny - 1 && p->bc[3] == ORC_BC_DIFFUSE);
}

/* (u1, u2, T) seen across side s of cell (i, j): the neighbour, or the ghost value. */
static void nb_uT(const orc_grid* g, const orc_params* p, const prim_t* P, int i, int j, int s,
                  double* u1, double* u2, double* T) {
  int ni = i, nj = j;
  if (s == 0) ni = i - 1;
  if (s == 1) ni = i + 1;
  if (s == 2) nj = j - 1;
  if (s == 3) nj = j + 1;
  const prim_t* c = &P[cell_of(g, i, j)];
  if (ni >= 0 && ni < g->nx && nj >= 0 && nj < g->ny) {
    const prim_t* n = &P[cell_of(g, ni, nj)];
    *u1 = n->u1; *u2 = n->u2; *T = n->T;
    return;
  }
  switch (p->bc[s]) {
    case ORC_BC_PERIODIC: {
      if (s < 2) ni = (ni + g->nx) % g->nx; else nj = (nj + g->ny) % g->ny;
      const prim_t* n = &P[cell_of(g, ni, nj)];
      *u1 = n->u1; *u2 = n->u2; *T = n->T;
      return;
    }
    case ORC_BC_SPECULAR:
      *u1 = s < 2 ? -c->u1 : c->u1;
      *u2 = s < 2 ? c->u2 : -c->u2;
      *T = c->T;
      return;
    default: /* extrapolation (and diffuse, not used here) */
      *u1 = c->u1; *u2 = c->u2; *T = c->T;
      return;
  }
}

/* Maxwellian seen across side s of cell (i, j) at velocity (k, l), for the wall form. */
static double nb_maxwell(const orc_grid* g, const orc_params* p, const prim_t* P, const double* Mc,
                         int i, int j, int k, int l, int s) {
  int ni = i, nj = j;
  if (s == 0) ni = i - 1;
  if (s == 1) ni = i + 1;
  if (s == 2) nj = j - 1;
  if (s == 3) nj = j + 1;
  const int nv = g->nv1 * g->nv2;
  size_t c = cell_of(g, i, j);
  if (ni >= 0 && ni < g->nx && nj >= 0 && nj < g->ny)
    return Mc[cell_of(g, ni, nj) * nv + (size_t)l * g->nv1 + k];
  switch (p->bc[s]) {
    case ORC_BC_PERIODIC:
      if (s < 2) ni = (ni + g->nx) % g->nx; else nj = (nj + g->ny) % g->ny;
      return Mc[cell_of(g, ni, nj) * nv + (size_t)l * g->nv1 + k];
    case ORC_BC_EXTRAP: return Mc[c * nv + (size_t)l * g->nv1 + k];
    case ORC_BC_SPECULAR:
      if (s < 2) return Mc[c * nv + (size_t)l * g->nv1 + (g->nv1 - 1 - k)];
      return Mc[c * nv + (size_t)(g->nv2 - 1 - l) * g->nv1 + k];
    default: {
      /* diffuse wall Maxwellian, Eqs. (lid_driven_bc_1..4) with the zero-mass-flux density of
       * Eq. (twodim_wall_densities_1/2) from the wall-adjacent cell at time n. */
      const prim_t* pc = &P[c];
      double Tw = p->wall_T[s], U = p->wall_U[s];
      double v1 = vel1(g, k), v2 = vel2(g, l);
      double rw, e;
      if (s < 2) {
        rw = pc->rho * orc_wall_R(pc->u1, pc->P11 / pc->rho, Tw, s == 0 ? -1 : +1);
        e = (v1 * v1 + (v2 - U) * (v2 - U)) / (2.0 * Tw);
      } else {
        rw = pc->rho * orc_wall_R(pc->u2, pc->P22 / pc->rho, Tw, s == 2 ? -1 : +1);
        e = ((v1 - U) * (v1 - U) + v2 * v2) / (2.0 * Tw);
      }
      return rw / (2.0 * ORC_PI * Tw) * exp(-e);
    }
  }
}

static void ghat_cell(const orc_grid* g, const orc_params* p, const prim_t* P, const double* Mc,
                      int i, int j, double eps, double* out, double* tmp) {
  const int nv1 = g->nv1, nv2 = g->nv2, nv = nv1 * nv2;
  const double dx = (g->x1 - g->x0) / g->nx, dy = (g->y1 - g->y0) / g->ny;
  size_t c = cell_of(g, i, j);
  const prim_t* pc = &P[c];
  const double* M = Mc + c * nv;
  if (is_diffuse_wall_cell(g, p, i, j)) {
    /* upwind v . grad M with wall ghost Maxwellians, then -(1/tau)(I - Pi_M) of it */
    for (int l = 0; l < nv2; ++l)
      for (int k = 0; k < nv1; ++k) {
        double v1 = vel1(g, k), v2 = vel2(g, l);
        double m0 = M[l * nv1 + k];
        double mL = nb_maxwell(g, p, P, Mc, i, j, k, l, 0);
        double mR = nb_maxwell(g, p, P, Mc, i, j, k, l, 1);
        double mB = nb_maxwell(g, p, P, Mc, i, j, k, l, 2);
        double mT = nb_maxwell(g, p, P, Mc, i, j, k, l, 3);
        double v1m = v1 < 0.0 ? v1 : 0.0, v1p = v1 > 0.0 ? v1 : 0.0;
        double v2m = v2 < 0.0 ? v2 : 0.0, v2p = v2 > 0.0 ? v2 : 0.0;
        tmp[l * nv1 + k] = v1m * ((mR - m0) / dx) + v1p * ((m0 - mL) / dx) +
                           v2m * ((mT - m0) / dy) + v2p * ((m0 - mB) / dy);
      }
    project(g, pc, tmp, out);
    for (int l = 0; l < nv2; ++l)
      for (int k = 0; k < nv1; ++k) {
        int id = l * nv1 + k;
        double val = -(1.0 / pc->tau) * (tmp[id] - out[id]);
        if (p->wall_keep_es_term)
          val += (gauss_es(pc, vel1(g, k), vel2(g, l)) - M[id]) / eps;
        out[id] = val;
      }
    return;
  }
  double uL1, uL2, TL, uR1, uR2, TR, uB1, uB2, TB, uT1, uT2, TT;
  nb_uT(g, p, P, i, j, 0, &uL1, &uL2, &TL);
  nb_uT(g, p, P, i, j, 1, &uR1, &uR2, &TR);
  nb_uT(g, p, P, i, j, 2, &uB1, &uB2, &TB);
  nb_uT(g, p, P, i, j, 3, &uT1, &uT2, &TT);
  /* face temperatures and centred velocity differences, Eqs. (5-97), (5-97more) */
  double Tface_xp = 0.5 * (TR + pc->T), Tface_xm = 0.5 * (pc->T + TL);
  double Tface_yp = 0.5 * (TT + pc->T), Tface_ym = 0.5 * (pc->T + TB);
  double dTdx = (Tface_xp - Tface_xm) / dx;
  double dTdy = (Tface_yp - Tface_ym) / dy;
  double Dx_u1 = (uR1 - uL1) / 2.0, Dx_u2 = (uR2 - uL2) / 2.0;
  double Dy_u1 = (uT1 - uB1) / 2.0, Dy_u2 = (uT2 - uB2) / 2.0;
  double s11 = Dx_u1 / dx - Dy_u2 / dy;
  double s12 = Dy_u1 / dy + Dx_u2 / dx;
  double s21 = s12;
  double s22 = -Dx_u1 / dx + Dy_u2 / dy;
  double T = pc->T;
  for (int l = 0; l < nv2; ++l)
    for (int k = 0; k < nv1; ++k) {
      double v1 = vel1(g, k), v2 = vel2(g, l);
      double c1 = v1 - pc->u1, c2 = v2 - pc->u2;
      /* B and C of Eq. (5-69) */
      double B11 = -c2 * c2 / (2.0 * T), B12 = c1 * c2 / (2.0 * T);
      double B21 = c1 * c2 / (2.0 * T), B22 = -c1 * c1 / (2.0 * T);
      double BS = B11 * s11 + B12 * s12 + B21 * s21 + B22 * s22;
      double cc = ((c1 * c1 + c2 * c2) / (2.0 * T) - 2.0) / T;
      double CT = cc * c1 * dTdx + cc * c2 * dTdy;
      double m = M[l * nv1 + k];
      out[l * nv1 + k] = -(1.0 / pc->tau) * (BS + CT) * m + (gauss_es(pc, v1, v2) - m) / eps;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* The 2D-2V manufactured solution of the convergence study (Section 6.1, "Method of           */
/* Manufactured Solutions Example"): f = phi(v) F(t, x, y) with                                 */
/*   phi = exp(-(v1-1)^2 - (v2-1)^2) + 2 exp(-(v1+1)^2 - (v2+1)^2),                            */
/*   F   = 2 - sin(2 pi (t - x)) cos(2 pi (t - y)),                                            */
/* whose moments are pi F (3, -1, -1, 9/2, 3, 9/2) (rho, rho u, E; the paper lists rho, rho u  */
/* and P = (25/6, 8/3, 25/6) pi F), and the residual                                            */
/*   S = f_t + v1 f_x + v2 f_y - (tau/eps)(Gcal[f] - f)                                         */
/* with tau and the ES Gaussian Gcal of the exact moments.                                     */
/* ------------------------------------------------------------------------------------------ */
static double mms_F(double t, double x, double y) {
  return 2.0 - sin(2.0 * ORC_PI * (t - x)) * cos(2.0 * ORC_PI * (t - y));
}

static double mms_phi(double v1, double v2) {
  return exp(-(v1 - 1.0) * (v1 - 1.0) - (v2 - 1.0) * (v2 - 1.0)) +
         2.0 * exp(-(v1 + 1.0) * (v1 + 1.0) - (v2 + 1.0) * (v2 + 1.0));
}

static void mms_q(double t, double x, double y, double q[6]) {
  double pf = ORC_PI * mms_F(t, x, y);
  q[0] = 3.0 * pf; q[1] = -pf; q[2] = -pf; q[3] = 4.5 * pf; q[4] = 3.0 * pf; q[5] = 4.5 * pf;
}

/* S at the velocity nodes of the cell centred at (x, y), time t; returns 0 or 4. */
static int mms_source(const orc_grid* g, const orc_params* p, double eps, double t, double x,
                      double y, double* S) {
  const double w = 2.0 * ORC_PI;
  const double s1 = sin(w * (t - x)), c1 = cos(w * (t - x));
  const double s2 = sin(w * (t - y)), c2 = cos(w * (t - y));
  const double F_t = -w * c1 * c2 + w * s1 * s2;  /* d/dt [2 - sin(w(t-x)) cos(w(t-y))] */
  const double F_x = w * c1 * c2;
  const double F_y = -w * s1 * s2;
  const double F = 2.0 - s1 * c2;
  double q[6];
  mms_q(t, x, y, q);
  prim_t e;
  if (prim_of(p, q, &e)) return 4;
  for (int l = 0; l < g->nv2; ++l)
    for (int k = 0; k < g->nv1; ++k) {
      const double v1 = vel1(g, k), v2 = vel2(g, l);
      const double ph = mms_phi(v1, v2);
      S[l * g->nv1 + k] = ph * (F_t + v1 * F_x + v2 * F_y) -
                          (e.tau / eps) * (gauss_es(&e, v1, v2) - ph * F);
    }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* macro helpers                                                                                */
/* ------------------------------------------------------------------------------------------ */

/* Collision half step of Section 5.4 with tau taken from q itself. */
/* The step needs rho > 0 and T > 0 (tau); the pressure tensor of its input need not be
 * positive definite (with a manufactured source the state before the last half step can leave
 * that set; the relaxation brings it back). */
static int coll_half(const orc_params* p, const double q[6], double eps, double dt, double out[6]) {
  const double rho = q[0];
  if (!(rho > 0.0) || !isfinite(rho)) return 4;
  const double u1 = q[1] / rho, u2 = q[2] / rho;
  const double P11 = q[3] - rho * u1 * u1;
  const double P12 = q[4] - rho * u1 * u2;
  const double P22 = q[5] - rho * u2 * u2;
  const double T = (P11 + P22) / (2.0 * rho);
  if (!(T > 0.0) || !isfinite(T) || !isfinite(P12) || !isfinite(u1) || !isfinite(u2)) return 4;
  double tau;
  switch (p->tau_model) {
    case ORC_TAU_RHO: tau = p->tau0 * rho; break;
    case ORC_TAU_HARDSPHERE2D: tau = 3.0 * ORC_PI * ORC_C25 * rho / (sqrt(2.0) * (1.0 - p->nu)); break;
    case ORC_TAU_PRESSURE: tau = p->tau0 * rho * T; break;
    default: tau = p->tau0; break;
  }
  double W = orc_trbdf2_W(tau, p->nu, eps, dt);
  double n11 = 0.5 * ((1.0 + W) * P11 + (1.0 - W) * P22);
  double n12 = 0.5 * (2.0 * W * P12);
  double n22 = 0.5 * ((1.0 - W) * P11 + (1.0 + W) * P22);
  out[0] = q[0];
  out[1] = q[1];
  out[2] = q[2];
  out[3] = rho * u1 * u1 + n11;
  out[4] = rho * u1 * u2 + n12;
  out[5] = rho * u2 * u2 + n22;
  return 0;
}

static void mirror_q(const double q[6], int dir, double o[6]) {
  o[0] = q[0];
  o[1] = dir == 1 ? -q[1] : q[1];
  o[2] = dir == 1 ? q[2] : -q[2];
  o[3] = q[3];
  o[4] = -q[4];
  o[5] = q[5];
}

/* Diffuse wall ghost state of Section 6.3, built from the wall-adjacent cell's moments q. */
static void wall_ghost_q(const orc_params* p, const double q[6], int side, double o[6]) {
  double rho = q[0];
  double u1 = q[1] / rho, u2 = q[2] / rho;
  double P11 = q[3] - rho * u1 * u1;
  double P22 = q[5] - rho * u2 * u2;
  double Tw = p->wall_T[side], U = p->wall_U[side];
  double rw, gu1, gu2;
  if (side < 2) {
    rw = rho * orc_wall_R(u1, P11 / rho, Tw, side == 0 ? -1 : +1);
    gu1 = 0.0; gu2 = U;
  } else {
    rw = rho * orc_wall_R(u2, P22 / rho, Tw, side == 2 ? -1 : +1);
    gu1 = U; gu2 = 0.0;
  }
  o[0] = rw;
  o[1] = rw * gu1;
  o[2] = rw * gu2;
  o[3] = rw * (gu1 * gu1 + Tw);
  o[4] = rw * gu1 * gu2;
  o[5] = rw * (gu2 * gu2 + Tw);
}

/* Numerical flux through x-face f (0..nx) of row j: face f lies between cells f-1 and f. */
static void face_flux_x(const orc_grid* g, const orc_params* p, const double* Qs, int f, int j,
                        double F[6]) {
  const int nx = g->nx, nc = g->nx * g->ny;
  double qa[6], qb[6], Fp[6], Fm[6], t[6];
  int left = f - 1, right = f;
  if (f > 0 && f < nx) {
    for (int m = 0; m < 6; ++m) { qa[m] = Qs[m * nc + cell_of(g, left, j)]; qb[m] = Qs[m * nc + cell_of(g, right, j)]; }
    orc_kfvs_half(qa, 1, Fp, t);
    orc_kfvs_half(qb, 1, t, Fm);
    for (int m = 0; m < 6; ++m) F[m] = Fp[m] + Fm[m];
    return;
  }
  int side = f == 0 ? 0 : 1;
  int cell = f == 0 ? 0 : nx - 1;
  double qc[6];
  for (int m = 0; m < 6; ++m) qc[m] = Qs[m * nc + cell_of(g, cell, j)];
  switch (p->bc[side]) {
    case ORC_BC_PERIODIC:
      for (int m = 0; m < 6; ++m) { qa[m] = Qs[m * nc + cell_of(g, nx - 1, j)]; qb[m] = Qs[m * nc + cell_of(g, 0, j)]; }
      break;
    case ORC_BC_EXTRAP:
      kfvs_full(qc, 1, F);
      return;
    case ORC_BC_SPECULAR:
      if (side == 0) { mirror_q(qc, 1, qa); memcpy(qb, qc, sizeof qb); }
      else { memcpy(qa, qc, sizeof qa); mirror_q(qc, 1, qb); }
      break;
    default:
      if (side == 0) { wall_ghost_q(p, qc, 0, qa); memcpy(qb, qc, sizeof qb); }
      else { memcpy(qa, qc, sizeof qa); wall_ghost_q(p, qc, 1, qb); }
      break;
  }
  orc_kfvs_half(qa, 1, Fp, t);
  orc_kfvs_half(qb, 1, t, Fm);
  for (int m = 0; m < 6; ++m) F[m] = Fp[m] + Fm[m];
}

static void face_flux_y(const orc_grid* g, const orc_params* p, const double* Qs, int i, int f,
                        double F[6]) {
  const int ny = g->ny, nc = g->nx * g->ny;
  double qa[6], qb[6], Fp[6], Fm[6], t[6];
  if (f > 0 && f < ny) {
    for (int m = 0; m < 6; ++m) { qa[m] = Qs[m * nc + cell_of(g, i, f - 1)]; qb[m] = Qs[m * nc + cell_of(g, i, f)]; }
    orc_kfvs_half(qa, 2, Fp, t);
    orc_kfvs_half(qb, 2, t, Fm);
    for (int m = 0; m < 6; ++m) F[m] = Fp[m] + Fm[m];
    return;
  }
  int side = f == 0 ? 2 : 3;
  int cell = f == 0 ? 0 : ny - 1;
  double qc[6];
  for (int m = 0; m < 6; ++m) qc[m] = Qs[m * nc + cell_of(g, i, cell)];
  switch (p->bc[side]) {
    case ORC_BC_PERIODIC:
      for (int m = 0; m < 6; ++m) { qa[m] = Qs[m * nc + cell_of(g, i, ny - 1)]; qb[m] = Qs[m * nc + cell_of(g, i, 0)]; }
      break;
    case ORC_BC_EXTRAP:
      kfvs_full(qc, 2, F);
      return;
    case ORC_BC_SPECULAR:
      if (side == 2) { mirror_q(qc, 2, qa); memcpy(qb, qc, sizeof qb); }
      else { memcpy(qa, qc, sizeof qa); mirror_q(qc, 2, qb); }
      break;
    default:
      if (side == 2) { wall_ghost_q(p, qc, 2, qa); memcpy(qb, qc, sizeof qb); }
      else { memcpy(qa, qc, sizeof qa); wall_ghost_q(p, qc, 3, qb); }
      break;
  }
  orc_kfvs_half(qa, 2, Fp, t);
  orc_kfvs_half(qb, 2, t, Fm);
  for (int m = 0; m < 6; ++m) F[m] = Fp[m] + Fm[m];
}

/* Heat flux H component h at x-face f of row j (Eq. 5-103 face averages and the BC rules). */
static double face_H_x(const orc_grid* g, const orc_params* p, const double* H, int f, int j, int h) {
  const int nx = g->nx, nc = g->nx * g->ny;
  if (f > 0 && f < nx) return 0.5 * (H[h * nc + cell_of(g, f, j)] + H[h * nc + cell_of(g, f - 1, j)]);
  int side = f == 0 ? 0 : 1;
  double hc = H[h * nc + cell_of(g, f == 0 ? 0 : nx - 1, j)];
  switch (p->bc[side]) {
    case ORC_BC_PERIODIC: return 0.5 * (H[h * nc + cell_of(g, 0, j)] + H[h * nc + cell_of(g, nx - 1, j)]);
    case ORC_BC_EXTRAP: return hc;
    case ORC_BC_SPECULAR: {
      /* ghost flips the components odd in c1: H111 (h=0) and H122 (h=2) */
      double hg = (h == 0 || h == 2) ? -hc : hc;
      return 0.5 * (hc + hg);
    }
    default: return 0.5 * hc;
  }
}
static double face_H_y(const orc_grid* g, const orc_params* p, const double* H, int i, int f, int h) {
  const int ny = g->ny, nc = g->nx * g->ny;
  if (f > 0 && f < ny) return 0.5 * (H[h * nc + cell_of(g, i, f)] + H[h * nc + cell_of(g, i, f - 1)]);
  int side = f == 0 ? 2 : 3;
  double hc = H[h * nc + cell_of(g, i, f == 0 ? 0 : ny - 1)];
  switch (p->bc[side]) {
    case ORC_BC_PERIODIC: return 0.5 * (H[h * nc + cell_of(g, i, 0)] + H[h * nc + cell_of(g, i, ny - 1)]);
    case ORC_BC_EXTRAP: return hc;
    case ORC_BC_SPECULAR: {
      /* ghost flips the components odd in c2: H112 (h=1) and H222 (h=3) */
      double hg = (h == 1 || h == 3) ? -hc : hc;
      return 0.5 * (hc + hg);
    }
    default: return 0.5 * hc;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* validation                                                                                   */
/* ------------------------------------------------------------------------------------------ */
static int check_args(const orc_grid* g, const orc_params* p) {
  if (!g || !p) return 1;
  if (g->nx < 1 || g->ny < 1 || g->nv1 < 1 || g->nv2 < 1) return 1;
  if (!(g->x1 > g->x0) || !(g->y1 > g->y0) || !(g->v1max > g->v1min) || !(g->v2max > g->v2min)) return 1;
  for (int s = 0; s < 4; ++s) if (p->bc[s] < 0 || p->bc[s] > 3) return 1;
  if ((p->bc[0] == ORC_BC_PERIODIC) != (p->bc[1] == ORC_BC_PERIODIC)) return 1;
  if ((p->bc[2] == ORC_BC_PERIODIC) != (p->bc[3] == ORC_BC_PERIODIC)) return 1;
  if (!(p->nu >= -1.0 && p->nu < 1.0)) return 1;
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* one full time step, Section 5.3 (micro) then Section 5.4 (macro)                             */
/* ------------------------------------------------------------------------------------------ */
/* One or more steps; with closure != NULL (one step): cells with refresh[c] != 0 first take
 * g^n = Ghat(Q^n); then cells with closure[c] != 0 keep g^n and take the heat flux Hcl[m][c] in
 * place of the relaxed micro solution and its moments.  With mms != 0 the manufactured source
 * S(t^n), t^n = t0 + n dt, enters Ghat as + (1/tau^n)(I - Pi_M)[S] and the macro update as
 * Q*** += dt int (1, v, v (x) v) S dv between the y transport and the last collision half step
 * (Section 6.1, Eq. macro2d-split3b). */
static int step_impl(const orc_grid* g, const orc_params* p, double* Q, double* G, double* H,
                     double dt, double eps, int nsteps, const unsigned char* closure,
                     const unsigned char* refresh, const double* Hcl, int mms, double t0) {
  if (check_args(g, p) || !Q || !G || !H || !(dt > 0.0) || !(eps > 0.0) || nsteps < 0) return 1;
  const int nx = g->nx, ny = g->ny, nv1 = g->nv1, nv2 = g->nv2, nv = nv1 * nv2;
  const int nc = nx * ny;
  const double dx = (g->x1 - g->x0) / nx, dy = (g->y1 - g->y0) / ny;
  const double dv1 = (g->v1max - g->v1min) / nv1, dv2 = (g->v2max - g->v2min) / nv2;
  size_t ng = (size_t)nc * nv;
  prim_t* P = (prim_t*)malloc(sizeof(prim_t) * nc);
  double* Mc = (double*)malloc(sizeof(double) * ng);
  double* Gs = (double*)malloc(sizeof(double) * ng);
  double* Gss = (double*)malloc(sizeof(double) * ng);
  double* Q1 = (double*)malloc(sizeof(double) * 6 * nc);
  double* Q2 = (double*)malloc(sizeof(double) * 6 * nc);
  int status = 0;
  if (!P || !Mc || !Gs || !Gss || !Q1 || !Q2) status = 2;

  for (int step = 0; step < nsteps && status == 0; ++step) {
    /* primitive variables and Maxwellian M^n on the phase-space grid */
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int c = 0; c < nc; ++c) {
      double q[6];
      for (int m = 0; m < 6; ++m) q[m] = Q[m * nc + c];
      if (prim_of(p, q, &P[c])) { bad = 1; continue; }
      for (int l = 0; l < nv2; ++l)
        for (int k = 0; k < nv1; ++k)
          Mc[(size_t)c * nv + l * nv1 + k] = maxwell(&P[c], vel1(g, k), vel2(g, l));
    }
    if (bad) { status = 4; break; }

    /* closure: refreshed cells start the step from Ghat(Q^n) */
    if (refresh) {
#pragma omp parallel
      {
        double* tmp = (double*)malloc(sizeof(double) * nv);
#pragma omp for schedule(static)
        for (int c = 0; c < nc; ++c)
          if (refresh[c]) ghat_cell(g, p, P, Mc, c % nx, c / nx, eps, G + (size_t)c * nv, tmp);
        free(tmp);
      }
    }

    /* micro: x sweep (G^n -> G*), y sweep (G* -> G**) */
    micro_sweep(g, p, P, Mc, G, Gs, dt, 1);
    micro_sweep(g, p, P, Mc, Gs, Gss, dt, 2);

    /* micro: backward-Euler relaxation toward Ghat (Eq. 5-98), then H^{n+1} (Eq. 5-99) */
#pragma omp parallel
    {
      double* gh = (double*)malloc(sizeof(double) * 2 * nv);  /* Ghat, then Pi_M[S] */
      double* tmp = (double*)malloc(sizeof(double) * nv);
#pragma omp for schedule(static)
      for (int c = 0; c < nc; ++c) {
        int i = c % nx, j = c / nx;
        const prim_t* pc = &P[c];
        if (closure && closure[c]) {
          for (int m = 0; m < 4; ++m) H[m * nc + c] = Hcl[m * nc + c];
          continue;
        }
        ghat_cell(g, p, P, Mc, i, j, eps, gh, tmp);
        if (mms) {
          const double dx = (g->x1 - g->x0) / nx, dy = (g->y1 - g->y0) / ny;
          const double tn = t0 + step * dt;
          if (mms_source(g, p, eps, tn, g->x0 + (i + 0.5) * dx, g->y0 + (j + 0.5) * dy, tmp) == 0) {
            project(g, pc, tmp, gh + nv);
            for (int id = 0; id < nv; ++id) gh[id] += (tmp[id] - gh[nv + id]) / pc->tau;
          }
        }
        double w1 = eps / (eps + dt * pc->tau);
        double w2 = dt * pc->tau / (eps + dt * pc->tau);
        double h111 = 0, h112 = 0, h122 = 0, h222 = 0;
        for (int l = 0; l < nv2; ++l)
          for (int k = 0; k < nv1; ++k) {
            size_t id = gidx(g, i, j, k, l);
            double gn = w1 * Gss[id] + w2 * gh[l * nv1 + k];
            G[id] = gn;
            double c1 = vel1(g, k) - pc->u1, c2 = vel2(g, l) - pc->u2;
            h111 += c1 * c1 * c1 * gn;
            h112 += c1 * c1 * c2 * gn;
            h122 += c1 * c2 * c2 * gn;
            h222 += c2 * c2 * c2 * gn;
          }
        H[0 * nc + c] = eps * dv1 * dv2 * h111;
        H[1 * nc + c] = eps * dv1 * dv2 * h112;
        H[2 * nc + c] = eps * dv1 * dv2 * h122;
        H[3 * nc + c] = eps * dv1 * dv2 * h222;
      }
      free(gh);
      free(tmp);
    }

    /* macro, Strang splitting (Eqs. macro2d-split1..4) */
    /* (1) collision half step with tau^n: Q^n -> Q* (stored in Q1) */
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int c = 0; c < nc; ++c) {
      double q[6], o[6];
      for (int m = 0; m < 6; ++m) q[m] = Q[m * nc + c];
      if (coll_half(p, q, eps, dt, o)) { bad = 1; continue; }
      for (int m = 0; m < 6; ++m) Q1[m * nc + c] = o[m];
    }
    if (bad) { status = 4; break; }
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int c = 0; c < nc; ++c) {
      prim_t t;
      double q[6];
      for (int m = 0; m < 6; ++m) q[m] = Q1[m * nc + c];
      if (prim_of(p, q, &t)) bad = 1;
    }
    if (bad) { status = 4; break; }
    /* (2) x transport: Q* -> Q** (stored in Q2), Eq. (5-103) first line */
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; ++c) {
      int i = c % nx, j = c / nx;
      double FL[6], FR[6];
      face_flux_x(g, p, Q1, i, j, FL);
      face_flux_x(g, p, Q1, i + 1, j, FR);
      double dH[3];
      for (int h = 0; h < 3; ++h) dH[h] = face_H_x(g, p, H, i + 1, j, h) - face_H_x(g, p, H, i, j, h);
      for (int m = 0; m < 6; ++m) {
        double v = Q1[m * nc + c] - dt / dx * (FR[m] - FL[m]);
        if (m >= 3) v -= dt * (dH[m - 3] / dx);
        Q2[m * nc + c] = v;
      }
    }
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int c = 0; c < nc; ++c) {
      prim_t t;
      double q[6];
      for (int m = 0; m < 6; ++m) q[m] = Q2[m * nc + c];
      if (prim_of(p, q, &t)) bad = 1;
    }
    if (bad) { status = 4; break; }
    /* (3) y transport: Q** -> Q*** (stored in Q1), Eq. (5-103) second line */
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; ++c) {
      int i = c % nx, j = c / nx;
      double FB[6], FT[6];
      face_flux_y(g, p, Q2, i, j, FB);
      face_flux_y(g, p, Q2, i, j + 1, FT);
      double dH[3];
      for (int h = 0; h < 3; ++h) dH[h] = face_H_y(g, p, H, i, j + 1, h + 1) - face_H_y(g, p, H, i, j, h + 1);
      for (int m = 0; m < 6; ++m) {
        double v = Q2[m * nc + c] - dt / dy * (FT[m] - FB[m]);
        if (m >= 3) v -= dt * (dH[m - 3] / dy);
        Q1[m * nc + c] = v;
      }
    }
    /* (3b) manufactured source: Q*** += dt int (1, v1, v2, v1^2, v1 v2, v2^2) S(t^n) dv */
    if (mms) {
      const double tn = t0 + step * dt;
#pragma omp parallel
      {
        double* S = (double*)malloc(sizeof(double) * nv);
#pragma omp for schedule(static) reduction(| : bad)
        for (int c = 0; c < nc; ++c) {
          int i = c % nx, j = c / nx;
          if (mms_source(g, p, eps, tn, g->x0 + (i + 0.5) * dx, g->y0 + (j + 0.5) * dy, S)) {
            bad = 1;
            continue;
          }
          double m[6] = {0, 0, 0, 0, 0, 0};
          for (int l = 0; l < nv2; ++l)
            for (int k = 0; k < nv1; ++k) {
              double v1 = vel1(g, k), v2 = vel2(g, l), sv = S[l * nv1 + k];
              m[0] += sv; m[1] += v1 * sv; m[2] += v2 * sv;
              m[3] += v1 * v1 * sv; m[4] += v1 * v2 * sv; m[5] += v2 * v2 * sv;
            }
          for (int q = 0; q < 6; ++q) Q1[q * nc + c] += dt * dv1 * dv2 * m[q];
        }
        free(S);
      }
      if (bad) { status = 4; break; }
    }
    /* (4) collision half step with tau***: Q*** -> Q^{n+1} */
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int c = 0; c < nc; ++c) {
      double q[6], o[6];
      for (int m = 0; m < 6; ++m) q[m] = Q1[m * nc + c];
      if (coll_half(p, q, eps, dt, o)) { bad = 1; continue; }
      for (int m = 0; m < 6; ++m) Q[m * nc + c] = o[m];
    }
    if (bad) { status = 4; break; }
  }
  free(P); free(Mc); free(Gs); free(Gss); free(Q1); free(Q2);
  return status;
}

int orc_step(const orc_grid* g, const orc_params* p, double* Q, double* G, double* H, double dt,
             double eps, int nsteps) {
  return step_impl(g, p, Q, G, H, dt, eps, nsteps, NULL, NULL, NULL, 0, 0.0);
}

int orc_step_closure(const orc_grid* g, const orc_params* p, double* Q, double* G, double* H,
                     double dt, double eps, const unsigned char* closure,
                     const unsigned char* refresh, const double* Hcl) {
  if (!closure || !refresh || !Hcl) return 1;
  return step_impl(g, p, Q, G, H, dt, eps, 1, closure, refresh, Hcl, 0, 0.0);
}

int orc_mms_source(const orc_grid* g, const orc_params* p, double eps, double t, double x,
                   double y, double* S) {
  if (check_args(g, p) || !S || !(eps > 0.0)) return 1;
  return mms_source(g, p, eps, t, x, y, S);
}

int orc_step_mms(const orc_grid* g, const orc_params* p, double* Q, double* G, double* H,
                 double dt, double eps, int nsteps, double t0) {
  return step_impl(g, p, Q, G, H, dt, eps, nsteps, NULL, NULL, NULL, 1, t0);
}

int orc_mms_exact(const orc_grid* g, const orc_params* p, double t, double eps, double* Q,
                  double* G) {
  if (check_args(g, p) || !Q || !G || !(eps > 0.0)) return 1;
  const int nx = g->nx, ny = g->ny, nv1 = g->nv1, nv2 = g->nv2, nc = nx * ny;
  const double dx = (g->x1 - g->x0) / nx, dy = (g->y1 - g->y0) / ny;
  for (int c = 0; c < nc; ++c) {
    const int i = c % nx, j = c / nx;
    const double x = g->x0 + (i + 0.5) * dx, y = g->y0 + (j + 0.5) * dy;
    double q[6];
    mms_q(t, x, y, q);
    for (int m = 0; m < 6; ++m) Q[m * nc + c] = q[m];
    prim_t e;
    if (prim_of(p, q, &e)) return 4;
    const double F = mms_F(t, x, y);
    for (int l = 0; l < nv2; ++l)
      for (int k = 0; k < nv1; ++k) {
        const double v1 = vel1(g, k), v2 = vel2(g, l);
        G[gidx(g, i, j, k, l)] = (mms_phi(v1, v2) * F - maxwell(&e, v1, v2)) / eps;
      }
  }
  return 0;
}

int orc_ghat(const orc_grid* g, const orc_params* p, const double* Q, double eps, double* Ghat) {
  if (check_args(g, p) || !Q || !Ghat || !(eps > 0.0)) return 1;
  const int nx = g->nx, ny = g->ny, nv1 = g->nv1, nv2 = g->nv2, nv = nv1 * nv2, nc = nx * ny;
  prim_t* P = (prim_t*)malloc(sizeof(prim_t) * nc);
  double* Mc = (double*)malloc(sizeof(double) * (size_t)nc * nv);
  if (!P || !Mc) { free(P); free(Mc); return 2; }
  int bad = 0;
  for (int c = 0; c < nc && !bad; ++c) {
    double q[6];
    for (int m = 0; m < 6; ++m) q[m] = Q[m * nc + c];
    if (prim_of(p, q, &P[c])) bad = 1;
    else
      for (int l = 0; l < nv2; ++l)
        for (int k = 0; k < nv1; ++k)
          Mc[(size_t)c * nv + l * nv1 + k] = maxwell(&P[c], vel1(g, k), vel2(g, l));
  }
  if (!bad) {
    double* tmp = (double*)malloc(sizeof(double) * nv);
    for (int c = 0; c < nc; ++c) ghat_cell(g, p, P, Mc, c % nx, c / nx, eps, Ghat + (size_t)c * nv, tmp);
    free(tmp);
  }
  free(P); free(Mc);
  return bad ? 4 : 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
