/*
 * Plain FP64 CPU oracle for the 1D-1V micro-macro scheme for the Boltzmann-BGK equation
 * (Rossmanith & Sar, arXiv 2509.21832, Sections 3 and 4: Eqs. 5-11, 5-16, 5-19 ... 5-27 and
 * the KFVS flux of Eq. flux1d_1/2), with the manufactured-solution source of the 1D convergence
 * study (Section 4.1, Table tab5-2).
 *
 * TEST INFRASTRUCTURE ONLY, like mm_oracle.c: only the test suite, the smoke check and the
 * benchmark's CPU leg load it.  It shares no code with the CUDA library.
 *
 * Layouts: Q[3][nx] = (rho, rho u, E) with E = rho T / 2 + rho u^2 / 2; G[nx][nv]; H[nx].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "mm_oracle.h"

#define PI1 3.14159265358979323846

static double v_of(const orc1d_grid* g, int k) {
  return g->vmin + (k + 0.5) * (g->vmax - g->vmin) / g->nv;
}

/* rho, u, T of a cell (Eq. 5-11: E = rho T / 2 + rho u^2 / 2); returns 0 or 4 */
static int prim1(const double* Q, int nx, int i, double* rho, double* u, double* T) {
  *rho = Q[i];
  if (!(*rho > 0.0) || !isfinite(*rho)) return 4;
  *u = Q[nx + i] / *rho;
  *T = 2.0 * Q[2 * nx + i] / *rho - *u * *u;
  if (!(*T > 0.0) || !isfinite(*T) || !isfinite(*u)) return 4;
  return 0;
}

/* tau: the hard-sphere value of Eq. (collision_parameter_1d), or a constant */
static double tau1(const orc1d_params* p, double rho, double T) {
  (void)rho;
  if (p->tau_model == ORC1D_TAU_HARDSPHERE) return 16.0 / 5.0 * sqrt(T / (2.0 * PI1));
  return p->tau0;
}

/* neighbour index across side s (0 left, 1 right): periodic wrap, else the cell itself */
static int nb1(const orc1d_params* p, int nx, int i, int s) {
  int n = s == 0 ? i - 1 : i + 1;
  if (n >= 0 && n < nx) return n;
  if (p->bc[s] == ORC_BC_PERIODIC) return (n + nx) % nx;
  return i;
}

/* Half-range Maxwellian fluxes of Eq. (flux1d_1/2): Fp = int_{v>0} v m M dv, Fm = int_{v<0} */
static void kfvs1(double rho, double u, double T, double Fp[3], double Fm[3]) {
  const double a = sqrt(T / (2.0 * PI1)) * exp(-u * u / (2.0 * T));
  const double e = erf(u / sqrt(2.0 * T));
  const double bp = 0.5 * (1.0 + e), bm = 0.5 * (1.0 - e);
  const double w[3] = {rho, rho * u, 0.5 * rho * (2.0 * T + u * u)};
  const double f[3] = {rho * u, rho * (T + u * u), 0.5 * rho * u * (3.0 * T + u * u)};
  for (int m = 0; m < 3; ++m) {
    Fp[m] = a * w[m] + bp * f[m];
    Fm[m] = -a * w[m] + bm * f[m];
  }
}

/* ---- manufactured solution (Section 4.1) ----------------------------------------------------
 * f = (exp(-(v-1)^2) + 2 exp(-(v+1)^2)) (2 + sin(2 pi (x - t))), rho = 3 sqrt(pi) F, u = -1/3,
 * T = 25/18; S = f_t + v f_x - (tau/eps)(M - f) with M and tau both of the exact state: the
 * passage defines S as a function of (t, x, v) alone, so nothing of the numerical state enters
 * it (with the hard-sphere tau of Eq. collision_parameter_1d, tau(T = 25/18) is a constant). */
static double mms1_phi(double v) { return exp(-(v - 1.0) * (v - 1.0)) + 2.0 * exp(-(v + 1.0) * (v + 1.0)); }
static double mms1_M(double v) { return 1.8 * exp(-0.04 * (3.0 * v + 1.0) * (3.0 * v + 1.0)); }

static void mms1_source(const orc1d_grid* g, double tau, double eps, double t, double x,
                        double* S) {
  const double F = 2.0 + sin(2.0 * PI1 * (x - t));
  const double Fx = 2.0 * PI1 * cos(2.0 * PI1 * (x - t));
  const double Ft = -Fx;
  for (int k = 0; k < g->nv; ++k) {
    const double v = v_of(g, k), ph = mms1_phi(v);
    S[k] = ph * (Ft + v * Fx) - (tau / eps) * (mms1_M(v) - ph) * F;
  }
}

/* Pi_M[F] of Eqs. (5-4), (5-5) with the midpoint rule (Eq. 5-21) for the Maxwellian (rho, u, T) */
static void proj1(const orc1d_grid* g, double rho, double u, double T, const double* Fv,
                  double* out) {
  const double dv = (g->vmax - g->vmin) / g->nv;
  const double sT = sqrt(T);
  double A1 = 0, A2 = 0, A3 = 0;
  for (int k = 0; k < g->nv; ++k) {
    const double c = (v_of(g, k) - u) / sT;
    A1 += Fv[k];
    A2 += c * Fv[k];
    A3 += sqrt(2.0) * (0.5 * c * c - 0.5) * Fv[k];
  }
  A1 *= dv / rho; A2 *= dv / rho; A3 *= dv / rho;
  for (int k = 0; k < g->nv; ++k) {
    const double v = v_of(g, k), c = (v - u) / sT;
    const double M = rho / sqrt(2.0 * PI1 * T) * exp(-(v - u) * (v - u) / (2.0 * T));
    out[k] = (A1 + c * A2 + sqrt(2.0) * (0.5 * c * c - 0.5) * A3) * M;
  }
}

static int check1(const orc1d_grid* g, const orc1d_params* p) {
  if (!g || !p || g->nx < 2 || g->nv < 1 || !(g->x1 > g->x0) || !(g->vmax > g->vmin)) return 1;
  for (int s = 0; s < 2; ++s)
    if (p->bc[s] != ORC_BC_PERIODIC && p->bc[s] != ORC_BC_EXTRAP) return 1;
  if ((p->bc[0] == ORC_BC_PERIODIC) != (p->bc[1] == ORC_BC_PERIODIC)) return 1;
  return 0;
}

int orc1d_step(const orc1d_grid* g, const orc1d_params* p, double* Q, double* G, double* H,
               double dt, double eps, int nsteps, int mms, double t0) {
  if (check1(g, p) || !Q || !G || !H || !(dt > 0.0) || !(eps > 0.0) || nsteps < 0) return 1;
  const int nx = g->nx, nv = g->nv;
  const double dx = (g->x1 - g->x0) / nx, dv = (g->vmax - g->vmin) / nv;
  double* rho = malloc(sizeof(double) * nx);
  double* u = malloc(sizeof(double) * nx);
  double* T = malloc(sizeof(double) * nx);
  double* Gn = malloc(sizeof(double) * (size_t)nx * nv);
  double* Z = malloc(sizeof(double) * nv);
  double* PZ = malloc(sizeof(double) * nv);
  double* S = malloc(sizeof(double) * nv);
  double* PS = malloc(sizeof(double) * nv);
  double* Qn = malloc(sizeof(double) * 3 * nx);
  int status = 0;
  if (!rho || !u || !T || !Gn || !Z || !PZ || !S || !PS || !Qn) status = 2;
  for (int step = 0; step < nsteps && status == 0; ++step) {
    const double tn = t0 + step * dt;
    for (int i = 0; i < nx && status == 0; ++i)
      if (prim1(Q, nx, i, &rho[i], &u[i], &T[i])) status = 4;
    if (status) break;
    /* micro: Eqs. (5-19), (5-20), (5-24), (5-21), (5-25) */
    for (int i = 0; i < nx; ++i) {
      const int iL = nb1(p, nx, i, 0), iR = nb1(p, nx, i, 1);
      const double tau = tau1(p, rho[i], T[i]);
      /* face temperatures: periodic average across the seam, extrapolation the cell itself */
      const double TR = 0.5 * (T[iR] + T[i]), TL = 0.5 * (T[i] + T[iL]);
      const double Tx = (TR - TL) / (dx * T[i]);
      for (int k = 0; k < nv; ++k) {
        const double v = v_of(g, k);
        const double vm = v < 0.0 ? v : 0.0, vp = v > 0.0 ? v : 0.0;
        const double gc = G[(size_t)i * nv + k];
        const int right_ok = !(i == nx - 1 && p->bc[1] != ORC_BC_PERIODIC);
        const int left_ok = !(i == 0 && p->bc[0] != ORC_BC_PERIODIC);
        double z = 0.0;
        if (right_ok) z += vm * (G[(size_t)iR * nv + k] - gc) / dx;
        if (left_ok) z += vp * (gc - G[(size_t)iL * nv + k]) / dx;
        Z[k] = z;
      }
      proj1(g, rho[i], u[i], T[i], Z, PZ);
      if (mms) {
        mms1_source(g, tau1(p, 0.0, 25.0 / 18.0), eps, tn, g->x0 + (i + 0.5) * dx, S);
        proj1(g, rho[i], u[i], T[i], S, PS);
      }
      const double w1 = eps / (eps + dt * tau), w2 = dt * tau / (eps + dt * tau);
      double h = 0.0;
      for (int k = 0; k < nv; ++k) {
        const double v = v_of(g, k), c = v - u[i];
        const double M = rho[i] / sqrt(2.0 * PI1 * T[i]) * exp(-c * c / (2.0 * T[i]));
        double gh = -(1.0 / tau) * (c * c * c / (2.0 * T[i]) - 1.5 * c) * Tx * M;
        if (mms) gh += (S[k] - PS[k]) / tau;
        const double gn = w1 * (G[(size_t)i * nv + k] - dt * (Z[k] - PZ[k])) + w2 * gh;
        Gn[(size_t)i * nv + k] = gn;
        h += v * v * v * gn;
      }
      H[i] = 0.5 * eps * dv * h;
    }
    memcpy(G, Gn, sizeof(double) * (size_t)nx * nv);
    /* macro: Eq. (5-27) with the KFVS flux of Eq. (flux1d_1) and the boundary rules of
     * Eqs. (1d_extrap_macro_1/2), (1d_periodic_macro) */
    for (int i = 0; i < nx; ++i) {
      double FL[3], FR[3], Fp[3], Fm[3], Gp[3], Gm[3];
      const int iL = nb1(p, nx, i, 0), iR = nb1(p, nx, i, 1);
      kfvs1(rho[i], u[i], T[i], Fp, Fm);
      double HL, HR;
      if (i == 0 && p->bc[0] != ORC_BC_PERIODIC) {
        for (int m = 0; m < 3; ++m) FL[m] = Fp[m] + Fm[m];
        HL = H[i];
      } else {
        kfvs1(rho[iL], u[iL], T[iL], Gp, Gm);
        for (int m = 0; m < 3; ++m) FL[m] = Gp[m] + Fm[m];
        HL = 0.5 * (H[i] + H[iL]);
      }
      if (i == nx - 1 && p->bc[1] != ORC_BC_PERIODIC) {
        for (int m = 0; m < 3; ++m) FR[m] = Fp[m] + Fm[m];
        HR = H[i];
      } else {
        kfvs1(rho[iR], u[iR], T[iR], Gp, Gm);
        for (int m = 0; m < 3; ++m) FR[m] = Fp[m] + Gm[m];
        HR = 0.5 * (H[iR] + H[i]);
      }
      for (int m = 0; m < 3; ++m) {
        double q = Q[m * nx + i] - dt / dx * (FR[m] - FL[m]);
        if (m == 2) q -= dt / dx * (HR - HL);
        Qn[m * nx + i] = q;
      }
      if (mms) {
        /* the closed-form source moments printed with the 1D convergence study */
        const double c = pow(PI1, 1.5) * cos(2.0 * PI1 * (g->x0 + (i + 0.5) * dx - tn));
        Qn[i] += dt * c * -8.0;
        Qn[nx + i] += dt * c * 11.0;
        Qn[2 * nx + i] += dt * c * -7.0;
      }
    }
    memcpy(Q, Qn, sizeof(double) * 3 * nx);
  }
  free(rho); free(u); free(T); free(Gn); free(Z); free(PZ); free(S); free(PS); free(Qn);
  return status;
}

int orc1d_mms_exact(const orc1d_grid* g, double t, double eps, double* Q, double* G) {
  if (!g || !Q || !G || g->nx < 1 || g->nv < 1 || !(eps > 0.0)) return 1;
  const int nx = g->nx, nv = g->nv;
  const double dx = (g->x1 - g->x0) / nx;
  for (int i = 0; i < nx; ++i) {
    const double F = 2.0 + sin(2.0 * PI1 * (g->x0 + (i + 0.5) * dx - t));
    const double rho = 3.0 * sqrt(PI1) * F, u = -1.0 / 3.0, T = 25.0 / 18.0;
    Q[i] = rho;
    Q[nx + i] = rho * u;
    Q[2 * nx + i] = 0.5 * rho * T + 0.5 * rho * u * u;
    for (int k = 0; k < nv; ++k) {
      const double v = v_of(g, k);
      G[(size_t)i * nv + k] = (mms1_phi(v) - mms1_M(v)) * F / eps;
    }
  }
  return 0;
}

double orc1d_dt(const orc1d_grid* g, double cfl, double t_final, int* nsteps_out) {
  const double dx = (g->x1 - g->x0) / g->nx;
  const double V = fmax(fabs(g->vmin), fabs(g->vmax));
  double dt = cfl * dx / V;
  int n = (int)ceil(t_final / dt * (1.0 - 1e-12));
  if (n < 1) n = 1;
  if (nsteps_out) *nsteps_out = n;
  return t_final / n;
}
