/*
 * Plain FP64 CPU oracle for one time step of the 2D-2V micro-macro KFVS scheme for the
 * Boltzmann-ES-BGK equation (Rossmanith & Sar, arXiv 2509.21832, Section 5).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product path never calls it.  It shares no source with the
 * CUDA library.
 *
 * Layouts (all row-major C arrays of double):
 *   Q[6][ny][nx]          (rho, rho*u1, rho*u2, E11, E12, E22)      -- Section 5.1, Eq. (5-40)
 *   G[ny][nx][nv2][nv1]   micro part g on the phase-space grid        -- Section 5.2
 *   H[4][ny][nx]          (H111, H112, H122, H222)                    -- Eq. (5-99)
 */
#ifndef MM_ORACLE_H
#define MM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary kinds, side order: 0 left (x=x0), 1 right (x=x1), 2 bottom (y=y0), 3 top (y=y1). */
enum { ORC_BC_PERIODIC = 0, ORC_BC_EXTRAP = 1, ORC_BC_SPECULAR = 2, ORC_BC_DIFFUSE = 3 };
/* Collision-frequency models for tau. */
enum { ORC_TAU_RHO = 0, ORC_TAU_HARDSPHERE2D = 1, ORC_TAU_PRESSURE = 2, ORC_TAU_CONST = 3 };
/* Time-step rules: the min form printed in Eq. (CFL-2D-part1) and the sum form. */
enum { ORC_CFL_MIN = 0, ORC_CFL_SUM = 1 };

typedef struct {
  int nx, ny;
  double x0, x1, y0, y1;
  int nv1, nv2;
  double v1min, v1max, v2min, v2max;
} orc_grid;

typedef struct {
  double nu;          /* ES-BGK parameter, -1 <= nu < 1 (Eq. mod-press-esbgk) */
  int tau_model;      /* ORC_TAU_* */
  double tau0;        /* scale factor of the tau model */
  int bc[4];          /* ORC_BC_* per side */
  double wall_T[4];   /* diffuse wall temperature per side */
  double wall_U[4];   /* diffuse wall tangential velocity per side */
  int wall_keep_es_term; /* 1: keep (G-M)/eps in wall-adjacent Ghat; 0: literal wall form */
} orc_params;

/* Advance (Q, G) by nsteps steps of size dt at Knudsen number eps; H receives the heat-flux
 * tensor of the last step.  Returns 0, or 4 if a non-physical state (rho<=0, T<=0, det<=0 or
 * a non-finite value) was met, or 1 on invalid arguments. */
int orc_step(const orc_grid* g, const orc_params* p, double* Q, double* G, double* H,
             double dt, double eps, int nsteps);

/* One step of the hybrid scheme with a heat-flux closure (the library's learned-closure
 * extension; the paper has no counterpart).  Cells with refresh[c] != 0 first set g^n to its
 * asymptotic-preserving limit Ghat(Q^n) (Eq. 5-97); then the step proceeds as orc_step, except
 * that cells with closure[c] != 0 skip the micro update (they keep g^n) and feed the heat flux
 * Hcl[4][ny][nx] to the macro step. */
int orc_step_closure(const orc_grid* g, const orc_params* p, double* Q, double* G, double* H,
                     double dt, double eps, const unsigned char* closure,
                     const unsigned char* refresh, const double* Hcl);
/* The 2D-2V manufactured solution of the convergence study (Section 6.1): f = phi(v) F(t, x, y),
 * phi = exp(-|v - (1,1)|^2) + 2 exp(-|v + (1,1)|^2), F = 2 - sin(2 pi (t-x)) cos(2 pi (t-y)).
 * orc_step_mms: nsteps steps starting at time t0 with the residual source S = f_t + v.grad f
 * - (tau/eps)(Gcal[f] - f) added to Ghat as (1/tau)(I - Pi_M)[S] and to the macro update as
 * dt int (1, v, v (x) v) S dv after the y transport (Eq. macro2d-split3b).
 * orc_mms_exact: the exact Q (cell-centre values) and g = (f - M[f])/eps at the nodes, time t.
 * Both return 0, 4 (non-physical) or 1 (invalid arguments). */
int orc_step_mms(const orc_grid* g, const orc_params* p, double* Q, double* G, double* H,
                 double dt, double eps, int nsteps, double t0);
int orc_mms_exact(const orc_grid* g, const orc_params* p, double t, double eps, double* Q,
                  double* G);
/* The residual S at the velocity nodes ([nv2][nv1]) of the point (x, y), time t. */
int orc_mms_source(const orc_grid* g, const orc_params* p, double eps, double t, double x,
                   double y, double* S);
/* ---- 1D-1V micro-macro scheme for Boltzmann-BGK (Sections 3 and 4) ------------------------
 * Q[3][nx] = (rho, rho u, E), E = rho T / 2 + rho u^2 / 2; G[nx][nv]; H[nx] = (eps/2) dv sum v^3 G.
 * Boundary kinds ORC_BC_PERIODIC or ORC_BC_EXTRAP on sides 0 (left) and 1 (right). */
typedef struct {
  int nx;
  double x0, x1;
  int nv;
  double vmin, vmax;
} orc1d_grid;
enum { ORC1D_TAU_HARDSPHERE = 0, ORC1D_TAU_CONST = 1 };
typedef struct {
  int bc[2];
  int tau_model; /* ORC1D_TAU_HARDSPHERE: tau = (16/5) sqrt(T / (2 pi)) (Eq. collision_parameter_1d) */
  double tau0;   /* ORC1D_TAU_CONST */
} orc1d_params;
/* nsteps steps (Eqs. 5-19 ... 5-27); with mms != 0 the manufactured source of Section 4.1 at
 * t^n = t0 + n dt enters Ghat as (1/tau)(I - Pi_M)[S] and the macro update as the printed
 * dt pi^{3/2} cos(2 pi (x - t^n)) (-8, 11, -7).  Returns 0, 4 (non-physical) or 1. */
int orc1d_step(const orc1d_grid* g, const orc1d_params* p, double* Q, double* G, double* H,
               double dt, double eps, int nsteps, int mms, double t0);
/* Exact Q and g of the 1D manufactured solution at time t. */
int orc1d_mms_exact(const orc1d_grid* g, double t, double eps, double* Q, double* G);
/* dt = CFL dx / max|v|, N = ceil(t_final / dt), dt reset to t_final / N (Section 3.2). */
double orc1d_dt(const orc1d_grid* g, double cfl, double t_final, int* nsteps_out);
/* Global time step (Eq. CFL-2D-part1/part2 and the 1D rule of Section 3.2). */
double orc_dt_for_cfl(const orc_grid* g, double cfl, double t_final, int form, int* nsteps_out);

/* Conservative state Q [6][ncell] from primitive fields rho, u1, u2, T [ncell] with an isotropic
 * temperature tensor T I: Q = (rho, rho u1, rho u2, E11, E12, E22), E = rho (u (x) u + T I), the
 * energy tensor of Section 2 (ES-BGK operator) as the paper's examples start (Section 6, g = 0).
 * Returns -1 (Q untouched) if some rho or T is not positive and finite, or u is not finite. */
int orc_q_from_prim(int ncell, const double* rho, const double* u1, const double* u2,
                    const double* T, double* Q);

/* ---- building blocks exposed for the pin tests ---- */

/* Primitive variables of one cell: out = (rho, u1, u2, T, P11, P12, P22, tau). */
int orc_prims(const orc_params* p, const double q[6], double out[8]);

/* Maxwellian M and ES Gaussian G of one cell's moments q evaluated at velocity (v1, v2). */
void orc_maxwellian_gauss(const orc_params* p, const double q[6], double v1, double v2,
                          double* M, double* Gs);

/* Pi_M[F] on the velocity grid for a Maxwellian with (rho, u1, u2, T), Eqs. (5-33), (5-33-plus)
 * with the midpoint rule of Section 5.3.  F and out are [nv2][nv1]. */
void orc_project(const orc_grid* g, double rho, double u1, double u2, double T,
                 const double* F, double* out);

/* Half-range KFVS fluxes of the Gaussian with moments q along direction dir (1 or 2):
 * Fp = int_{v_dir>0} v_dir m G dv, Fm = int_{v_dir<0} v_dir m G dv  (Eq. flux-2D-1/2). */
void orc_kfvs_half(const double q[6], int dir, double Fp[6], double Fm[6]);

/* Wall density factor R_a^{+-} of Eq. (twodim_wall_densities_1); sign = +1 or -1. */
double orc_wall_R(double ua, double Taa, double Tw, int sign);

/* TR-BDF2 mixing factor W of the macro collision half step (Section 5.4). */
double orc_trbdf2_W(double tau, double nu, double eps, double dt);

/* Ghat of Eq. (5-97) (interior) / the wall form of Section 6.3 for every cell, from Q alone.
 * Ghat is [ny][nx][nv2][nv1].  Returns 0 or 4 (non-physical). */
int orc_ghat(const orc_grid* g, const orc_params* p, const double* Q, double eps, double* Ghat);

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
