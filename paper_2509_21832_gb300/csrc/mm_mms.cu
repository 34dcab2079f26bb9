// Manufactured-solution harness of the paper's 2D convergence study (Section 6.1, "Method of
// Manufactured Solutions Example"): f = phi(v) F(t, x, y) with
//   phi = exp(-(v1-1)^2 - (v2-1)^2) + 2 exp(-(v1+1)^2 - (v2+1)^2),
//   F   = 2 - sin(2 pi (t-x)) cos(2 pi (t-y)),
// moments pi F (3, -1, -1, 9/2, 3, 9/2) (rho, rho u, E), and the residual
//   S = f_t + v1 f_x + v2 f_y - (tau/eps)(Gcal[f] - f),
// which the step adds to Ghat as (1/tau^n)(I - Pi_M)[S] (so to g^{n+1} as
// dt/(eps + dt tau^n) (I - Pi_M)[S]) and to the macro update as dt int (1, v, v (x) v) S dv
// after the y transport (Eq. macro2d-split3b).
//
// u and the temperature tensor of f are constant; only rho = 3 pi F varies, so
// Gcal[f] = F gam(v) and phi(v) are velocity tables computed once per context.
#include <cmath>

#include "mm_body_macro.cuh"
#include "mm_body_micro.cuh"

namespace mmk {

namespace {

constexpr double kPiM = 3.14159265358979323846;

__device__ __forceinline__ void mms_q(double t, double x, double y, double q[6]) {
  const double pf = kPiM * (2.0 - sin(2.0 * kPiM * (t - x)) * cos(2.0 * kPiM * (t - y)));
  q[0] = 3.0 * pf;
  q[1] = -pf;
  q[2] = -pf;
  q[3] = 4.5 * pf;
  q[4] = 3.0 * pf;
  q[5] = 4.5 * pf;
}

// Inverse ES tensor and its determinant for the moments q (Eq. 2-19).
__device__ __forceinline__ void es_tensor(const KParams& p, const double q[6], double& Ti11,
                                          double& Ti12, double& Ti22, double& det, double& T) {
  const double rho = q[0], u1 = q[1] / rho, u2 = q[2] / rho;
  const double t11 = (q[3] - rho * u1 * u1) / rho;
  const double t12 = (q[4] - rho * u1 * u2) / rho;
  const double t22 = (q[5] - rho * u2 * u2) / rho;
  T = 0.5 * (t11 + t22);
  const double s11 = (1.0 - p.nu) * T + p.nu * t11;
  const double s12 = p.nu * t12;
  const double s22 = (1.0 - p.nu) * T + p.nu * t22;
  det = s11 * s22 - s12 * s12;
  Ti11 = s22 / det;
  Ti12 = -s12 / det;
  Ti22 = s11 / det;
}

// Velocity tables: phi[e] and gam[e] = Gcal[f]/F at node e = l nv1 + k.
__global__ void k_mms_tables(double* __restrict__ phi, double* __restrict__ gam, KGrid g,
                             KParams p) {
  const int nv = g.nv1 * g.nv2;
  // the moments of f at F = 1
  const double q[6] = {3.0 * kPiM, -kPiM, -kPiM, 4.5 * kPiM, 3.0 * kPiM, 4.5 * kPiM};
  double Ti11, Ti12, Ti22, det, T;
  es_tensor(p, q, Ti11, Ti12, Ti22, det, T);
  const double u1 = q[1] / q[0], u2 = q[2] / q[0];
  const double K = q[0] / (2.0 * kPiM * sqrt(det));
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += gridDim.x * blockDim.x) {
    const int k = e % g.nv1, l = e / g.nv1;
    const double v1 = fma(k + 0.5, g.dv1, g.v1min), v2 = fma(l + 0.5, g.dv2, g.v2min);
    phi[e] = exp(-(v1 - 1.0) * (v1 - 1.0) - (v2 - 1.0) * (v2 - 1.0)) +
             2.0 * exp(-(v1 + 1.0) * (v1 + 1.0) - (v2 + 1.0) * (v2 + 1.0));
    const double c1 = v1 - u1, c2 = v2 - u2;
    gam[e] = K * exp(-0.5 * (Ti11 * c1 * c1 + 2.0 * Ti12 * c1 * c2 + Ti22 * c2 * c2));
  }
}

// Exact state at time t: Q (cell-centre values) and g = (f - M[f]) / eps at the nodes.
__global__ void k_mms_exact(double* __restrict__ Q, double* __restrict__ G,
                            const double* __restrict__ phi, KGrid g, KParams p, double t,
                            double eps, double x0, double y0) {
  const int nc = g.nx * g.ny, nv = g.nv1 * g.nv2;
  const int cell = blockIdx.x;
  const int i = cell % g.nx, j = cell / g.nx;
  const double x = x0 + (i + 0.5) * g.dx, y = y0 + (j + 0.5) * g.dy;
  double q[6];
  mms_q(t, x, y, q);
  if (threadIdx.x < 6) Q[threadIdx.x * nc + cell] = q[threadIdx.x];
  const double F = q[0] / (3.0 * kPiM);
  const double rho = q[0], u1 = q[1] / rho, u2 = q[2] / rho;
  const double T = 0.5 * ((q[3] - rho * u1 * u1) + (q[5] - rho * u2 * u2)) / rho;
  const double mu = rho / (2.0 * kPiM * T);
  const double ie = 1.0 / eps;
  double* Gc = G + (size_t)cell * nv;
  for (int e = threadIdx.x; e < nv; e += blockDim.x) {
    const int k = e % g.nv1, l = e / g.nv1;
    const double c1 = fma(k + 0.5, g.dv1, g.v1min) - u1, c2 = fma(l + 0.5, g.dv2, g.v2min) - u2;
    Gc[e] = (phi[e] * F - mu * exp(-(c1 * c1 + c2 * c2) / (2.0 * T))) * ie;
  }
}

// Per cell: the source term of g^{n+1}, dt/(eps + dt tau^n) (I - Pi_M)[S], into src_g (the
// layout of G), and int (1, v1, v2, v1^2, v1 v2, v2^2) S dv into src_q [6][ny][nx].  Pi_M uses
// the Maxwellian of Q^n (prims) and the midpoint moments of Section 5.3.
__global__ void k_mms_source(const double* __restrict__ prim, const double* __restrict__ phi,
                             const double* __restrict__ gam, double* __restrict__ src_g,
                             double* __restrict__ src_q, KGrid g, KParams p, double t, double dt,
                             double eps, double x0, double y0) {
  extern __shared__ double sm[];
  double* red = sm;                      // block_sum4 scratch (kRed doubles)
  double* e2t = sm + micro_body::kRed;   // e2[l] of the Maxwellian of Q^n
  double* e1t = e2t + g.nv2;             // e1[k]
  const int nc = g.nx * g.ny, nv = g.nv1 * g.nv2;
  const int cell = blockIdx.x;
  const int i = cell % g.nx, j = cell / g.nx;
  const double x = x0 + (i + 0.5) * g.dx, y = y0 + (j + 0.5) * g.dy;
  const double w = 2.0 * kPiM;
  const double s1 = sin(w * (t - x)), c1x = cos(w * (t - x));
  const double s2 = sin(w * (t - y)), c2y = cos(w * (t - y));
  const double F = 2.0 - s1 * c2y;
  const double Ft = -w * c1x * c2y + w * s1 * s2, Fx = w * c1x * c2y, Fy = -w * s1 * s2;
  double q[6];
  mms_q(t, x, y, q);
  const double Te = 0.5 * ((q[3] - q[1] * q[1] / q[0]) + (q[5] - q[2] * q[2] / q[0])) / q[0];
  const double ctau = macro_body::tau_of(p, q[0], Te) / eps;  // tau/eps of the exact state
  const double u1 = prim[P_U1 * nc + cell], u2 = prim[P_U2 * nc + cell];
  const double inv2T = prim[P_INV2T * nc + cell], iT = prim[P_IT * nc + cell];
  const double tau = prim[P_TAU * nc + cell];
  for (int l = threadIdx.x; l < g.nv2; l += blockDim.x) {
    const double c2 = fma(l + 0.5, g.dv2, g.v2min) - u2;
    e2t[l] = expd(-c2 * c2 * inv2T);
  }
  for (int k = threadIdx.x; k < g.nv1; k += blockDim.x) {
    const double c1 = fma(k + 0.5, g.dv1, g.v1min) - u1;
    e1t[k] = expd(-c1 * c1 * inv2T);
  }
  __syncthreads();
  // pass 1: moments of S against the projector basis (c = v - u^n) and the macro basis
  double a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0}, cm[4] = {0, 0, 0, 0};
  for (int e = threadIdx.x; e < nv; e += blockDim.x) {
    const int k = e % g.nv1, l = e / g.nv1;
    const double v1 = fma(k + 0.5, g.dv1, g.v1min), v2 = fma(l + 0.5, g.dv2, g.v2min);
    const double ph = phi[e];
    const double S = ph * (Ft + v1 * Fx + v2 * Fy) - ctau * (gam[e] * F - ph * F);
    const double c1 = v1 - u1, c2 = v2 - u2;
    a[0] += S;
    a[1] = fma(c1, S, a[1]);
    a[2] = fma(c2, S, a[2]);
    a[3] = fma(c1 * c1 + c2 * c2, S, a[3]);
    b[0] = fma(v1, S, b[0]);
    b[1] = fma(v2, S, b[1]);
    b[2] = fma(v1 * v1, S, b[2]);
    b[3] = fma(v1 * v2, S, b[3]);
    cm[0] = fma(v2 * v2, S, cm[0]);
  }
  micro_body::block_sum4(a, red);
  micro_body::block_sum4(b, red);
  micro_body::block_sum4(cm, red);
  const double dv = g.dv1 * g.dv2;
  if (threadIdx.x == 0) {
    src_q[cell] = dv * a[0];
    src_q[nc + cell] = dv * b[0];
    src_q[2 * nc + cell] = dv * b[1];
    src_q[3 * nc + cell] = dv * b[2];
    src_q[4 * nc + cell] = dv * b[3];
    src_q[5 * nc + cell] = dv * cm[0];
  }
  // Pi_M[S] = (dv / (2 pi T)) e1 e2 (b0 + b1 c1 + b2 c2 + gm |c|^2)
  const double b0 = fma(-a[3], inv2T, 2.0 * a[0]);
  const double b1 = a[1] * iT, b2 = a[2] * iT;
  const double gm = fma(0.25 * a[3], iT * iT, -a[0] * inv2T);
  const double kp = dv / (2.0 * kPiM) * iT;
  const double wgt = dt / (eps + dt * tau);
  double* Sg = src_g + (size_t)cell * nv;
  for (int e = threadIdx.x; e < nv; e += blockDim.x) {
    const int k = e % g.nv1, l = e / g.nv1;
    const double v1 = fma(k + 0.5, g.dv1, g.v1min), v2 = fma(l + 0.5, g.dv2, g.v2min);
    const double ph = phi[e];
    const double S = ph * (Ft + v1 * Fx + v2 * Fy) - ctau * (gam[e] * F - ph * F);
    const double c1 = v1 - u1, c2 = v2 - u2;
    const double PS = kp * e1t[k] * e2t[l] * fma(gm, c1 * c1 + c2 * c2, fma(b2, c2, fma(b1, c1, b0)));
    Sg[e] = wgt * (S - PS);
  }
}

// Per-cell partial sums of |Q - Qe|^2, |Qe|^2, |G - ge|^2, |ge|^2 at time t.
__global__ void k_mms_errors(const double* __restrict__ Q, const double* __restrict__ G,
                             const double* __restrict__ phi, double* __restrict__ sums, KGrid g,
                             KParams p, double t, double eps, double x0, double y0) {
  extern __shared__ double sm[];
  const int nc = g.nx * g.ny, nv = g.nv1 * g.nv2;
  const int cell = blockIdx.x;
  const int i = cell % g.nx, j = cell / g.nx;
  const double x = x0 + (i + 0.5) * g.dx, y = y0 + (j + 0.5) * g.dy;
  double q[6];
  mms_q(t, x, y, q);
  const double F = q[0] / (3.0 * kPiM);
  const double rho = q[0], u1 = q[1] / rho, u2 = q[2] / rho;
  const double T = 0.5 * ((q[3] - rho * u1 * u1) + (q[5] - rho * u2 * u2)) / rho;
  const double mu = rho / (2.0 * kPiM * T);
  const double ie = 1.0 / eps;
  const double* Gc = G + (size_t)cell * nv;
  double s[4] = {0, 0, 0, 0};
  for (int e = threadIdx.x; e < nv; e += blockDim.x) {
    const int k = e % g.nv1, l = e / g.nv1;
    const double c1 = fma(k + 0.5, g.dv1, g.v1min) - u1, c2 = fma(l + 0.5, g.dv2, g.v2min) - u2;
    const double ge = (phi[e] * F - mu * exp(-(c1 * c1 + c2 * c2) / (2.0 * T))) * ie;
    const double d = Gc[e] - ge;
    s[2] = fma(d, d, s[2]);
    s[3] = fma(ge, ge, s[3]);
  }
  micro_body::block_sum4(s, sm);
  if (threadIdx.x == 0) {
    double dq = 0.0, qq = 0.0;
    for (int m = 0; m < 6; ++m) {
      const double d = Q[m * nc + cell] - q[m];
      dq += d * d;
      qq += q[m] * q[m];
    }
    sums[cell] = dq;
    sums[nc + cell] = qq;
    sums[2 * nc + cell] = s[2];
    sums[3 * nc + cell] = s[3];
  }
}

int mms_threads(const KGrid& g) {
  const int nv = g.nv1 * g.nv2;
  return nv >= 256 ? 256 : (nv + 31) / 32 * 32;
}

}  // namespace

void launch_mms_tables(double* phi, double* gam, const KGrid& g, const KParams& p,
                       cudaStream_t s) {
  k_mms_tables<<<152, 256, 0, s>>>(phi, gam, g, p);
}

void launch_mms_exact(double* Q, double* G, const double* phi, const KGrid& g, const KParams& p,
                      double t, double eps, double x0, double y0, cudaStream_t s) {
  k_mms_exact<<<g.nx * g.ny, mms_threads(g), 0, s>>>(Q, G, phi, g, p, t, eps, x0, y0);
}

void launch_mms_source(const double* prim, const double* phi, const double* gam, double* src_g,
                       double* src_q, const KGrid& g, const KParams& p, double t, double dt,
                       double eps, double x0, double y0, cudaStream_t s) {
  const size_t smem = sizeof(double) * (micro_body::kRed + g.nv1 + g.nv2);
  k_mms_source<<<g.nx * g.ny, mms_threads(g), smem, s>>>(prim, phi, gam, src_g, src_q, g, p, t,
                                                        dt, eps, x0, y0);
}

void launch_mms_errors(const double* Q, const double* G, const double* phi, double* sums,
                       const KGrid& g, const KParams& p, double t, double eps, double x0,
                       double y0, cudaStream_t s) {
  k_mms_errors<<<g.nx * g.ny, mms_threads(g), sizeof(double) * micro_body::kRed, s>>>(
      Q, G, phi, sums, g, p, t, eps, x0, y0);
}

}  // namespace mmk
