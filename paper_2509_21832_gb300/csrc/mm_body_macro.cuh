// Device bodies of the per-cell kernels (one thread per spatial cell per call), shared by the
// single-problem kernels and the batched persistent kernels.
#pragma once

#include <cmath>

#include "mm_erf.cuh"
#include "mm_exp.cuh"
#include "mm_internal.cuh"

// Pointer qualifier of the device bodies: __restrict__ by default; a translation unit whose
// kernel reads data that other CTAs of the same launch wrote defines MMK_R as empty before
// including this header, so that no load of the bodies may take the non-coherent read-only path.
#ifndef MMK_R
#define MMK_R __restrict__
#endif

namespace mmk {
namespace macro_body {


constexpr double kPi = 3.14159265358979323846;
constexpr double kC25 = 0.436;
constexpr double kInvSqrtPi = 0.56418958354775628695;  // 1/sqrt(pi)
constexpr double kInv2Pi = 0.15915494309189533577;     // 1/(2 pi)

__device__ __forceinline__ double tau_of(const KParams& p, double rho, double T) {
  switch (p.tau_model) {
    case MM_TAU_RHO: return p.tau0 * rho;
    case MM_TAU_HARDSPHERE2D: return 3.0 * kPi * kC25 * rho / (sqrt(2.0) * (1.0 - p.nu));
    case MM_TAU_PRESSURE: return p.tau0 * rho * T;
    default: return p.tau0;
  }
}

__device__ __forceinline__ void load_q(const double* Q, int nc, int c, double q[6]) {
#pragma unroll
  for (int m = 0; m < 6; ++m) q[m] = Q[m * nc + c];
}

// Primitive quantities of a moment vector; returns false for a non-physical state.
__device__ __forceinline__ bool prim6(const double q[6], double& rho, double& u1, double& u2,
                                      double& P11, double& P12, double& P22, double& ir) {
  rho = q[0];
  ir = 1.0 / rho;
  u1 = q[1] * ir;
  u2 = q[2] * ir;
  P11 = q[3] - rho * u1 * u1;
  P12 = q[4] - rho * u1 * u2;
  P22 = q[5] - rho * u2 * u2;
  return rho > 0.0 && P11 > 0.0 && P22 > 0.0 && P11 * P22 - P12 * P12 > 0.0 && isfinite(u1) &&
         isfinite(u2) && isfinite(P12) && isfinite(P11 + P22);
}

// Collision half step (Section 5.4): P <- (1/2)[[1+W,0,1-W],[0,2W,0],[1-W,0,1+W]] P with the
// TR-BDF2 factor W of tau(q); rho and rho u unchanged; E = rho u (x) u + P.  The step needs
// rho > 0 and T > 0; the input's pressure tensor need not be positive definite (with a
// manufactured source the state before the last half step can leave that set).
__device__ __forceinline__ bool coll_half(const KParams& p, const double q[6], double eps,
                                          double dt, double o[6], double& ir) {
  double rho, u1, u2, P11, P12, P22;
  prim6(q, rho, u1, u2, P11, P12, P22, ir);
  const double T = (P11 + P22) * (0.5 * ir);
  const bool ok = rho > 0.0 && T > 0.0 && isfinite(T) && isfinite(u1) && isfinite(u2) &&
                  isfinite(P12);
  const double a = tau_of(p, rho, T) * (1.0 - p.nu);
  const double W = (48.0 * eps * eps - 10.0 * a * eps * dt) /
                   (48.0 * eps * eps + 14.0 * a * eps * dt + (a * dt) * (a * dt));
  const double n11 = 0.5 * ((1.0 + W) * P11 + (1.0 - W) * P22);
  const double n12 = 0.5 * (2.0 * W * P12);
  const double n22 = 0.5 * ((1.0 - W) * P11 + (1.0 + W) * P22);
  o[0] = q[0];
  o[1] = q[1];
  o[2] = q[2];
  o[3] = rho * u1 * u1 + n11;
  o[4] = rho * u1 * u2 + n12;
  o[5] = rho * u2 * u2 + n22;
  return ok;
}

// a, b, J, K of Eq. (flux-2D-1) (dir 1) / (flux-2D-2) (dir 2) for the Gaussian with moments q:
// a = sqrt(2 th/pi) exp(-u^2/(2 th)), b = erf(u/sqrt(2 th)), th = P_nn/rho (the normal
// temperature); ir = 1/rho (from the caller, which has it already) and one reciprocal square
// root h = 1/sqrt(2 th), from which 1/P_nn = 2 h^2 / rho (a few ulp, in a correction term of J).
__device__ __forceinline__ void abJK(const double q[6], double ir, int dir, double& a, double& b,
                                     double J[6], double K[6]) {
  const double rho = q[0];
  const double u1 = q[1] * ir, u2 = q[2] * ir;
  const double P11 = q[3] - rho * u1 * u1;
  const double P12 = q[4] - rho * u1 * u2;
  const double P22 = q[5] - rho * u2 * u2;
  const double Pn = dir == 1 ? P11 : P22;
  const double un = dir == 1 ? u1 : u2;
  const double s2 = 2.0 * Pn * ir;  // 2 th
  const double h = rsqrt(s2);       // 1 / sqrt(2 th)
  const double iPn = 2.0 * (h * h) * ir;
  a = kInvSqrtPi * (s2 * h) * expd(-(un * h) * (un * h));
  b = erfd(un * h);
  if (dir == 1) {
    J[0] = rho;
    J[1] = rho * u1;
    J[2] = rho * u2;
    J[3] = rho * u1 * u1 + 2.0 * P11;
    J[4] = rho * u1 * u2 + 2.0 * P12;
    J[5] = rho * u2 * u2 + P22 + P12 * P12 * iPn;
    K[0] = rho * u1;
    K[1] = rho * u1 * u1 + P11;
    K[2] = rho * u1 * u2 + P12;
    K[3] = rho * u1 * u1 * u1 + 3.0 * u1 * P11;
    K[4] = rho * u1 * u1 * u2 + u2 * P11 + 2.0 * u1 * P12;
    K[5] = rho * u1 * u2 * u2 + u1 * P22 + 2.0 * u2 * P12;
  } else {
    J[0] = rho;
    J[1] = rho * u1;
    J[2] = rho * u2;
    J[3] = rho * u1 * u1 + P11 + P12 * P12 * iPn;
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

__device__ __forceinline__ void half_fluxes(const double q[6], double ir, int dir, double Fp[6],
                                            double Fm[6], double Kf[6]) {
  double a, b, J[6], K[6];
  abJK(q, ir, dir, a, b, J, K);
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    Fp[m] = 0.5 * (a * J[m] + (1.0 + b) * K[m]);
    Fm[m] = 0.5 * (-a * J[m] + (1.0 - b) * K[m]);
    Kf[m] = K[m];
  }
}

__device__ __forceinline__ void mirror_q(const double q[6], int dir, double o[6]) {
  o[0] = q[0];
  o[1] = dir == 1 ? -q[1] : q[1];
  o[2] = dir == 1 ? q[2] : -q[2];
  o[3] = q[3];
  o[4] = -q[4];
  o[5] = q[5];
}

// Eq. (twodim_wall_densities_1)
__device__ __forceinline__ double wall_R(double ua, double Taa, double Tw, double sgn) {
  return sqrt(Taa / Tw) * exp(-ua * ua / (2.0 * Taa)) +
         ua * sqrt(kPi / (2.0 * Tw)) * (erf(ua / sqrt(2.0 * Taa)) + sgn);
}

// Ghost state of a diffuse wall (Section 6.3): (rho_wall, wall velocity, T_wall I).
__device__ __forceinline__ void wall_ghost(const KParams& p, const double q[6], int side,
                                           double o[6]) {
  const double rho = q[0];
  const double u1 = q[1] / rho, u2 = q[2] / rho;
  const double P11 = q[3] - rho * u1 * u1;
  const double P22 = q[5] - rho * u2 * u2;
  const double Tw = p.wall_T[side], U = p.wall_U[side];
  double rw, g1, g2;
  if (side < 2) {
    rw = rho * wall_R(u1, P11 / rho, Tw, side == 0 ? -1.0 : 1.0);
    g1 = 0.0;
    g2 = U;
  } else {
    rw = rho * wall_R(u2, P22 / rho, Tw, side == 2 ? -1.0 : 1.0);
    g1 = U;
    g2 = 0.0;
  }
  o[0] = rw;
  o[1] = rw * g1;
  o[2] = rw * g2;
  o[3] = rw * (g1 * g1 + Tw);
  o[4] = rw * g1 * g2;
  o[5] = rw * (g2 * g2 + Tw);
}

// Heat-flux face value for component h at the face on side s of boundary cell value hc.
__device__ __forceinline__ double boundary_H(const KParams& p, double hc, double hper, int s,
                                             int h) {
  switch (p.bc[s]) {
    case MM_BC_PERIODIC: return 0.5 * (hc + hper);
    case MM_BC_EXTRAP: return hc;
    case MM_BC_SPECULAR: {
      const bool odd = s < 2 ? (h == 0 || h == 2) : (h == 1 || h == 3);
      return 0.5 * (hc + (odd ? -hc : hc));
    }
    default: return 0.5 * hc;
  }
}

// (u1, u2, T) of cell c from its moments.
__device__ __forceinline__ void uT_of(const double* Q, int nc, int c, double& u1, double& u2,
                                      double& T) {
  const double rho = Q[c];
  const double ir = 1.0 / rho;
  u1 = Q[nc + c] * ir;
  u2 = Q[2 * nc + c] * ir;
  const double P11 = Q[3 * nc + c] - rho * u1 * u1;
  const double P22 = Q[5 * nc + c] - rho * u2 * u2;
  T = (P11 + P22) * (0.5 * ir);
}

// (u1, u2, T) of cell c into its per-cell fields (the values uT_of gives, bit for bit), so that
// the prims of its neighbours read them instead of recomputing them.
__device__ __forceinline__ void uT_body(const double* MMK_R Q, double* MMK_R prim,
                                        int nc, int c) {
  double u1, u2, T;
  uT_of(Q, nc, c, u1, u2, T);
  prim[P_U1 * nc + c] = u1;
  prim[P_U2 * nc + c] = u2;
  prim[P_T * nc + c] = T;
}

// (u1, u2, T) across side s of cell (i, j) for the centred differences of Eq. (5-97more): the
// neighbour (periodic wrap; from its moments, or from its per-cell fields when FROM_PRIM), the
// cell itself (extrapolation; diffuse-wall cells do not use these values), or the mirrored ghost
// (specular: normal velocity negated).
template <bool FROM_PRIM = false>
__device__ __forceinline__ void side_uT(const double* Q, const double* prim, const KGrid& g,
                                        const KParams& p, int nc, int i, int j, int s, double cu1,
                                        double cu2, double cT, double& u1, double& u2,
                                        double& T) {
  int ni = i + (s == 0 ? -1 : s == 1 ? 1 : 0);
  int nj = j + (s == 2 ? -1 : s == 3 ? 1 : 0);
  bool inside = ni >= 0 && ni < g.nx && nj >= 0 && nj < g.ny;
  if (!inside && p.bc[s] == MM_BC_PERIODIC) {
    ni = (ni + g.nx) % g.nx;
    nj = (nj + g.ny) % g.ny;
    inside = true;
  }
  if (inside) {
    const int n = nj * g.nx + ni;
    if (FROM_PRIM) {
      u1 = prim[P_U1 * nc + n];
      u2 = prim[P_U2 * nc + n];
      T = prim[P_T * nc + n];
    } else {
      uT_of(Q, nc, n, u1, u2, T);
    }
  } else if (p.bc[s] == MM_BC_SPECULAR) {
    u1 = s < 2 ? -cu1 : cu1;
    u2 = s < 2 ? cu2 : -cu2;
    T = cT;
  } else {
    u1 = cu1;
    u2 = cu2;
    T = cT;
  }
}

// Per-cell fields of cell c.  FROM_PRIM: the neighbours' (u1, u2, T) are already in prim (written
// by uT_body over all cells); otherwise they are recomputed from Q.  ieps = 1/eps.
template <bool FROM_PRIM = false>
__device__ __forceinline__ void prims_body(const double* MMK_R Q, double* MMK_R prim,
                        float* MMK_R primf, KGrid g, KParams p, double dt, double eps,
                        double ieps, int* MMK_R err, int c) {
  const int nc = g.nx * g.ny;
  const int i = c % g.nx, j = c / g.nx;
  const double rho = Q[c];
  const double ir = 1.0 / rho;
  // the cell's own (u1, u2, T): as its neighbours see them
  const double u1 = FROM_PRIM ? prim[P_U1 * nc + c] : Q[nc + c] * ir;
  const double u2 = FROM_PRIM ? prim[P_U2 * nc + c] : Q[2 * nc + c] * ir;
  const double P11 = Q[3 * nc + c] - rho * u1 * u1;
  const double P12 = Q[4 * nc + c] - rho * u1 * u2;
  const double P22 = Q[5 * nc + c] - rho * u2 * u2;
  const double T = FROM_PRIM ? prim[P_T * nc + c] : (P11 + P22) * (0.5 * ir);
  const double nu = p.nu;
  const double t11 = P11 * ir, t12 = P12 * ir, t22 = P22 * ir;
  const double s11 = (1.0 - nu) * T + nu * t11;
  const double s12 = nu * t12;
  const double s22 = (1.0 - nu) * T + nu * t22;
  const double det = s11 * s22 - s12 * s12;
  const bool ok = rho > 0.0 && P11 > 0.0 && P22 > 0.0 && t11 * t22 - t12 * t12 > 0.0 &&
                  det > 0.0 && T > 0.0 && isfinite(u1) && isfinite(u2) && isfinite(P12) &&
                  isfinite(T);
  if (!ok) atomicOr(err, ERR_NONPHYS_PRIM);
  const double tau = tau_of(p, rho, T);
  const double idet = 1.0 / det;
  const double KG = rho * kInv2Pi * rsqrt(det);
  prim[P_RHO * nc + c] = rho;
  if (!FROM_PRIM) {  // else already there, read by the neighbours
    prim[P_U1 * nc + c] = u1;
    prim[P_U2 * nc + c] = u2;
    prim[P_T * nc + c] = T;
  }
  prim[P_TAU * nc + c] = tau;
  prim[P_TI11 * nc + c] = s22 * idet;
  prim[P_TI12 * nc + c] = -s12 * idet;
  prim[P_TI22 * nc + c] = s11 * idet;
  prim[P_KG * nc + c] = KG;
  prim[P_TH11 * nc + c] = t11;
  prim[P_TH22 * nc + c] = t22;

  // discrete strain and temperature gradient, Eqs. (5-97), (5-97more)
  double uL1, uL2, TL, uR1, uR2, TR, uB1, uB2, TB, uT1, uT2, TT;
  side_uT<FROM_PRIM>(Q, prim, g, p, nc, i, j, 0, u1, u2, T, uL1, uL2, TL);
  side_uT<FROM_PRIM>(Q, prim, g, p, nc, i, j, 1, u1, u2, T, uR1, uR2, TR);
  side_uT<FROM_PRIM>(Q, prim, g, p, nc, i, j, 2, u1, u2, T, uB1, uB2, TB);
  side_uT<FROM_PRIM>(Q, prim, g, p, nc, i, j, 3, u1, u2, T, uT1, uT2, TT);
  const double dTdx = (0.5 * (TR + T) - 0.5 * (T + TL)) * g.idx;
  const double dTdy = (0.5 * (TT + T) - 0.5 * (T + TB)) * g.idy;
  const double Dxu1 = (uR1 - uL1) * 0.5, Dxu2 = (uR2 - uL2) * 0.5;
  const double Dyu1 = (uT1 - uB1) * 0.5, Dyu2 = (uT2 - uB2) * 0.5;
  const double sg11 = Dxu1 * g.idx - Dyu2 * g.idy;
  const double sg12 = Dyu1 * g.idy + Dxu2 * g.idx;

  const double iT = 1.0 / T;
  const double kap = dt * g.dv1 * g.dv2 * kInv2Pi * iT;
  const double iden = 1.0 / (eps + dt * tau);
  const double om1 = eps * iden;
  const double om2 = dt * tau * iden;
  const double mu = rho * kInv2Pi * iT;
  const double wt = dt * iden * mu;  // om2 mu / tau
  const double h2T2 = 0.5 * iT * iT;
  const double gam0 = om2 * ieps * KG;
  const double ome = om2 * mu * ieps;
  const double w[9] = {wt * (-2.0 * dTdx * iT), wt * (0.5 * sg11 * iT), wt * (h2T2 * dTdx),
                       wt * (-2.0 * dTdy * iT), wt * (sg12 * iT),       wt * (h2T2 * dTdy),
                       wt * (-0.5 * sg11 * iT), wt * (h2T2 * dTdx),     wt * (h2T2 * dTdy)};
  prim[P_IT * nc + c] = iT;
  prim[P_INV2T * nc + c] = 0.5 * iT;
  prim[P_KAP * nc + c] = kap;
  prim[P_OM1 * nc + c] = om1;
  prim[P_OM1KAP * nc + c] = om1 * kap;
  prim[P_GAM0 * nc + c] = gam0;
  prim[P_OME * nc + c] = ome;
  // B:sigma + C.grad T = p0 + p1 c2 + p2 c2^2 + p3 c2^3 (Eq. 5-69) with
  // p0 = (s11/2T) c1^2 + (Tx/2T^2) c1^3 - (2Tx/T) c1, p1 = (s12/T) c1 + (Ty/2T^2) c1^2 - 2Ty/T,
  // p2 = -s11/2T + (Tx/2T^2) c1, p3 = Ty/2T^2; stored times om2 mu / tau
  for (int m = 0; m < 9; ++m) prim[(P_W01 + m) * nc + c] = w[m];
  if (primf) {
    primf[F_U1 * nc + c] = (float)u1;
    primf[F_U2 * nc + c] = (float)u2;
    primf[F_INV2T * nc + c] = (float)(0.5 * iT);
    primf[F_IT * nc + c] = (float)iT;
    primf[F_KAP * nc + c] = (float)kap;
    primf[F_OM1 * nc + c] = (float)om1;
    primf[F_OM1KAP * nc + c] = (float)(om1 * kap);
    primf[F_GAM0 * nc + c] = (float)gam0;
    primf[F_OME * nc + c] = (float)ome;
    primf[F_TI11H * nc + c] = (float)(0.5 * s22 * idet);
    primf[F_TI12 * nc + c] = (float)(-s12 * idet);
    primf[F_TI22H * nc + c] = (float)(0.5 * s11 * idet);
    for (int m = 0; m < 9; ++m) primf[(F_W01 + m) * nc + c] = (float)w[m];
  }
}

// The FP32 coefficients of cell c for the FP32-g phase-space kernels, the same quantities as
// prims_body's primf (neighbours' (u1, u2, T) from uT_body).  FP64, rounded once: the pressure,
// the ES tensor with its determinant, inverse and normalisation, 1/T and the projector scale, and
// the centred strain and temperature differences (the validity check and cancellation need it).
// FP32: the relaxation weights and the coefficients of the transport term, products of those
// rounded values.  No FP64 per-cell field is written besides uT_body's.
__device__ __forceinline__ void prims_f32_body(const double* MMK_R Q, const double* MMK_R prim,
                                               float* MMK_R primf, KGrid g, KParams p, double dt,
                                               double eps, int* MMK_R err, int c) {
  const int nc = g.nx * g.ny;
  const int i = c % g.nx, j = c / g.nx;
  const double rho = Q[c];
  const double ir = 1.0 / rho;
  const double u1 = prim[P_U1 * nc + c], u2 = prim[P_U2 * nc + c], T = prim[P_T * nc + c];
  const double P11 = Q[3 * nc + c] - rho * u1 * u1;
  const double P12 = Q[4 * nc + c] - rho * u1 * u2;
  const double P22 = Q[5 * nc + c] - rho * u2 * u2;
  const double nu = p.nu;
  const double t11 = P11 * ir, t12 = P12 * ir, t22 = P22 * ir;
  const double s11 = (1.0 - nu) * T + nu * t11;
  const double s12 = nu * t12;
  const double s22 = (1.0 - nu) * T + nu * t22;
  const double det = s11 * s22 - s12 * s12;
  const bool ok = rho > 0.0 && P11 > 0.0 && P22 > 0.0 && t11 * t22 - t12 * t12 > 0.0 &&
                  det > 0.0 && T > 0.0 && isfinite(u1) && isfinite(u2) && isfinite(P12) &&
                  isfinite(T);
  if (!ok) atomicOr(err, ERR_NONPHYS_PRIM);
  double uL1, uL2, TL, uR1, uR2, TR, uB1, uB2, TB, uT1, uT2, TT;
  side_uT<true>(Q, prim, g, p, nc, i, j, 0, u1, u2, T, uL1, uL2, TL);
  side_uT<true>(Q, prim, g, p, nc, i, j, 1, u1, u2, T, uR1, uR2, TR);
  side_uT<true>(Q, prim, g, p, nc, i, j, 2, u1, u2, T, uB1, uB2, TB);
  side_uT<true>(Q, prim, g, p, nc, i, j, 3, u1, u2, T, uT1, uT2, TT);
  const float dTdx = (float)((0.5 * (TR + T) - 0.5 * (T + TL)) * g.idx);
  const float dTdy = (float)((0.5 * (TT + T) - 0.5 * (T + TB)) * g.idy);
  const float sg11 = (float)((uR1 - uL1) * 0.5 * g.idx - (uT2 - uB2) * 0.5 * g.idy);
  const float sg12 = (float)((uT1 - uB1) * 0.5 * g.idy + (uR2 - uL2) * 0.5 * g.idx);
  // reciprocals through reciprocal square roots (a few FP64 ulp, far below the FP32 rounding
  // that follows; cheaper than divisions on the FP64 pipe)
  const double rsd = rsqrt(det), rsT = rsqrt(T);
  const double idet = rsd * rsd, iTd = rsT * rsT;
  const float KG = (float)(rho * kInv2Pi * rsd);
  const float iT = (float)iTd;
  const float kap = (float)(dt * g.dv1 * g.dv2 * kInv2Pi * iTd);
  const float tau = (float)tau_of(p, rho, T);
  // FP32 from here
  const float rhof = (float)rho, dtf = (float)dt, epsf = (float)eps;
  const float iden = 1.0f / fmaf(dtf, tau, epsf);
  const float om1 = epsf * iden;
  const float om2 = dtf * tau * iden;
  const float mu = rhof * (float)kInv2Pi * iT;
  const float wt = dtf * iden * mu;
  const float h2T2 = 0.5f * iT * iT;
  const float ieps = 1.0f / epsf;
  const float w[9] = {wt * (-2.0f * dTdx * iT), wt * (0.5f * sg11 * iT), wt * (h2T2 * dTdx),
                      wt * (-2.0f * dTdy * iT), wt * (sg12 * iT),        wt * (h2T2 * dTdy),
                      wt * (-0.5f * sg11 * iT), wt * (h2T2 * dTdx),      wt * (h2T2 * dTdy)};
  primf[F_U1 * nc + c] = (float)u1;
  primf[F_U2 * nc + c] = (float)u2;
  primf[F_INV2T * nc + c] = (float)(0.5 * iTd);
  primf[F_IT * nc + c] = iT;
  primf[F_KAP * nc + c] = kap;
  primf[F_OM1 * nc + c] = om1;
  primf[F_OM1KAP * nc + c] = om1 * kap;
  primf[F_GAM0 * nc + c] = om2 * ieps * KG;
  primf[F_OME * nc + c] = om2 * mu * ieps;
  primf[F_TI11H * nc + c] = (float)(0.5 * s22 * idet);
  primf[F_TI12 * nc + c] = (float)(-s12 * idet);
  primf[F_TI22H * nc + c] = (float)(0.5 * s11 * idet);
  for (int m = 0; m < 9; ++m) primf[(F_W01 + m) * nc + c] = w[m];
}

// Flux through the boundary face on side s of boundary cell state qc, given that cell's own
// half fluxes (Fp, Fm) and full flux K along the face normal.
__device__ __forceinline__ void boundary_face(const KParams& p, const double qc[6], int s,
                                              int dir, const double Fp[6], const double Fm[6],
                                              const double K[6], double F[6]) {
  if (p.bc[s] == MM_BC_EXTRAP) {
    for (int m = 0; m < 6; ++m) F[m] = K[m];
    return;
  }
  double gq[6], Gp[6], Gm[6], GK[6];
  if (p.bc[s] == MM_BC_SPECULAR) mirror_q(qc, dir, gq);
  else wall_ghost(p, qc, s, gq);
  half_fluxes(gq, 1.0 / gq[0], dir, Gp, Gm, GK);
  const bool low = s == 0 || s == 2;  // the ghost is the left / bottom state
  for (int m = 0; m < 6; ++m) F[m] = low ? Gp[m] + Fm[m] : Fp[m] + Gm[m];
}

// (1) collision half step with tau^n: Q^n -> Q*, and the x half fluxes of Q* (plus the fluxes
// through the non-periodic x boundary faces).
__device__ __forceinline__ void macro_x1_body(const double* MMK_R Qn, MacroBufs mb, KGrid g, KParams p,
                           double dt, double eps, int* MMK_R err, int c) {
  const int nc = g.nx * g.ny;
  const int i = c % g.nx, j = c / g.nx;
  double q[6], qs[6];
  load_q(Qn, nc, c, q);
  double ir;  // 1/rho: the collision half step leaves rho unchanged
  const bool ok = coll_half(p, q, eps, dt, qs, ir);
  double Fp[6], Fm[6], K[6];
  half_fluxes(qs, ir, 1, Fp, Fm, K);
  for (int m = 0; m < 6; ++m) {
    mb.Q1[m * nc + c] = qs[m];
    mb.FX[m * nc + c] = Fp[m];
    mb.FX[(6 + m) * nc + c] = Fm[m];
  }
  double F[6];
  if (i == 0 && p.bc[0] != MM_BC_PERIODIC) {
    boundary_face(p, qs, 0, 1, Fp, Fm, K, F);
    for (int m = 0; m < 6; ++m) mb.BX[m * g.ny + j] = F[m];
  }
  if (i == g.nx - 1 && p.bc[1] != MM_BC_PERIODIC) {
    boundary_face(p, qs, 1, 1, Fp, Fm, K, F);
    for (int m = 0; m < 6; ++m) mb.BX[(6 + m) * g.ny + j] = F[m];
  }
  if (!ok) atomicOr(err, ERR_NONPHYS_MACRO);
}

// (2) x transport (Eq. 5-103, first line): Q* -> Q**, then the y half fluxes of Q**.
__device__ __forceinline__ void macro_x2_body(const double* MMK_R H, MacroBufs mb, KGrid g, KParams p,
                           double dt, int* MMK_R err, int c) {
  const int nc = g.nx * g.ny;
  const int i = c % g.nx, j = c / g.nx;
  const int cl = j * g.nx + (i > 0 ? i - 1 : g.nx - 1);
  const int cr = j * g.nx + (i < g.nx - 1 ? i + 1 : 0);
  double FL[6], FR[6];
  for (int m = 0; m < 6; ++m) {
    FL[m] = (i > 0 || p.bc[0] == MM_BC_PERIODIC) ? mb.FX[m * nc + cl] + mb.FX[(6 + m) * nc + c]
                                                 : mb.BX[m * g.ny + j];
    FR[m] = (i < g.nx - 1 || p.bc[1] == MM_BC_PERIODIC)
                ? mb.FX[m * nc + c] + mb.FX[(6 + m) * nc + cr]
                : mb.BX[(6 + m) * g.ny + j];
  }
  // heat-flux faces: components (H111, H112, H122) enter (E11, E12, E22)
  double dH[3];
  for (int h = 0; h < 3; ++h) {
    const double hc = H[h * nc + c];
    const double hl = H[h * nc + cl];
    const double hr = H[h * nc + cr];
    const double HL = i > 0 ? 0.5 * (hc + hl) : boundary_H(p, hc, hl, 0, h);
    const double HR = i < g.nx - 1 ? 0.5 * (hr + hc) : boundary_H(p, hc, hr, 1, h);
    dH[h] = HR - HL;
  }
  const double lam = dt * g.idx;
  double q2[6];
  for (int m = 0; m < 6; ++m) {
    double v = mb.Q1[m * nc + c] - lam * (FR[m] - FL[m]);
    if (m >= 3) v -= dt * (dH[m - 3] * g.idx);
    q2[m] = v;
    mb.Q2[m * nc + c] = v;
  }
  double r0, r1, r2, r3, r4, r5, ir;
  const bool ok = prim6(q2, r0, r1, r2, r3, r4, r5, ir);
  double Fp[6], Fm[6], K[6];
  half_fluxes(q2, ir, 2, Fp, Fm, K);
  for (int m = 0; m < 6; ++m) {
    mb.FY[m * nc + c] = Fp[m];
    mb.FY[(6 + m) * nc + c] = Fm[m];
  }
  double F[6];
  if (j == 0 && p.bc[2] != MM_BC_PERIODIC) {
    boundary_face(p, q2, 2, 2, Fp, Fm, K, F);
    for (int m = 0; m < 6; ++m) mb.BY[m * g.nx + i] = F[m];
  }
  if (j == g.ny - 1 && p.bc[3] != MM_BC_PERIODIC) {
    boundary_face(p, q2, 3, 2, Fp, Fm, K, F);
    for (int m = 0; m < 6; ++m) mb.BY[(6 + m) * g.nx + i] = F[m];
  }
  if (!ok) atomicOr(err, ERR_NONPHYS_MACRO);
}

// (3) y transport (Eq. 5-103, second line), then the collision half step with tau***:
// Q** -> Q^{n+1}.
__device__ __forceinline__ void macro_y_body(const double* MMK_R H, MacroBufs mb, double* MMK_R Qn,
                          KGrid g, KParams p, double dt, double eps, int* MMK_R err, int c,
                          const double* MMK_R srcq = nullptr) {
  const int nc = g.nx * g.ny;
  const int i = c % g.nx, j = c / g.nx;
  const int cb = (j > 0 ? j - 1 : g.ny - 1) * g.nx + i;
  const int ct = (j < g.ny - 1 ? j + 1 : 0) * g.nx + i;
  double FB[6], FT[6];
  for (int m = 0; m < 6; ++m) {
    FB[m] = (j > 0 || p.bc[2] == MM_BC_PERIODIC) ? mb.FY[m * nc + cb] + mb.FY[(6 + m) * nc + c]
                                                 : mb.BY[m * g.nx + i];
    FT[m] = (j < g.ny - 1 || p.bc[3] == MM_BC_PERIODIC)
                ? mb.FY[m * nc + c] + mb.FY[(6 + m) * nc + ct]
                : mb.BY[(6 + m) * g.nx + i];
  }
  // heat-flux faces: components (H112, H122, H222) enter (E11, E12, E22)
  double dH[3];
  for (int h = 1; h < 4; ++h) {
    const double hc = H[h * nc + c];
    const double hb = H[h * nc + cb];
    const double ht = H[h * nc + ct];
    const double HB = j > 0 ? 0.5 * (hc + hb) : boundary_H(p, hc, hb, 2, h);
    const double HT = j < g.ny - 1 ? 0.5 * (ht + hc) : boundary_H(p, hc, ht, 3, h);
    dH[h - 1] = HT - HB;
  }
  const double lam = dt * g.idy;
  double q3[6];
  for (int m = 0; m < 6; ++m) {
    double v = mb.Q2[m * nc + c] - lam * (FT[m] - FB[m]);
    if (m >= 3) v -= dt * (dH[m - 3] * g.idy);
    q3[m] = v;
  }
  // optional source between the y transport and the collision half step (Eq. macro2d-split3b)
  if (srcq)
    for (int m = 0; m < 6; ++m) q3[m] = fma(dt, srcq[m * nc + c], q3[m]);
  double o[6], ir;
  const bool ok = coll_half(p, q3, eps, dt, o, ir);
  for (int m = 0; m < 6; ++m) Qn[m * nc + c] = o[m];
  if (!ok) atomicOr(err, ERR_NONPHYS_MACRO);
}

}  // namespace macro_body
}  // namespace mmk
