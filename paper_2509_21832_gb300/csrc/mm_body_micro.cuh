// Device bodies of the FP64 phase-space kernels (one spatial cell per call, the whole CTA
// cooperating), shared by the single-problem kernels and the batched persistent kernels.
#pragma once

#include <cmath>

#include "mm_exp.cuh"
#include "mm_internal.cuh"

// Pointer qualifier of the device bodies: __restrict__ by default; a translation unit whose
// kernel reads data that other CTAs of the same launch wrote defines MMK_R as empty before
// including this header, so that no load of the bodies may take the non-coherent read-only path.
#ifndef MMK_R
#define MMK_R __restrict__
#endif

namespace mmk {
namespace micro_body {


constexpr double kPi = 3.14159265358979323846;
constexpr int kRed = 132;
constexpr int kMaxThreads = 512;  // CTA size limit of the micro kernels (register budget)  // shared doubles reserved for block reductions (32 warps x 4 + 4)

// Sum four values over the CTA; every thread receives the four totals.  Within a warp the
// values are reduced with a transposing butterfly (6 adds per lane instead of 20).
__device__ __forceinline__ void block_sum4(double v[4], double* red) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool h16 = lane & 16;
  double s0 = h16 ? v[0] : v[2];
  double s1 = h16 ? v[1] : v[3];
  double k0 = (h16 ? v[2] : v[0]) + __shfl_xor_sync(full, s0, 16);
  double k1 = (h16 ? v[3] : v[1]) + __shfl_xor_sync(full, s1, 16);
  const bool h8 = lane & 8;
  double s = h8 ? k0 : k1;
  double kk = (h8 ? k1 : k0) + __shfl_xor_sync(full, s, 8);
  kk += __shfl_xor_sync(full, kk, 4);
  kk += __shfl_xor_sync(full, kk, 2);
  kk += __shfl_xor_sync(full, kk, 1);
  if ((lane & 7) == 0) red[warp * 4 + (lane >> 3)] = kk;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w * 4 + threadIdx.x];
    red[128 + threadIdx.x] = t;
  }
  __syncthreads();
  v[0] = red[128];
  v[1] = red[129];
  v[2] = red[130];
  v[3] = red[131];
}

// Upwind neighbour of cell (i, j) across side s, following the boundary rules of the micro
// step: periodic wrap; extrapolation drops the outside difference (neighbour = the cell itself);
// specular uses the cell itself at the mirrored velocity; diffuse sets the inflow of g to zero.
struct Upwind {
  int cell;     // neighbour cell index
  bool mirror;  // read the mirrored velocity index
  bool zero;    // inflow value is zero
};

__device__ __forceinline__ Upwind upwind_x(const KGrid& g, const KParams& p, int i, int j, int s) {
  Upwind u{0, false, false};
  int ni = s == 0 ? i - 1 : i + 1;
  if (ni < 0 || ni >= g.nx) {
    const int bc = p.bc[s];
    if (bc == MM_BC_PERIODIC) ni = (ni + g.nx) % g.nx;
    else if (bc == MM_BC_EXTRAP) ni = i;
    else if (bc == MM_BC_SPECULAR) { ni = i; u.mirror = true; }
    else { ni = i; u.zero = true; }
  }
  u.cell = j * g.nx + ni;
  return u;
}

__device__ __forceinline__ Upwind upwind_y(const KGrid& g, const KParams& p, int i, int j, int s) {
  Upwind u{0, false, false};
  int nj = s == 2 ? j - 1 : j + 1;
  if (nj < 0 || nj >= g.ny) {
    const int bc = p.bc[s];
    if (bc == MM_BC_PERIODIC) nj = (nj + g.ny) % g.ny;
    else if (bc == MM_BC_EXTRAP) nj = j;
    else if (bc == MM_BC_SPECULAR) { nj = j; u.mirror = true; }
    else { nj = j; u.zero = true; }
  }
  u.cell = nj * g.nx + i;
  return u;
}

__device__ __forceinline__ bool diffuse_wall_cell(const KGrid& g, const KParams& p, int i, int j) {
  return (i == 0 && p.bc[0] == MM_BC_DIFFUSE) || (i == g.nx - 1 && p.bc[1] == MM_BC_DIFFUSE) ||
         (j == 0 && p.bc[2] == MM_BC_DIFFUSE) || (j == g.ny - 1 && p.bc[3] == MM_BC_DIFFUSE);
}

// Raw row sums of the velocity column k of a cell's g block: Rm[(cell * 3 + j) * nv1 + k] =
// sum_l v2(l)^j g(k, l), j = 0, 1, 2, accumulated over l in ascending order as
// R0 += g, R1 = fma(v2, g, R1), R2 = fma(v2 v2, g, R2) with v2 = fma(l + 1/2, dv2, v2min): the y
// sweep leaves them for G^{n+1} (they also give its heat-flux sums), row_sums_body forms them
// for any g in exactly the same way, and the next x sweep takes the moments of its upwind
// differences from two cells' sums instead of from every velocity.  Only for one row per pass
// (R = 1: the thread of column k holds all its rows).
__device__ __forceinline__ void store_row_sums(double* MMK_R Rm, int cell, int nv1, int k,
                                               double R0, double R1, double R2) {
  double* o = Rm + (size_t)cell * 3 * nv1 + k;
  o[0] = R0;
  o[nv1] = R1;
  o[2 * nv1] = R2;
}

// The row sums of cell `cell` of G (blockDim >= nv1; thread k = column k); vt holds v2 and v2^2
// of every row ([2][nv2], formed as fma(l + 1/2, dv2, v2min) and its square).
template <typename Tg>
__device__ __forceinline__ void row_sums_body(const Tg* MMK_R G, double* MMK_R Rm,
                                              const KGrid& g, int cell,
                                              const double* MMK_R vt) {
  const int nv1 = g.nv1, nv2 = g.nv2;
  const int k = threadIdx.x;
  if (k >= nv1) return;
  const Tg* Gc = G + (size_t)cell * nv1 * nv2 + k;
  double R0 = 0.0, R1 = 0.0, R2 = 0.0;
  constexpr int kB = 8;  // loads issued ahead; the sums still run over l in ascending order
  for (int l0 = 0; l0 < nv2; l0 += kB) {
    double ov[kB];
#pragma unroll
    for (int m = 0; m < kB; ++m) ov[m] = l0 + m < nv2 ? (double)Gc[(l0 + m) * nv1] : 0.0;
#pragma unroll
    for (int m = 0; m < kB; ++m) {
      const int l = l0 + m;
      if (l < nv2) {
        R0 += ov[m];
        R1 = fma(vt[l], ov[m], R1);
        R2 = fma(vt[nv2 + l], ov[m], R2);
      }
    }
  }
  store_row_sums(Rm, cell, nv1, k, R0, R1, R2);
}

// Central heat-flux sums sum_l c2^j g (c2 = v2 - u2, j = 0..3) from the raw sums R_j.
__device__ __forceinline__ void central_sums(double u2, double R0, double R1, double R2, double R3,
                                             double& H0, double& H1, double& H2, double& H3) {
  H0 = R0;
  H1 = fma(-u2, R0, R1);
  H2 = fma(u2, fma(u2, R0, -2.0 * R1), R2);
  H3 = fma(u2, fma(u2, fma(-u2, R0, 3.0 * R1), -3.0 * R2), R3);
}

// ------------------------------------------------------------------------------------------
// x sweep: Eqs. (zmicrox), (coeffs-2D-xdir), (zhat-2D-xdir), (update-micro-2D-xdir)
// ------------------------------------------------------------------------------------------
// NR > 0: every active thread owns exactly NR rows (nv2 == NR R); the upwind differences of pass
// 1 stay in registers for pass 2.  NR = 0: any shape, differences recomputed in pass 2.
template <typename Tg, int NR = 0>
__device__ __forceinline__ void micro_x_body(const Tg* MMK_R Gin,
                                                    Tg* MMK_R Gout,
                                                    const double* MMK_R prim, KGrid g,
                                                    KParams p, double dtidx, int R, int cell, double* sm,
                                                    double* MMK_R Ee = nullptr) {
  const int nv1 = g.nv1, nv2 = g.nv2;
  double* red = sm;
  double* c2t = sm + kRed;
  double* c2q = c2t + nv2;
  double* e2t = c2q + nv2;
  double* qet = e2t + nv2;

  const int nc = g.nx * g.ny;
  const int i = cell % g.nx, j = cell / g.nx;
  const int t = threadIdx.x;
  const int k = t % nv1, r = t / nv1;
  const bool active = r < R;

  const double u1 = prim[P_U1 * nc + cell], u2 = prim[P_U2 * nc + cell];
  const double inv2T = prim[P_INV2T * nc + cell], iT = prim[P_IT * nc + cell];
  const double kap = prim[P_KAP * nc + cell];

  // with Ee: the cell's Maxwellian factors for the y sweep, Ee[cell (nv1 + nv2) + k] = e1(k),
  // Ee[cell (nv1 + nv2) + nv1 + l] = e2(l)
  double* Eec = Ee ? Ee + (size_t)cell * (nv1 + nv2) : nullptr;
  for (int l = t; l < nv2; l += blockDim.x) {
    const double c2 = fma(l + 0.5, g.dv2, g.v2min) - u2;
    const double q = c2 * c2;
    const double e2 = expd(-q * inv2T);
    c2t[l] = c2;
    c2q[l] = q;
    e2t[l] = e2;
    if (Eec) Eec[nv1 + l] = e2;
  }

  const double v1 = fma(k + 0.5, g.dv1, g.v1min);
  const double c1 = v1 - u1;
  const double av = fabs(v1);
  const double sig = -av * g.idx;  // Z = sig * (G_up - G)
  const double lam = av * dtidx;   // -dt Z = lam * (G_up - G)
  const Upwind up = upwind_x(g, p, i, j, v1 > 0.0 ? 0 : 1);
  const int ku = up.mirror ? nv1 - 1 - k : k;
  const size_t nv = (size_t)nv1 * nv2;
  const Tg* Gc = Gin + (size_t)cell * nv + k;
  const Tg* Gu = Gin + (size_t)up.cell * nv + ku;
  __syncthreads();

  // pass 1: velocity moments of Z
  double D0 = 0.0, D1 = 0.0, D2 = 0.0;
  double dr[NR > 0 ? NR : 1];
  if (active) {
    if constexpr (NR > 0) {
#pragma unroll
      for (int m = 0; m < NR; ++m) {
        const int l = r + m * R;
        const double gv = (double)Gc[l * nv1];
        const double gu = up.zero ? 0.0 : (double)Gu[l * nv1];
        const double d = gu - gv;
        dr[m] = d;
        D0 += d;
        D1 = fma(c2t[l], d, D1);
        D2 = fma(c2q[l], d, D2);
      }
    } else {
      for (int l = r; l < nv2; l += R) {
        const double gv = (double)Gc[l * nv1];
        const double gu = up.zero ? 0.0 : (double)Gu[l * nv1];
        const double d = gu - gv;
        D0 += d;
        D1 = fma(c2t[l], d, D1);
        D2 = fma(c2q[l], d, D2);
      }
    }
  }
  const double sD0 = sig * D0;
  double S[4] = {sD0, c1 * sD0, sig * D1, fma(c1 * c1, sD0, sig * D2)};
  block_sum4(S, red);

  // projection coefficients: Zhat = (dv1 dv2 / (2 pi T)) e1 e2 (b0 + b1 c1 + b2 c2 + gm |c|^2)
  const double b0 = fma(-S[3], inv2T, 2.0 * S[0]);
  const double b1 = S[1] * iT, b2 = S[2] * iT;
  const double gm = fma(0.25 * S[3], iT * iT, -S[0] * inv2T);
  for (int l = t; l < nv2; l += blockDim.x) qet[l] = e2t[l] * fma(b2, c2t[l], gm * c2q[l]);
  const double e1 = expd(-c1 * c1 * inv2T);
  if (Eec && t < nv1) Eec[k] = e1;
  const double bk = kap * e1;
  const double ak = bk * fma(gm * c1, c1, fma(b1, c1, b0));
  __syncthreads();

  // pass 2: G* = G - dt Z + dt Zhat
  if (active) {
    Tg* Go = Gout + (size_t)cell * nv + k;
    if constexpr (NR > 0) {
#pragma unroll
      for (int m = 0; m < NR; ++m) {
        const int l = r + m * R;
        const double gv = (double)Gc[l * nv1];
        double o = fma(lam, dr[m], gv);
        o = fma(ak, e2t[l], o);
        o = fma(bk, qet[l], o);
        Go[l * nv1] = (Tg)o;
      }
    } else {
      for (int l = r; l < nv2; l += R) {
        const double gv = (double)Gc[l * nv1];
        const double gu = up.zero ? 0.0 : (double)Gu[l * nv1];
        const double d = gu - gv;
        double o = fma(lam, d, gv);
        o = fma(ak, e2t[l], o);
        o = fma(bk, qet[l], o);
        Go[l * nv1] = (Tg)o;
      }
    }
  }
}

// x sweep with the moments of Z from the row sums Rm of G^n (one row per pass, R = 1): with
// d = G_up - G of column k, sum_l c2^j d for j = 0, 1, 2 follows from the differences of the two
// cells' raw sums (c2 = v2 - u2), so one pass over the velocities forms
// G* = G + lam d + ak e2 + bk qet (Eq. update-micro-2D-xdir) without accumulating per velocity.
// With Ee it also leaves the cell's Maxwellian factors for the y sweep, which needs the same
// ones: Ee[cell (nv1 + nv2) + k] = e1(k), Ee[cell (nv1 + nv2) + nv1 + l] = e2(l).
template <typename Tg>
__device__ __forceinline__ void micro_x_rows_body(const Tg* MMK_R Gin,
                                                  Tg* MMK_R Gout,
                                                  const double* MMK_R prim,
                                                  const double* MMK_R Rm,
                                                  double* MMK_R Ee, KGrid g, KParams p,
                                                  double dtidx, int cell, double* sm) {
  const int nv1 = g.nv1, nv2 = g.nv2;
  double* red = sm;
  double* c2t = sm + kRed;
  double* c2q = c2t + nv2;
  double* e2t = c2q + nv2;
  double* qet = e2t + nv2;

  const int nc = g.nx * g.ny;
  const int i = cell % g.nx, j = cell / g.nx;
  const int t = threadIdx.x;
  const int k = t % nv1;
  const bool active = t < nv1;

  const double u1 = prim[P_U1 * nc + cell], u2 = prim[P_U2 * nc + cell];
  const double inv2T = prim[P_INV2T * nc + cell], iT = prim[P_IT * nc + cell];
  const double kap = prim[P_KAP * nc + cell];

  double* Eec = Ee ? Ee + (size_t)cell * (nv1 + nv2) : nullptr;
  for (int l = t; l < nv2; l += blockDim.x) {
    const double c2 = fma(l + 0.5, g.dv2, g.v2min) - u2;
    const double q = c2 * c2;
    const double e2 = expd(-q * inv2T);
    c2t[l] = c2;
    c2q[l] = q;
    e2t[l] = e2;
    if (Eec) Eec[nv1 + l] = e2;
  }

  const double v1 = fma(k + 0.5, g.dv1, g.v1min);
  const double c1 = v1 - u1;
  const double av = fabs(v1);
  const double sig = -av * g.idx;
  const double lam = av * dtidx;
  const Upwind up = upwind_x(g, p, i, j, v1 > 0.0 ? 0 : 1);
  const int ku = up.mirror ? nv1 - 1 - k : k;
  const size_t nv = (size_t)nv1 * nv2;
  const Tg* Gc = Gin + (size_t)cell * nv + k;
  const Tg* Gu = Gin + (size_t)up.cell * nv + ku;

  // moments of the upwind differences: sum_l (1, c2, c2^2) d from the raw sums
  double D0 = 0.0, D1 = 0.0, D2 = 0.0;
  if (active) {
    const double* Ro = Rm + (size_t)cell * 3 * nv1 + k;
    const double* Ru = Rm + (size_t)up.cell * 3 * nv1 + ku;
    const double r0 = (up.zero ? 0.0 : Ru[0]) - Ro[0];
    const double r1 = (up.zero ? 0.0 : Ru[nv1]) - Ro[nv1];
    const double r2 = (up.zero ? 0.0 : Ru[2 * nv1]) - Ro[2 * nv1];
    D0 = r0;
    D1 = fma(-u2, r0, r1);
    D2 = fma(u2, fma(u2, r0, -2.0 * r1), r2);
  }
  __syncthreads();
  const double sD0 = sig * D0;
  double S[4] = {sD0, c1 * sD0, sig * D1, fma(c1 * c1, sD0, sig * D2)};
  block_sum4(S, red);

  const double b0 = fma(-S[3], inv2T, 2.0 * S[0]);
  const double b1 = S[1] * iT, b2 = S[2] * iT;
  const double gm = fma(0.25 * S[3], iT * iT, -S[0] * inv2T);
  for (int l = t; l < nv2; l += blockDim.x) qet[l] = e2t[l] * fma(b2, c2t[l], gm * c2q[l]);
  const double e1 = expd(-c1 * c1 * inv2T);
  if (Eec && active) Eec[k] = e1;
  const double bk = kap * e1;
  const double ak = bk * fma(gm * c1, c1, fma(b1, c1, b0));
  __syncthreads();

  // the single pass: G* = G - dt Z + dt Zhat
  if (active) {
    Tg* Go = Gout + (size_t)cell * nv + k;
    for (int l = 0; l < nv2; ++l) {
      const double gv = (double)Gc[l * nv1];
      const double gu = up.zero ? 0.0 : (double)Gu[l * nv1];
      double o = fma(lam, gu - gv, gv);
      o = fma(ak, e2t[l], o);
      o = fma(bk, qet[l], o);
      Go[l * nv1] = (Tg)o;
    }
  }
}

// ------------------------------------------------------------------------------------------
// y sweep + relaxation + heat flux for cells not adjacent to a diffuse wall:
// Eqs. (zmicroy)-(update-micro-2D-ydir), (5-97), (5-97more), (5-98), (5-99)
// ------------------------------------------------------------------------------------------
constexpr int kYTables = 13;

template <typename Tg>
__device__ __forceinline__ void micro_y_body(const Tg* MMK_R Gs,
                                                    Tg* MMK_R Gout,
                                                    double* MMK_R Hout,
                                                    const double* MMK_R prim, KGrid g,
                                                    KParams p, double dtidy, double hscale, int R,
                                                    int* MMK_R err, int cell, double* sm,
                                                    const double* MMK_R src = nullptr,
                                                    double* MMK_R Rm = nullptr,
                                                    const double* MMK_R Ee = nullptr) {
  const int nv1 = g.nv1, nv2 = g.nv2;
  const int nc = g.nx * g.ny;
  const int i = cell % g.nx, j = cell / g.nx;
  if (diffuse_wall_cell(g, p, i, j)) return;  // handled by k_micro_y_wall

  double* red = sm;
  double* tb = sm + kRed;
  double* c2t = tb;
  double* c2q = tb + nv2;
  double* c2c = tb + 2 * nv2;
  double* e2t = tb + 3 * nv2;
  double* g2t = tb + 4 * nv2;
  double* w2t = tb + 5 * nv2;  // om1 - wlt: weight of the cell's own G* in the update
  double* s0t = tb + 6 * nv2;
  double* s1t = tb + 7 * nv2;
  double* s2t = tb + 8 * nv2;
  double* wlt = tb + 9 * nv2;
  double* E1t = tb + 10 * nv2;
  double* E2t = tb + 11 * nv2;
  double* E3t = tb + 12 * nv2;

  const int t = threadIdx.x;
  const int k = t % nv1, r = t / nv1;
  const bool active = r < R;

  const double u1 = prim[P_U1 * nc + cell], u2 = prim[P_U2 * nc + cell];
  const double inv2T = prim[P_INV2T * nc + cell], iT = prim[P_IT * nc + cell];
  const double Ti11 = prim[P_TI11 * nc + cell], Ti12 = prim[P_TI12 * nc + cell];
  const double Ti22 = prim[P_TI22 * nc + cell];
  const double om1 = prim[P_OM1 * nc + cell], om1kap = prim[P_OM1KAP * nc + cell];
  const double gam0 = prim[P_GAM0 * nc + cell], ome = prim[P_OME * nc + cell];

  // l-dependent tables; nneg = number of rows with v2 < 0 (v2 increases with l), so that the
  // upwind side of a row is an integer comparison
  int nneg = 0;
  for (int base = 0; base < nv2; base += blockDim.x) {
    const int l = base + t;
    bool neg = false;
    if (l < nv2) {
      const double v2 = fma(l + 0.5, g.dv2, g.v2min);
      const double c2 = v2 - u2;
      const double q = c2 * c2;
      // e2 as the x sweep formed it (Ee), or formed here the same way
      const double e2 = Ee ? Ee[(size_t)cell * (nv1 + nv2) + nv1 + l] : expd(-q * inv2T);
      const double av = fabs(v2);
      const double sg = -av * g.idy;
      const double wl = om1 * (av * dtidy);
      c2t[l] = v2;  // raw powers of v2 for the row sums (heat flux from central_sums)
      c2q[l] = v2 * v2;
      c2c[l] = v2 * v2 * v2;
      e2t[l] = e2;
      g2t[l] = expd(-0.5 * Ti22 * q);
      w2t[l] = om1 - wl;
      s0t[l] = sg;
      s1t[l] = sg * c2;
      s2t[l] = sg * q;
      wlt[l] = wl;
      E1t[l] = e2 * c2;
      E2t[l] = e2 * q;
      E3t[l] = e2 * q * c2;
      neg = v2 < 0.0;
    }
    nneg += __syncthreads_count(neg);
  }

  const Upwind ub = upwind_y(g, p, i, j, 2);  // upwind for v2 > 0
  const Upwind ut = upwind_y(g, p, i, j, 3);  // upwind for v2 < 0
  const size_t nv = (size_t)nv1 * nv2;
  const Tg* Gc = Gs + (size_t)cell * nv + k;
  const Tg* Gb = Gs + (size_t)ub.cell * nv + k;
  const Tg* Gt = Gs + (size_t)ut.cell * nv + k;

  const double v1 = fma(k + 0.5, g.dv1, g.v1min);
  const double c1 = v1 - u1;
  const double c1q = c1 * c1;
  __syncthreads();

  // pass 1: velocity moments of Z*
  double E0 = 0.0, E1 = 0.0, E2 = 0.0;
  if (active) {
    for (int l = r; l < nv2; l += R) {
      const double gv = (double)Gc[l * nv1];
      const bool top = l < nneg;
      const Upwind& u = top ? ut : ub;
      const Tg* Gu = top ? Gt : Gb;
      const int lu = u.mirror ? nv2 - 1 - l : l;
      const double gu = u.zero ? 0.0 : (double)Gu[lu * nv1];
      const double d = gu - gv;
      E0 = fma(s0t[l], d, E0);
      E1 = fma(s1t[l], d, E1);
      E2 = fma(s2t[l], d, E2);
    }
  }
  double S[4] = {E0, c1 * E0, E1, fma(c1q, E0, E2)};
  block_sum4(S, red);

  const double b0 = fma(-S[3], inv2T, 2.0 * S[0]);
  const double b1 = S[1] * iT, b2 = S[2] * iT;
  const double gm = fma(0.25 * S[3], iT * iT, -S[0] * inv2T);
  // om1 dt Zhat* and om2 Ghat's Maxwellian part as one cubic in c2 times e1 e2
  const double w01 = prim[P_W01 * nc + cell], w02 = prim[P_W02 * nc + cell];
  const double w03 = prim[P_W03 * nc + cell], w10 = prim[P_W10 * nc + cell];
  const double w11 = prim[P_W11 * nc + cell], w12 = prim[P_W12 * nc + cell];
  const double w20 = prim[P_W20 * nc + cell], w21 = prim[P_W21 * nc + cell];
  const double w30 = prim[P_W30 * nc + cell];
  const double C0 = om1kap * fma(gm, c1q, fma(b1, c1, b0)) - c1 * fma(c1, fma(c1, w03, w02), w01) - ome;
  const double C1 = fma(om1kap, b2, -fma(c1, fma(c1, w12, w11), w10));
  const double C2 = fma(om1kap, gm, -fma(c1, w21, w20));
  const double C3 = -w30;
  const double e1 = Ee ? Ee[(size_t)cell * (nv1 + nv2) + k] : expd(-c1q * inv2T);
  const double A0 = e1 * C0, A1 = e1 * C1, A2 = e1 * C2, A3 = e1 * C3;
  const double c2r = fma(r + 0.5, g.dv2, g.v2min) - u2;
  // gam0 exp(-Ti11 c1^2 / 2 - Ti12 c1 c2) of row l (the factor of the ES Gaussian that depends on
  // c1), advanced by rat per row
  double x = gam0 * expd(-c1 * fma(0.5 * Ti11, c1, Ti12 * c2r));
  const double rat = expd(-Ti12 * c1 * (R * g.dv2));

  // pass 2: G^{n+1} = om1 (G* - dt Z* + dt Zhat*) + om2 Ghat, and its heat-flux moments;
  // om1 G* - om1 dt Z* = wl G*_upwind + (om1 - wl) G*
  double R0 = 0.0, R1 = 0.0, R2 = 0.0, R3 = 0.0;  // raw row sums of G^{n+1}
  // optional source term of g^{n+1} (same layout as G), e.g. the manufactured residual
  const double* Sc = src ? src + (size_t)cell * nv + k : nullptr;
  if (active) {
    Tg* Go = Gout + (size_t)cell * nv + k;
    for (int l = r; l < nv2; l += R) {
      const double gv = (double)Gc[l * nv1];
      const bool top = l < nneg;
      const Upwind& u = top ? ut : ub;
      const Tg* Gu = top ? Gt : Gb;
      const int lu = u.mirror ? nv2 - 1 - l : l;
      const double gu = u.zero ? 0.0 : (double)Gu[lu * nv1];
      double o = fma(wlt[l], gu, w2t[l] * gv);
      o = fma(A0, e2t[l], o);
      o = fma(A1, E1t[l], o);
      o = fma(A2, E2t[l], o);
      o = fma(A3, E3t[l], o);
      o = fma(g2t[l], x, o);
      x *= rat;
      if (Sc) o += Sc[l * nv1];
      const Tg os = (Tg)o;
      Go[l * nv1] = os;
      const double ov = (double)os;
      R0 += ov;
      R1 = fma(c2t[l], ov, R1);
      R2 = fma(c2q[l], ov, R2);
      R3 = fma(c2c[l], ov, R3);
    }
    if (Rm) store_row_sums(Rm, cell, nv1, k, R0, R1, R2);  // only with R = 1
  }
  double H0, H1, H2, H3;
  central_sums(u2, R0, R1, R2, R3, H0, H1, H2, H3);
  double Hs[4] = {c1q * c1 * H0, c1q * H1, c1 * H2, H3};
  block_sum4(Hs, red);
  if (t == 0) {
    bool ok = true;
    for (int m = 0; m < 4; ++m) {
      Hout[m * nc + cell] = hscale * Hs[m];
      ok = ok && isfinite(Hs[m]);
    }
    if (!ok) atomicOr(err, ERR_NONFINITE_G);
  }
}

// ------------------------------------------------------------------------------------------
// y sweep + relaxation + heat flux for cells adjacent to a diffuse wall (Section 6.3): Ghat is
// -(1/tau)(I - Pi_M)[upwind v.grad M] with ghost wall Maxwellians, plus (G - M)/eps if kept.
// ------------------------------------------------------------------------------------------
struct SideM {
  int kind;  // 0 neighbour/periodic, 1 extrapolation (the cell's own M), 2 specular, 3 diffuse
  double rho, u1, u2, T;  // kind 0: neighbour prims; kind 3: wall density, velocity, temperature
};


// Shared memory of the wall body: reduction scratch, the x and y factors of five Maxwellians,
// their prefactors and the row factor of the ES Gaussian.
__host__ __device__ constexpr size_t wall_smem_doubles(int nv1, int nv2) {
  return kRed + 5 * ((size_t)nv1 + (size_t)nv2) + 8 + (size_t)nv2;
}

// Eq. (twodim_wall_densities_1)
__device__ __forceinline__ double wall_R(double ua, double Taa, double Tw, double sgn) {
  return sqrt(Taa / Tw) * exp(-ua * ua / (2.0 * Taa)) +
         ua * sqrt(kPi / (2.0 * Tw)) * (erf(ua / sqrt(2.0 * Taa)) + sgn);
}

template <typename Tg>
__device__ __forceinline__ void micro_y_wall_body(const Tg* MMK_R Gs, Tg* MMK_R Gout,
                               double* MMK_R Hout, const double* MMK_R prim,
                               KGrid g, KParams p, double dt,
                               double eps, int R, int* MMK_R err, int cell, double* sm,
                               double* MMK_R Rm = nullptr) {
  double* red = sm;
  const int nv1 = g.nv1, nv2 = g.nv2;
  const int nc = g.nx * g.ny;
  const int i = cell % g.nx, j = cell / g.nx;
  const int t = threadIdx.x;
  const int k = t % nv1, r = t / nv1;
  const bool active = r < R;

  const double rho = prim[P_RHO * nc + cell];
  const double u1 = prim[P_U1 * nc + cell], u2 = prim[P_U2 * nc + cell];
  const double T = prim[P_T * nc + cell];
  const double tau = prim[P_TAU * nc + cell];
  const double Ti11 = prim[P_TI11 * nc + cell], Ti12 = prim[P_TI12 * nc + cell];
  const double Ti22 = prim[P_TI22 * nc + cell];
  const double KG = prim[P_KG * nc + cell];
  const double Th11 = prim[P_TH11 * nc + cell], Th22 = prim[P_TH22 * nc + cell];
  const double inv2T = 0.5 / T, iT = 1.0 / T;
  const double om1 = eps / (eps + dt * tau);
  const double om2 = dt * tau / (eps + dt * tau);

  SideM sd[4];
  for (int s = 0; s < 4; ++s) {
    int ni = i + (s == 0 ? -1 : s == 1 ? 1 : 0);
    int nj = j + (s == 2 ? -1 : s == 3 ? 1 : 0);
    bool inside = ni >= 0 && ni < g.nx && nj >= 0 && nj < g.ny;
    if (!inside && p.bc[s] == MM_BC_PERIODIC) {
      ni = (ni + g.nx) % g.nx;
      nj = (nj + g.ny) % g.ny;
      inside = true;
    }
    if (inside) {
      const int c = nj * g.nx + ni;
      sd[s] = SideM{0, prim[P_RHO * nc + c], prim[P_U1 * nc + c], prim[P_U2 * nc + c],
                    prim[P_T * nc + c]};
    } else if (p.bc[s] == MM_BC_EXTRAP) {
      sd[s] = SideM{1, 0, 0, 0, 0};
    } else if (p.bc[s] == MM_BC_SPECULAR) {
      sd[s] = SideM{2, 0, 0, 0, 0};
    } else {
      const double Tw = p.wall_T[s], U = p.wall_U[s];
      const double sgn = (s == 0 || s == 2) ? -1.0 : 1.0;
      const double rw = s < 2 ? rho * wall_R(u1, Th11, Tw, sgn) : rho * wall_R(u2, Th22, Tw, sgn);
      sd[s] = SideM{3, rw, s < 2 ? 0.0 : U, s < 2 ? U : 0.0, Tw};
    }
  }

  const Upwind ub = upwind_y(g, p, i, j, 2);
  const Upwind ut = upwind_y(g, p, i, j, 3);
  const size_t nv = (size_t)nv1 * nv2;
  const Tg* Gc = Gs + (size_t)cell * nv + k;
  const Tg* Gb = Gs + (size_t)ub.cell * nv + k;
  const Tg* Gt = Gs + (size_t)ut.cell * nv + k;
  const double v1 = g.v1min + (k + 0.5) * g.dv1;
  const double c1 = v1 - u1;

  // The Maxwellians of the four sides (neighbour or wall ghost) and of the cell (index 4) are
  // separable: rho/(2 pi T) X_q(v1) Y_q(v2).  Their factors are tabulated once per cell, so the
  // upwind v . grad M needs no exponential per velocity.
  double* Xt = sm + kRed;         // [5][nv1]
  double* Yt = Xt + 5 * nv1;      // [5][nv2]
  double* pfq = Yt + 5 * nv2;     // [5]
  auto par = [&](int q, double& pu1, double& pu2, double& pT, double& prho) {
    if (q < 4 && (sd[q].kind == 0 || sd[q].kind == 3)) {
      pu1 = sd[q].u1; pu2 = sd[q].u2; pT = sd[q].T; prho = sd[q].rho;
    } else {
      pu1 = u1; pu2 = u2; pT = T; prho = rho;
    }
  };
  for (int e = t; e < 5 * nv1; e += blockDim.x) {
    const int q = e / nv1, kk = e % nv1;
    double a1, a2, aT, ar;
    par(q, a1, a2, aT, ar);
    const double d = g.v1min + (kk + 0.5) * g.dv1 - a1;
    Xt[e] = exp(-d * d / (2.0 * aT));
  }
  for (int e = t; e < 5 * nv2; e += blockDim.x) {
    const int q = e / nv2, ll = e % nv2;
    double a1, a2, aT, ar;
    par(q, a1, a2, aT, ar);
    const double d = g.v2min + (ll + 0.5) * g.dv2 - a2;
    Yt[e] = exp(-d * d / (2.0 * aT));
  }
  if (t < 5) {
    double a1, a2, aT, ar;
    par(t, a1, a2, aT, ar);
    pfq[t] = ar / (2.0 * kPi * aT);
  }
  // ES Gaussian exp(-c.Tcal^{-1}c/2) = exp(-Ti11 c1^2/2) exp(-Ti22 c2^2/2) exp(-Ti12 c1 c2): the
  // row factor tabulated, the column factor per thread, the cross factor by a recurrence
  double* Et = pfq + 8;  // [nv2]
  if (p.keep_es)
    for (int l = t; l < nv2; l += blockDim.x) {
      const double c2 = g.v2min + (l + 0.5) * g.dv2 - u2;
      Et[l] = exp(-0.5 * Ti22 * c2 * c2);
    }
  __syncthreads();

  // upwind v . grad M at (k, l) with the ghost Maxwellians of each side (reciprocals of dx, dy,
  // tau and of the cell's Maxwellian prefactor hoisted out of the velocity loops)
  const int km = nv1 - 1 - k;
  const double idx = g.idx, idy = g.idy;
  auto side_m = [&](int s, double m0, int l) -> double {
    const SideM& q = sd[s];
    if (q.kind == 1) return m0;
    if (q.kind == 2)
      return s < 2 ? pfq[4] * Xt[4 * nv1 + km] * Yt[4 * nv2 + l]
                   : pfq[4] * Xt[4 * nv1 + k] * Yt[4 * nv2 + (nv2 - 1 - l)];
    return pfq[s] * Xt[s * nv1 + k] * Yt[s * nv2 + l];
  };
  auto mup = [&](int l, double v2, double m0) -> double {
    double z = 0.0;
    if (v1 > 0.0) z += v1 * ((m0 - side_m(0, m0, l)) * idx);
    if (v1 < 0.0) z += v1 * ((side_m(1, m0, l) - m0) * idx);
    if (v2 > 0.0) z += v2 * ((m0 - side_m(2, m0, l)) * idy);
    if (v2 < 0.0) z += v2 * ((side_m(3, m0, l) - m0) * idy);
    return z;
  };
  const double xk = Xt[4 * nv1 + k];  // the cell's Maxwellian / (rho / (2 pi T)) = xk * Yt[l]
  const double x4 = pfq[4] * xk;

  // pass 1: moments of Z* and of the upwind v.grad M
  double E0 = 0, E1 = 0, E2 = 0, W0 = 0, W1 = 0, W2 = 0;
  if (active) {
    for (int l = r; l < nv2; l += R) {
      const double v2 = g.v2min + (l + 0.5) * g.dv2;
      const double c2 = v2 - u2;
      const double gv = (double)Gc[l * nv1];
      const bool top = v2 < 0.0;
      const Upwind& u = top ? ut : ub;
      const Tg* Gu = top ? Gt : Gb;
      const int lu = u.mirror ? nv2 - 1 - l : l;
      const double gu = u.zero ? 0.0 : (double)Gu[lu * nv1];
      const double z = -fabs(v2) * idy * (gu - gv);
      E0 += z;
      E1 += c2 * z;
      E2 += c2 * c2 * z;
      const double mz = mup(l, v2, x4 * Yt[4 * nv2 + l]);
      W0 += mz;
      W1 += c2 * mz;
      W2 += c2 * c2 * mz;
    }
  }
  double S[4] = {E0, c1 * E0, E1, c1 * c1 * E0 + E2};
  block_sum4(S, red);
  double Wm[4] = {W0, c1 * W0, W1, c1 * c1 * W0 + W2};
  block_sum4(Wm, red);

  const double kap = g.dv1 * g.dv2 / (2.0 * kPi * T);
  // the projection polynomials b0 + b1 c1 + b2 c2 + gm |c|^2 of Z* (S) and of v.grad M (Wm),
  // times kap, as a0 + c2 (a1 + a2 c2) for this thread's c1
  auto coeffs = [&](const double* sm4, double& a0, double& a1, double& a2) {
    const double b0 = 2.0 * sm4[0] - sm4[3] * inv2T;
    const double b1 = sm4[1] * iT, b2 = sm4[2] * iT;
    const double gm = 0.25 * sm4[3] * iT * iT - sm4[0] * inv2T;
    a0 = kap * (b0 + b1 * c1 + gm * c1 * c1);
    a1 = kap * b2;
    a2 = kap * gm;
  };
  double sa0, sa1, sa2, wa0, wa1, wa2;
  coeffs(S, sa0, sa1, sa2);
  coeffs(Wm, wa0, wa1, wa2);
  const double itau = 1.0 / tau;
  const double ieps = 1.0 / eps;
  // ES Gaussian at this thread's first row and the ratio of its cross factor between rows
  const double c2r = g.v2min + (r + 0.5) * g.dv2 - u2;
  double ex = p.keep_es ? KG * exp(-0.5 * Ti11 * c1 * c1 - Ti12 * c1 * c2r) : 0.0;
  const double rat = p.keep_es ? exp(-Ti12 * c1 * (R * g.dv2)) : 0.0;

  double R0 = 0.0, R1 = 0.0, R2 = 0.0, R3 = 0.0;  // raw row sums of G^{n+1}
  if (active) {
    Tg* Go = Gout + (size_t)cell * nv + k;
    for (int l = r; l < nv2; l += R) {
      const double v2 = g.v2min + (l + 0.5) * g.dv2;
      const double c2 = v2 - u2;
      const double gv = (double)Gc[l * nv1];
      const bool top = v2 < 0.0;
      const Upwind& u = top ? ut : ub;
      const Tg* Gu = top ? Gt : Gb;
      const int lu = u.mirror ? nv2 - 1 - l : l;
      const double gu = u.zero ? 0.0 : (double)Gu[lu * nv1];
      const double z = -fabs(v2) * idy * (gu - gv);
      const double ml = xk * Yt[4 * nv2 + l];  // M / (rho / (2 pi T))
      const double m = pfq[4] * ml;
      const double gstar2 = gv + dt * ((sa0 + c2 * (sa1 + sa2 * c2)) * ml - z);
      const double mz = mup(l, v2, m);
      const double pim = (wa0 + c2 * (wa1 + wa2 * c2)) * ml;
      double gh = -itau * (mz - pim);
      if (p.keep_es) {
        gh += (ex * Et[l] - m) * ieps;
        ex *= rat;
      }
      const double o = om1 * gstar2 + om2 * gh;
      const Tg os = (Tg)o;
      Go[l * nv1] = os;
      const double ov = (double)os;
      // the raw sums with v2 in the same form (and the same operations) as the other sweeps
      const double v2r = fma(l + 0.5, g.dv2, g.v2min);
      const double v2q = v2r * v2r;
      R0 += ov;
      R1 = fma(v2r, ov, R1);
      R2 = fma(v2q, ov, R2);
      R3 = fma(v2q * v2r, ov, R3);
    }
    if (Rm) store_row_sums(Rm, cell, nv1, k, R0, R1, R2);  // only with R = 1
  }
  double H0, H1, H2, H3;
  central_sums(u2, R0, R1, R2, R3, H0, H1, H2, H3);
  double Hs[4] = {c1 * c1 * c1 * H0, c1 * c1 * H1, c1 * H2, H3};
  block_sum4(Hs, red);
  if (t == 0) {
    const double f = eps * g.dv1 * g.dv2;
    bool ok = true;
    for (int m = 0; m < 4; ++m) {
      Hout[m * nc + cell] = f * Hs[m];
      ok = ok && isfinite(Hs[m]);
    }
    if (!ok) atomicOr(err, ERR_NONFINITE_G);
  }
}

}  // namespace micro_body
}  // namespace mmk
