// Internal declarations shared by the CUDA translation units of libmmkfvs (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mmkfvs.h"

namespace mmk {

// Grid quantities used on the device (derived once on the host).
struct KGrid {
  int nx, ny, nv1, nv2;
  double dx, dy, v1min, v2min, dv1, dv2;
  double idx, idy;  // 1/dx, 1/dy
};

// FP32 copies of the grid quantities for the FP32-g kernels (rounded once on the host).
struct KGridF {
  float v1min, v2min, dv1, dv2, idx, idy;
};

// Physical parameters used on the device.
struct KParams {
  double nu, tau0;
  int tau_model;
  int bc[4];
  double wall_T[4], wall_U[4];
  int keep_es;
};

// Per-cell fields produced by the prims kernel, SoA [NPRIM][ny][nx]: primitive variables of
// Q^n, then per-cell coefficients of the micro step (they depend on dt, eps and, through the
// discrete strain and temperature gradient of Eq. 5-97more, on the neighbours), computed once
// per cell so that the phase-space kernels never divide or repeat per-cell work in every lane.
enum PrimField {
  P_RHO = 0, P_U1, P_U2, P_T, P_TAU,
  P_TI11, P_TI12, P_TI22,  // inverse of the ES tensor Tcal (Eq. 2-19)
  P_KG,                    // rho / (2 pi sqrt(det Tcal)): normalisation of the ES Gaussian
  P_TH11, P_TH22,          // diagonal of the temperature tensor P / rho
  P_IT, P_INV2T,           // 1/T, 1/(2T)
  P_KAP,                   // dt dv1 dv2 / (2 pi T): Zhat = kap/dt e1 e2 (projection polynomial)
  P_OM1, P_OM1KAP,         // eps/(eps + dt tau), and times kap
  P_GAM0,                  // om2/eps * KG: prefactor of the ES Gaussian in the relaxation
  P_OME,                   // om2 mu / eps, mu = rho/(2 pi T)
  // om2 mu / tau times the coefficients of B:sigma + C.grad T as a cubic in c2 (Eq. 5-69):
  // p0 = c1 (w01 + c1 (w02 + c1 w03)), p1 = w10 + c1 (w11 + c1 w12), p2 = w20 + c1 w21, p3 = w30
  P_W01, P_W02, P_W03, P_W10, P_W11, P_W12, P_W20, P_W21, P_W30,
  NPRIM
};

// FP32 copies of the per-cell coefficients used by the FP32-g phase-space kernels, SoA
// [NPRIMF][ny][nx] (rounded once per cell by the prims kernel).
enum PrimFieldF {
  F_U1 = 0, F_U2, F_INV2T, F_IT, F_KAP, F_OM1, F_OM1KAP, F_GAM0, F_OME,
  F_TI11H, F_TI12, F_TI22H,  // Ti11/2, Ti12, Ti22/2
  F_W01, F_W02, F_W03, F_W10, F_W11, F_W12, F_W20, F_W21, F_W30,
  NPRIMF
};

// Bits of the device error word.
enum { ERR_NONPHYS_PRIM = 1, ERR_NONPHYS_MACRO = 2, ERR_NONFINITE_G = 4, ERR_WAIT_TIMEOUT = 8 };

// Launch shape of the micro kernels: R rows of v2 per pass, threads = R * nv1 rounded up to 32.
struct MicroShape {
  int R;
  int threads;
  size_t smem_x, smem_y;
  size_t smem_ghat;  // closure Ghat kernel
  int xrows;         // rows per thread of the register-resident x sweep (0: generic kernel)
};
MicroShape micro_shape(int nv1, int nv2);

// Per-cell fields: launch_prims_uT writes every cell's (u1, u2, T) into prim, then
// launch_prims the rest (it reads the neighbours' (u1, u2, T) there): always in this order.
void launch_prims_uT(const double* Q, double* prim, const KGrid& g, cudaStream_t s);
// The FP32 coefficients of every cell for the FP32-g kernels (after launch_prims_uT; writes no
// other FP64 field).
void launch_prims_f32(const double* Q, const double* prim, float* primf, const KGrid& g,
                      const KParams& p, double dt, double eps, int* err, cudaStream_t s);
// Q [6][nc] from primitive fields P4 [4][nc] = (rho, u1, u2, T), isotropic temperature tensor
void launch_q_from_prim(const double* P4, double* Q, int nc, cudaStream_t s);
void launch_prims(const double* Q, double* prim, float* primf, const KGrid& g, const KParams& p,
                  double dt, double eps, int* err, cudaStream_t s);
// The sweeps over the cells [cell0, cell0 + ncells) (ncells < 0: every cell from cell0 = 0).
template <typename Tg>
void launch_micro_x(const Tg* Gin, Tg* Gout, const double* prim, const KGrid& g,
                    const KParams& p, double dt, const MicroShape& ms, cudaStream_t s,
                    int cell0 = 0, int ncells = -1, double* Ee = nullptr);
// src (optional): a term added to g^{n+1} at every node, same layout as G
// Rm (optional, used only with one row per pass, ms.R == 1): receives the raw row sums of
// G^{n+1} [cell][3][nv1] for the next step's launch_micro_x_rows.
// Ee (optional): the Maxwellian factors e1, e2 [cell][nv1 + nv2] that the x sweep
// (launch_micro_x or launch_micro_x_rows with Ee) left for every cell of this sweep in the same
// step (the values the sweep would form itself).
template <typename Tg>
void launch_micro_y(const Tg* Gs, Tg* Gout, double* H, const double* prim, const KGrid& g,
                    const KParams& p, double dt, double eps, const MicroShape& ms, int* err,
                    cudaStream_t s, const double* src = nullptr, int cell0 = 0,
                    int ncells = -1, double* Rm = nullptr, const double* Ee = nullptr);
// The x sweep from the row sums Rm of G^n left by the previous y sweep (needs ms.R == 1 and
// every cell's sums current); with Ee it leaves each cell's e1, e2 for the y sweep.
template <typename Tg>
void launch_micro_x_rows(const Tg* Gin, Tg* Gout, const double* prim, const double* Rm,
                         const KGrid& g, const KParams& p, double dt, const MicroShape& ms,
                         cudaStream_t s, int cell0 = 0, int ncells = -1, double* Ee = nullptr);
// The row sums of G for the cells [cell0, cell0 + ncells) (every cell for ncells < 0): whenever
// G is set other than by a sweep (needs ms.R == 1).
void launch_row_sums_rect(const double* G, double* Rm, const KGrid& g, int i0, int i1, int j0,
                          int j1, cudaStream_t s);
void launch_row_sums(const double* G, double* Rm, const KGrid& g, cudaStream_t s, int cell0 = 0,
                     int ncells = -1);
template <typename Tg>
void launch_micro_y_wall(const Tg* Gs, Tg* Gout, double* H, const double* prim,
                         const int* wall_cells, int n_wall, const KGrid& g, const KParams& p,
                         double dt, double eps, const MicroShape& ms, int* err, cudaStream_t s,
                         double* Rm = nullptr);
// Diffuse-wall cells of the FP32-g step from the G* the fused kernel exported (Gs): G^{n+1} of
// those cells into Gout and their heat flux into H (FP64); one CTA per cell, per-velocity
// arithmetic in FP32.  Reads Q^n and the (u1, u2, T) fields of launch_prims_uT.
void launch_wall_f32(const float* Gs, float* Gout, double* H, const double* Q,
                     const double* prim, const int* wall_cells, int n_wall, const KGrid& g,
                     const KParams& p, double dt, double eps, int* err, cudaStream_t s);
// Fused FP32-g micro step (x sweep, y sweep, relaxation, heat flux) streaming over column
// segments: reads Gin once and writes Gout (a different buffer); cells next to a diffuse wall are
// left to the wall kernel, which reads the G* this kernel exports to Gexp.  One warp per cell
// column (needs nv1 <= 32); no FP64 instruction runs in it: velocity sums are FP32 warp
// butterflies and the heat flux leaves as (hi, lo) FP32 pairs Hf[8][ny][nx] that
// launch_h_unpack combines in FP64.
int fused_segments_f32(const KGrid& g, const MicroShape& ms);
// Shared memory per CTA of the FP32-g kernel chosen for this mesh (bytes)
size_t fused_smem_f32(const KGrid& g);
// Opt-in shared memory per CTA of the target GPU (sm_103a)
constexpr size_t kMaxSmemPerCta = 227 * 1024;
// nseg row segments of seg_rows = ceil(ny / nseg) rows each
void launch_micro_fused_f32(const float* Gin, float* Gout, float* Gexp, float* Hf,
                            const float* primf, const KGrid& g, const KParams& p, double dt,
                            const MicroShape& ms, int nseg, int* err, cudaStream_t s);
// Buffers of the macro step: Q* and Q**, each cell's half fluxes along x (of Q*) and y (of Q**)
// [Fp(6) Fm(6)][ny][nx], and the fluxes through the non-periodic boundary faces
// BX [2 sides][6][ny], BY [2 sides][6][nx].
struct MacroBufs {
  double* Q1;
  double* Q2;
  double* FX;
  double* FY;
  double* BX;
  double* BY;
};
constexpr size_t macro_doubles(int nx, int ny) {
  return (size_t)nx * ny * (6 + 6 + 12 + 12) + 12 * (size_t)ny + 12 * (size_t)nx;
}
void launch_macro_x1(const double* Qn, const MacroBufs& mb, const KGrid& g, const KParams& p,
                     double dt, double eps, int* err, cudaStream_t s);
void launch_macro_x2(const double* H, const MacroBufs& mb, const KGrid& g, const KParams& p,
                     double dt, int* err, cudaStream_t s);
// srcq (optional): [6][ny][nx] rates added times dt after the y transport
void launch_macro_y(const double* H, const MacroBufs& mb, double* Qn, const KGrid& g,
                    const KParams& p, double dt, double eps, int* err, cudaStream_t s,
                    const double* srcq = nullptr);
void launch_h_unpack(const float* Hf, double* H, const KGrid& g, double eps, cudaStream_t s);
__host__ __device__ inline MacroBufs carve_macro(double* base, int nx, int ny) {
  const size_t nc = (size_t)nx * ny;
  MacroBufs mb;
  mb.Q1 = base;
  mb.Q2 = mb.Q1 + 6 * nc;
  mb.FX = mb.Q2 + 6 * nc;
  mb.FY = mb.FX + 12 * nc;
  mb.BX = mb.FY + 12 * nc;
  mb.BY = mb.BX + 12 * (size_t)ny;
  return mb;
}
// Micro sweeps over a device-resident cell list (persistent CTAs; count read on the device).
// Rm (optional, with ms.R == 1): the x sweep takes its moments from the row sums, the y sweep
// leaves them for G^{n+1}.
template <typename Tg>
void launch_micro_x_list(const Tg* Gin, Tg* Gout, const double* prim, const KGrid& g,
                         const KParams& p, double dt, const MicroShape& ms, const int* list,
                         const int* count, int blocks, cudaStream_t s, const double* Rm = nullptr,
                         double* Ee = nullptr);
template <typename Tg>
void launch_micro_y_list(const Tg* Gs, Tg* Gout, double* H, const double* prim, const KGrid& g,
                         const KParams& p, double dt, double eps, const MicroShape& ms, int* err,
                         const int* list, const int* count, int blocks, cudaStream_t s,
                         double* Rm = nullptr, const double* Ee = nullptr);
int micro_list_blocks(const MicroShape& ms, bool ysweep);
// Learned closure (FP64 path): features + Chapman-Enskog flux + scale (aux [5][ny][nx]),
// training targets, decision, work lists [x | y | refresh][nc] with counts[3], Ghat write.
// (needs the prims of Q from launch_prims)
void launch_closure_features(const double* Q, const double* prim, const KGrid& g,
                             const KParams& p, double eps, double dt, float* X, double* aux,
                             cudaStream_t s);
void launch_closure_targets(const double* H, const double* aux, float* Y, const KGrid& g,
                            cudaStream_t s);
void launch_closure_decide(const float* Y, const double* aux, double thr, const KGrid& g,
                           const KParams& p, unsigned char* flags, double* H,
                           unsigned long long* nclosure, cudaStream_t s);
void launch_closure_lists(const unsigned char* flags, unsigned char* valid, const KGrid& g,
                          const KParams& p, int* lists, int* counts, cudaStream_t s);
void launch_closure_stale(unsigned char* valid, const KGrid& g, int* list, int* count,
                          cudaStream_t s);
int closure_ghat_blocks(const MicroShape& ms);
// Rm (optional, with ms.R == 1): the row sums of the new g of the listed cells.
void launch_closure_ghat(double* G, const double* prim, const KGrid& g, double dt, double eps,
                         const MicroShape& ms, const int* list, const int* count, int blocks,
                         cudaStream_t s, double* Rm = nullptr);
// Manufactured-solution harness (mm_mms.cu): velocity tables phi, gam [nv]; exact state; the
// source terms of one step at time t; per-cell error partial sums [4][ny][nx].
void launch_mms_tables(double* phi, double* gam, const KGrid& g, const KParams& p,
                       cudaStream_t s);
void launch_mms_exact(double* Q, double* G, const double* phi, const KGrid& g, const KParams& p,
                      double t, double eps, double x0, double y0, cudaStream_t s);
void launch_mms_source(const double* prim, const double* phi, const double* gam, double* src_g,
                       double* src_q, const KGrid& g, const KParams& p, double t, double dt,
                       double eps, double x0, double y0, cudaStream_t s);
void launch_mms_errors(const double* Q, const double* G, const double* phi, double* sums,
                       const KGrid& g, const KParams& p, double t, double eps, double x0,
                       double y0, cudaStream_t s);
// Network inference on the stream s (mm_mlp.cu), and the network's device parameters (BF16
// weights, FP32 normalisation) for kernels that evaluate it inline.
void mlp_forward_async(const mm_mlp* m, const float* X, float* Y, int n, cudaStream_t s);
void mlp_device_params(const mm_mlp* m, const __nv_bfloat16** w, const float** norm);
// Fused features + network + decision of the hybrid step (one thread per cell, persistent CTAs).
void launch_closure_predict(const double* Q, const double* prim, const mm_mlp* m,
                            const KGrid& g, const KParams& p, double eps, double dt, double thr,
                            unsigned char* flags, double* H, double* aux,
                            unsigned long long* nclosure, cudaStream_t s);
void launch_diag_exp(const double* x, double* yf, double* yl, size_t n, cudaStream_t s);
void launch_convert_f64_to_f32(const double* in, float* out, size_t n, cudaStream_t s);
void launch_convert_f32_to_f64(const float* in, double* out, size_t n, cudaStream_t s);

}  // namespace mmk
