// Per-cell kernels of the micro-macro KFVS step (Rossmanith & Sar, arXiv 2509.21832):
//  - primitive variables of Q^n for the micro kernels (Section 2: u, P, T; Eq. 2-19: ES tensor;
//    Eq. tau-for-2d-es-bgk: tau),
//  - the Strang-split macro update of Section 5.4: TR-BDF2 collision half steps and the KFVS
//    finite-volume transport in x then y with the central heat-flux differences of Eq. (5-103),
//    with the boundary rules of Sections 5.4.1, 5.4.2 and 6.3.
// One thread per spatial cell.  A face flux is evaluated by both cells that share the face, from
// the same operands in the same order, so both see bitwise the same value.
#include <algorithm>
#include <cmath>

#include "mm_body_macro.cuh"

namespace mmk {

namespace {

using namespace macro_body;

// One thread per cell c < nc = nx ny.
__global__ void k_prims_uT(const double* __restrict__ Q, double* __restrict__ prim, int nc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) uT_body(Q, prim, nc, c);
}

__global__ void k_prims(const double* __restrict__ Q, double* __restrict__ prim,
                        float* __restrict__ primf, KGrid g, KParams p, double dt, double eps,
                        double ieps, int* __restrict__ err) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.nx * g.ny) prims_body<true>(Q, prim, primf, g, p, dt, eps, ieps, err, c);
}

__global__ void k_prims_f32(const double* __restrict__ Q, const double* __restrict__ prim,
                            float* __restrict__ primf, KGrid g, KParams p, double dt, double eps,
                            int* __restrict__ err) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.nx * g.ny) prims_f32_body(Q, prim, primf, g, p, dt, eps, err, c);
}

__global__ void k_macro_x1(const double* __restrict__ Qn, MacroBufs mb, KGrid g, KParams p,
                           double dt, double eps, int* __restrict__ err) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.nx * g.ny) macro_x1_body(Qn, mb, g, p, dt, eps, err, c);
}

__global__ void k_macro_x2(const double* __restrict__ H, MacroBufs mb, KGrid g, KParams p,
                           double dt, int* __restrict__ err) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.nx * g.ny) macro_x2_body(H, mb, g, p, dt, err, c);
}

__global__ void k_macro_y(const double* __restrict__ H, MacroBufs mb, double* __restrict__ Qn,
                          KGrid g, KParams p, double dt, double eps, int* __restrict__ err,
                          const double* __restrict__ srcq) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.nx * g.ny) macro_y_body(H, mb, Qn, g, p, dt, eps, err, c, srcq);
}

// Heat flux of the FP32-g kernels: compensated FP32 (hi, lo) totals -> FP64, times eps dv1 dv2.
__global__ void k_h_unpack(const float* __restrict__ Hf, double* __restrict__ H, int nc,
                           double hscale) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  for (int m = 0; m < 4; ++m)
    H[m * nc + c] = hscale * ((double)Hf[(2 * m) * nc + c] + (double)Hf[(2 * m + 1) * nc + c]);
}

// Q = (rho, rho u1, rho u2, E11, E12, E22) from primitive fields staged as P4 [4][nc] = (rho, u1,
// u2, T) with an isotropic temperature tensor: E = rho (u (x) u + T I) (Section 2, ES-BGK
// operator), as E11 = rho (u1 u1 + T), E12 = rho (u1 u2), E22 = rho (u2 u2 + T), every product
// and sum rounded once in that order (no contraction).
__global__ void k_q_from_prim(const double* __restrict__ P4, double* __restrict__ Q, int nc) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const double rho = P4[c], u1 = P4[nc + c], u2 = P4[2 * nc + c], T = P4[3 * nc + c];
    Q[c] = rho;
    Q[nc + c] = __dmul_rn(rho, u1);
    Q[2 * nc + c] = __dmul_rn(rho, u2);
    Q[3 * nc + c] = __dmul_rn(rho, __dadd_rn(__dmul_rn(u1, u1), T));
    Q[4 * nc + c] = __dmul_rn(rho, __dmul_rn(u1, u2));
    Q[5 * nc + c] = __dmul_rn(rho, __dadd_rn(__dmul_rn(u2, u2), T));
  }
}

__global__ void k_diag_erf(const double* __restrict__ x, double* __restrict__ yf,
                           double* __restrict__ yl, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x) {
    yf[q] = erfd(x[q]);
    yl[q] = erf(x[q]);
  }
}

}  // namespace

namespace {
int blocks_of(const KGrid& g, int t) { return (g.nx * g.ny + t - 1) / t; }
}  // namespace

void launch_prims(const double* Q, double* prim, float* primf, const KGrid& g, const KParams& p,
                  double dt, double eps, int* err, cudaStream_t s) {
  k_prims<<<blocks_of(g, 128), 128, 0, s>>>(Q, prim, primf, g, p, dt, eps, 1.0 / eps, err);
}

void launch_q_from_prim(const double* P4, double* Q, int nc, cudaStream_t s) {
  if (nc > 0) k_q_from_prim<<<std::min((nc + 255) / 256, 152 * 8), 256, 0, s>>>(P4, Q, nc);
}

void launch_prims_f32(const double* Q, const double* prim, float* primf, const KGrid& g,
                      const KParams& p, double dt, double eps, int* err, cudaStream_t s) {
  k_prims_f32<<<blocks_of(g, 128), 128, 0, s>>>(Q, prim, primf, g, p, dt, eps, err);
}

void launch_prims_uT(const double* Q, double* prim, const KGrid& g, cudaStream_t s) {
  k_prims_uT<<<blocks_of(g, 256), 256, 0, s>>>(Q, prim, g.nx * g.ny);
}

void launch_macro_x1(const double* Qn, const MacroBufs& mb, const KGrid& g, const KParams& p,
                     double dt, double eps, int* err, cudaStream_t s) {
  k_macro_x1<<<blocks_of(g, 128), 128, 0, s>>>(Qn, mb, g, p, dt, eps, err);
}

void launch_macro_x2(const double* H, const MacroBufs& mb, const KGrid& g, const KParams& p,
                     double dt, int* err, cudaStream_t s) {
  k_macro_x2<<<blocks_of(g, 128), 128, 0, s>>>(H, mb, g, p, dt, err);
}

void launch_macro_y(const double* H, const MacroBufs& mb, double* Qn, const KGrid& g,
                    const KParams& p, double dt, double eps, int* err, cudaStream_t s,
                    const double* srcq) {
  k_macro_y<<<blocks_of(g, 128), 128, 0, s>>>(H, mb, Qn, g, p, dt, eps, err, srcq);
}

void launch_h_unpack(const float* Hf, double* H, const KGrid& g, double eps, cudaStream_t s) {
  k_h_unpack<<<blocks_of(g, 128), 128, 0, s>>>(Hf, H, g.nx * g.ny, eps * g.dv1 * g.dv2);
}

}  // namespace mmk

extern "C" mm_status mm_diag_erf(const double* x_dev, double* y_fast_dev, double* y_lib_dev,
                                 size_t n, void* cuda_stream) {
  if (!x_dev || !y_fast_dev || !y_lib_dev) return MM_ERR_INVALID_ARG;
  if (n == 0) return MM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  mmk::k_diag_erf<<<152 * 4, 256, 0, s>>>(x_dev, y_fast_dev, y_lib_dev, n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}
