// Micro (phase-space) kernels of the micro-macro KFVS step: Section 5.3 of Rossmanith & Sar,
// arXiv 2509.21832 (split upwind transport with the projector Pi_M, backward-Euler relaxation
// toward Ghat, Eq. 5-99 heat-flux moments) and the diffuse-wall Ghat of Section 6.3.
//
// Mapping: one CTA per spatial cell.  Thread t owns the v1 index k = t % nv1 and the v2 rows
// l = t / nv1 + m R (m = 0, 1, ...), where R rows are covered per pass so that R * nv1 fills
// whole warps.  Everything that depends on k only (c1, the Maxwellian factor e1[k], upwind
// coefficients, polynomial coefficients) lives in registers; everything that depends on l only
// lives in shared-memory tables.  The Maxwellian is separable, M = rho/(2 pi T) e1[k] e2[l]; the
// ES Gaussian is K e^{-a c1^2/2} e^{-d c2^2/2} e^{-b c1 c2}, the last factor advanced along a
// thread's rows by a multiplicative recurrence.  Velocity sums are accumulated per thread in the
// order of its rows, then combined across the CTA with warp shuffles and shared memory.
#include <algorithm>
#include <cmath>

#include "mm_body_micro.cuh"

namespace mmk {

namespace {

using namespace micro_body;

template <typename Tg, int NR>
__global__ void __launch_bounds__(NR > 0 ? 256 : 512, 1) k_micro_x(const Tg* __restrict__ Gin,
                                                    Tg* __restrict__ Gout,
                                                    const double* __restrict__ prim, KGrid g,
                                                    KParams p, double dtidx, int R, int cell0,
                                                    double* __restrict__ Ee) {
  extern __shared__ double sm[];
  micro_x_body<Tg, NR>(Gin, Gout, prim, g, p, dtidx, R, cell0 + (int)blockIdx.x, sm, Ee);
}

template <typename Tg>
__global__ void __launch_bounds__(32) k_micro_x_rows(const Tg* __restrict__ Gin,
                                                     Tg* __restrict__ Gout,
                                                     const double* __restrict__ prim,
                                                     const double* __restrict__ Rm,
                                                     double* __restrict__ Ee, KGrid g, KParams p,
                                                     double dtidx, int cell0) {
  extern __shared__ double sm[];
  micro_x_rows_body<Tg>(Gin, Gout, prim, Rm, Ee, g, p, dtidx, cell0 + (int)blockIdx.x, sm);
}

// The x sweep from the row sums over a list of cells (persistent CTAs of one warp).
template <typename Tg>
__global__ void __launch_bounds__(32) k_micro_x_rows_list(const Tg* __restrict__ Gin,
                                                          Tg* __restrict__ Gout,
                                                          const double* __restrict__ prim,
                                                          const double* __restrict__ Rm,
                                                          double* __restrict__ Ee, KGrid g,
                                                          KParams p, double dtidx,
                                                          const int* __restrict__ list,
                                                          const int* __restrict__ count) {
  extern __shared__ double sm[];
  const int n = *count;
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    micro_x_rows_body<Tg>(Gin, Gout, prim, Rm, Ee, g, p, dtidx, list[q], sm);
    __syncthreads();
  }
}

// Row sums of the cells [cell0, cell0 + ncells): persistent one-warp CTAs, each tabulating v2 and
// v2^2 of the rows once in shared memory.
__global__ void __launch_bounds__(32) k_row_sums(const double* __restrict__ G,
                                                 double* __restrict__ Rm, KGrid g, int cell0,
                                                 int ncells) {
  extern __shared__ double vt[];
  for (int l = threadIdx.x; l < g.nv2; l += 32) {
    const double v2 = fma(l + 0.5, g.dv2, g.v2min);
    vt[l] = v2;
    vt[g.nv2 + l] = v2 * v2;
  }
  __syncwarp();
  for (int q = blockIdx.x; q < ncells; q += gridDim.x)
    row_sums_body<double>(G, Rm, g, cell0 + q, vt);
}


template <typename Tg>
__global__ void __launch_bounds__(512, 1) k_micro_y(const Tg* __restrict__ Gs,
                                                    Tg* __restrict__ Gout,
                                                    double* __restrict__ Hout,
                                                    const double* __restrict__ prim, KGrid g,
                                                    KParams p, double dtidy, double hscale, int R,
                                                    int* __restrict__ err,
                                                    const double* __restrict__ src, int cell0,
                                                    double* __restrict__ Rm,
                                                    const double* __restrict__ Ee) {
  extern __shared__ double sm[];
  micro_y_body<Tg>(Gs, Gout, Hout, prim, g, p, dtidy, hscale, R, err, cell0 + (int)blockIdx.x, sm,
                   src, Rm, Ee);
}

template <typename Tg>
__global__ void __launch_bounds__(512, 1) k_micro_y_wall(const Tg* __restrict__ Gs,
                                                         Tg* __restrict__ Gout,
                                                         double* __restrict__ Hout,
                                                         const double* __restrict__ prim,
                                                         const int* __restrict__ wall_cells,
                                                         KGrid g, KParams p, double dt, double eps,
                                                         int R, int* __restrict__ err,
                                                         double* __restrict__ Rm) {
  extern __shared__ double sm[];
  micro_y_wall_body<Tg>(Gs, Gout, Hout, prim, g, p, dt, eps, R, err, wall_cells[blockIdx.x], sm,
                        Rm);
}

// The same sweeps over a list of cells: persistent CTAs take cells q = blockIdx.x + m gridDim.x.
template <typename Tg, int NR>
__global__ void __launch_bounds__(NR > 0 ? 256 : 512, 1) k_micro_x_list(const Tg* __restrict__ Gin,
                                                         Tg* __restrict__ Gout,
                                                         const double* __restrict__ prim, KGrid g,
                                                         KParams p, double dtidx, int R,
                                                         const int* __restrict__ list,
                                                         const int* __restrict__ count,
                                                         double* __restrict__ Ee) {
  extern __shared__ double sm[];
  const int n = *count;
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    micro_x_body<Tg, NR>(Gin, Gout, prim, g, p, dtidx, R, list[q], sm, Ee);
    __syncthreads();
  }
}

template <typename Tg>
__global__ void __launch_bounds__(512, 1) k_micro_y_list(const Tg* __restrict__ Gs,
                                                         Tg* __restrict__ Gout,
                                                         double* __restrict__ Hout,
                                                         const double* __restrict__ prim, KGrid g,
                                                         KParams p, double dtidy, double hscale,
                                                         int R, int* __restrict__ err,
                                                         const int* __restrict__ list,
                                                         const int* __restrict__ count,
                                                         double* __restrict__ Rm,
                                                         const double* __restrict__ Ee) {
  extern __shared__ double sm[];
  const int n = *count;
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    micro_y_body<Tg>(Gs, Gout, Hout, prim, g, p, dtidy, hscale, R, err, list[q], sm, nullptr,
                     Rm, Ee);
    __syncthreads();
  }
}

__global__ void k_diag_exp(const double* __restrict__ x, double* __restrict__ yf,
                           double* __restrict__ yl, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x) {
    yf[q] = expd(x[q]);
    yl[q] = exp(x[q]);
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x)
    out[q] = (float)in[q];
}
__global__ void k_f32_to_f64(const float* __restrict__ in, double* __restrict__ out, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x)
    out[q] = (double)in[q];
}

}  // namespace

int x_rows(const MicroShape& ms, int nv2);

MicroShape micro_shape(int nv1, int nv2) {
  MicroShape ms{1, 32, 0, 0, 0, 0};
  double best = -1.0;
  // nv1 <= 32: one warp per cell, R = 32 div nv1 rows per pass.  Measured on GB300 (FP64 step,
  // 160^2 cells): against CTAs of several warps with full lanes it is 1.2x faster at 24^2 and
  // 1.6-4x at 17^2 ... 22^2 -- no cross-warp reductions, and the per-cell work (tables, sums,
  // coefficients) spread over the most rows per thread outweigh the idle lanes.
  if (nv1 <= 32) {
    ms.R = std::min(32 / nv1, nv2);
    ms.threads = 32;
    best = 2.0;
  }
  // wider meshes: the CTA size (whole warps, at most kMaxThreads) with the fewest idle lanes
  for (int R = 1; R <= 32 && best < 2.0; ++R) {
    const int thr = R * nv1;
    if (thr > micro_body::kMaxThreads) break;
    const int thr32 = (thr + 31) / 32 * 32;
    const int passes = (nv2 + R - 1) / R;
    const double u = (double)thr / thr32 * ((double)nv2 / (R * passes));
    if (u > best + 1e-9) {
      best = u;
      ms.R = R;
      ms.threads = thr32;
    }
    if (R >= nv2) break;
  }
  ms.smem_x = sizeof(double) * (micro_body::kRed + 4 * (size_t)nv2);
  ms.smem_y = sizeof(double) * (micro_body::kRed + micro_body::kYTables * (size_t)nv2);
  ms.smem_ghat = sizeof(double) * 5 * (size_t)nv2;
  ms.xrows = x_rows(ms, nv2);
  return ms;
}

// Rows per thread when the x sweep keeps its upwind differences in registers (the shapes of the
// common velocity meshes: 32^2 with R = 1, 16^2 with R = 2, 24^2 with R = 4; CTAs of at most
// 256 threads, so that a thread may hold up to 255 registers), else 0.
int x_rows(const MicroShape& ms, int nv2) {
  const int nr = nv2 % ms.R == 0 ? nv2 / ms.R : 0;
  return ms.threads <= 256 && (nr == 32 || nr == 24 || nr == 8 || nr == 6) ? nr : 0;
}

template <typename Tg, typename F>
void with_x_kernel(int nr, F&& f) {
  switch (nr) {
    case 32: f(k_micro_x<Tg, 32>); break;
    case 24: f(k_micro_x<Tg, 24>); break;
    case 8: f(k_micro_x<Tg, 8>); break;
    case 6: f(k_micro_x<Tg, 6>); break;
    default: f(k_micro_x<Tg, 0>); break;
  }
}

template <typename Tg, typename F>
void with_x_list_kernel(int nr, F&& f) {
  switch (nr) {
    case 32: f(k_micro_x_list<Tg, 32>); break;
    case 24: f(k_micro_x_list<Tg, 24>); break;
    case 8: f(k_micro_x_list<Tg, 8>); break;
    case 6: f(k_micro_x_list<Tg, 6>); break;
    default: f(k_micro_x_list<Tg, 0>); break;
  }
}

int micro_list_blocks(const MicroShape& ms, bool ysweep) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (ysweep) {
    if (ms.smem_y > 48 * 1024)
      cudaFuncSetAttribute(k_micro_y_list<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms.smem_y);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_micro_y_list<double>, ms.threads, ms.smem_y);
  } else {
    with_x_list_kernel<double>(ms.xrows, [&](auto kern) {
      if (ms.smem_x > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms.smem_x);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, ms.threads, ms.smem_x);
    });
  }
  return (nsm > 0 ? nsm : 1) * (per > 0 ? per : 1);
}

template <typename Tg>
void launch_micro_x_list(const Tg* Gin, Tg* Gout, const double* prim, const KGrid& g,
                         const KParams& p, double dt, const MicroShape& ms, const int* list,
                         const int* count, int blocks, cudaStream_t s, const double* Rm,
                         double* Ee) {
  if (Rm && ms.R == 1) {
    k_micro_x_rows_list<Tg><<<blocks, 32, ms.smem_x, s>>>(Gin, Gout, prim, Rm, Ee, g, p,
                                                          dt * g.idx, list, count);
    return;
  }
  with_x_list_kernel<Tg>(ms.xrows, [&](auto kern) {
    kern<<<blocks, ms.threads, ms.smem_x, s>>>(Gin, Gout, prim, g, p, dt * g.idx, ms.R, list,
                                              count, Ee);
  });
}

template <typename Tg>
void launch_micro_y_list(const Tg* Gs, Tg* Gout, double* H, const double* prim, const KGrid& g,
                         const KParams& p, double dt, double eps, const MicroShape& ms, int* err,
                         const int* list, const int* count, int blocks, cudaStream_t s,
                         double* Rm, const double* Ee) {
  k_micro_y_list<Tg><<<blocks, ms.threads, ms.smem_y, s>>>(Gs, Gout, H, prim, g, p, dt * g.idy,
                                                           eps * g.dv1 * g.dv2, ms.R, err, list,
                                                           count, ms.R == 1 ? Rm : nullptr, Ee);
}

void launch_row_sums(const double* G, double* Rm, const KGrid& g, cudaStream_t s, int cell0,
                     int ncells) {
  const int n = ncells < 0 ? g.nx * g.ny : ncells;
  if (n > 0)
    k_row_sums<<<std::min(n, 152 * 32), 32, 2 * (size_t)g.nv2 * sizeof(double), s>>>(G, Rm, g,
                                                                                     cell0, n);
}


// Row sums of the cells of a rectangle [i0, i0 + wi) x [j0, j0 + n / wi): persistent one-warp
// CTAs, as k_row_sums.
__global__ void __launch_bounds__(32) k_row_sums_rect(const double* __restrict__ G,
                                                      double* __restrict__ Rm, KGrid g, int i0,
                                                      int wi, int j0, int n) {
  extern __shared__ double vt[];
  for (int l = threadIdx.x; l < g.nv2; l += 32) {
    const double v2 = fma(l + 0.5, g.dv2, g.v2min);
    vt[l] = v2;
    vt[g.nv2 + l] = v2 * v2;
  }
  __syncwarp();
  for (int q = blockIdx.x; q < n; q += gridDim.x)
    row_sums_body<double>(G, Rm, g, (j0 + q / wi) * g.nx + i0 + q % wi, vt);
}

void launch_row_sums_rect(const double* G, double* Rm, const KGrid& g, int i0, int i1, int j0,
                          int j1, cudaStream_t s) {
  const int wi = i1 - i0, n = wi * (j1 - j0);
  if (wi > 0 && n > 0)
    k_row_sums_rect<<<std::min(n, 152 * 32), 32, 2 * (size_t)g.nv2 * sizeof(double), s>>>(
        G, Rm, g, i0, wi, j0, n);
}

template void launch_micro_x_list<double>(const double*, double*, const double*, const KGrid&,
                                          const KParams&, double, const MicroShape&, const int*,
                                          const int*, int, cudaStream_t, const double*, double*);
template void launch_micro_y_list<double>(const double*, double*, double*, const double*,
                                          const KGrid&, const KParams&, double, double,
                                          const MicroShape&, int*, const int*, const int*, int,
                                          cudaStream_t, double*, const double*);

template <typename Tg>
void launch_micro_x(const Tg* Gin, Tg* Gout, const double* prim, const KGrid& g,
                    const KParams& p, double dt, const MicroShape& ms, cudaStream_t s, int cell0,
                    int ncells, double* Ee) {
  const int n = ncells < 0 ? g.nx * g.ny : ncells;
  if (n <= 0) return;
  with_x_kernel<Tg>(ms.xrows, [&](auto kern) {
    if (ms.smem_x > 48 * 1024)
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms.smem_x);
    kern<<<n, ms.threads, ms.smem_x, s>>>(Gin, Gout, prim, g, p, dt * g.idx, ms.R, cell0, Ee);
  });
}

template <typename Tg>
void launch_micro_y(const Tg* Gs, Tg* Gout, double* H, const double* prim, const KGrid& g,
                    const KParams& p, double dt, double eps, const MicroShape& ms, int* err,
                    cudaStream_t s, const double* src, int cell0, int ncells, double* Rm,
                    const double* Ee) {
  const int n = ncells < 0 ? g.nx * g.ny : ncells;
  if (n <= 0) return;
  if (ms.smem_y > 48 * 1024)
    cudaFuncSetAttribute(k_micro_y<Tg>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms.smem_y);
  k_micro_y<Tg><<<n, ms.threads, ms.smem_y, s>>>(Gs, Gout, H, prim, g, p, dt * g.idy,
                                                 eps * g.dv1 * g.dv2, ms.R, err, src, cell0,
                                                 ms.R == 1 ? Rm : nullptr, Ee);
}

template <typename Tg>
void launch_micro_x_rows(const Tg* Gin, Tg* Gout, const double* prim, const double* Rm,
                         const KGrid& g, const KParams& p, double dt, const MicroShape& ms,
                         cudaStream_t s, int cell0, int ncells, double* Ee) {
  const int n = ncells < 0 ? g.nx * g.ny : ncells;
  if (n <= 0) return;
  if (ms.smem_x > 48 * 1024)
    cudaFuncSetAttribute(k_micro_x_rows<Tg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ms.smem_x);
  k_micro_x_rows<Tg><<<n, 32, ms.smem_x, s>>>(Gin, Gout, prim, Rm, Ee, g, p, dt * g.idx, cell0);
}

template <typename Tg>
void launch_micro_y_wall(const Tg* Gs, Tg* Gout, double* H, const double* prim,
                         const int* wall_cells, int n_wall, const KGrid& g, const KParams& p,
                         double dt, double eps, const MicroShape& ms, int* err, cudaStream_t s,
                         double* Rm) {
  if (n_wall <= 0) return;
  const size_t smem = sizeof(double) * micro_body::wall_smem_doubles(g.nv1, g.nv2);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_micro_y_wall<Tg>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_micro_y_wall<Tg><<<n_wall, ms.threads, smem, s>>>(
      Gs, Gout, H, prim, wall_cells, g, p, dt, eps, ms.R, err, ms.R == 1 ? Rm : nullptr);
}

template void launch_micro_x<double>(const double*, double*, const double*, const KGrid&,
                                     const KParams&, double, const MicroShape&, cudaStream_t, int,
                                     int, double*);
template void launch_micro_y<double>(const double*, double*, double*, const double*,
                                     const KGrid&, const KParams&, double, double,
                                     const MicroShape&, int*, cudaStream_t, const double*, int,
                                     int, double*, const double*);
template void launch_micro_x_rows<double>(const double*, double*, const double*, const double*,
                                          const KGrid&, const KParams&, double, const MicroShape&,
                                          cudaStream_t, int, int, double*);
template void launch_micro_y_wall<double>(const double*, double*, double*, const double*,
                                          const int*, int, const KGrid&, const KParams&, double,
                                          double, const MicroShape&, int*, cudaStream_t, double*);

// FP64 pipe probe: 8 independent FMA chains per thread, so that issue, not latency, bounds it.
__global__ void k_diag_fp64_fma(double* __restrict__ out, int iters, double a, double b) {
  double d[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) d[c] = 1.0 + (threadIdx.x + 32 * c) / 256.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) d[c] = fma(a, d[c], b);
  }
  double sum = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) sum += d[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

void launch_diag_fp64_fma(double* out, int ctas, int iters, cudaStream_t s) {
  k_diag_fp64_fma<<<ctas, 256, 0, s>>>(out, iters, 1.0 - 0x1p-20, 0x1p-30);
}

void launch_diag_exp(const double* x, double* yf, double* yl, size_t n, cudaStream_t s) {
  k_diag_exp<<<152 * 4, 256, 0, s>>>(x, yf, yl, n);
}

void launch_convert_f64_to_f32(const double* in, float* out, size_t n, cudaStream_t s) {
  k_f64_to_f32<<<152 * 8, 256, 0, s>>>(in, out, n);
}
void launch_convert_f32_to_f64(const float* in, double* out, size_t n, cudaStream_t s) {
  k_f32_to_f64<<<152 * 8, 256, 0, s>>>(in, out, n);
}

}  // namespace mmk

extern "C" mm_status mm_diag_fp64_fma(double* out_dev, int ctas, int iters, void* cuda_stream) {
  if (!out_dev || ctas < 1 || iters < 1) return MM_ERR_INVALID_ARG;
  mmk::launch_diag_fp64_fma(out_dev, ctas, iters, static_cast<cudaStream_t>(cuda_stream));
  return cudaGetLastError() == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

extern "C" mm_status mm_diag_exp(const double* x_dev, double* y_fast_dev, double* y_lib_dev,
                                 size_t n, void* cuda_stream) {
  if (!x_dev || !y_fast_dev || !y_lib_dev) return MM_ERR_INVALID_ARG;
  if (n == 0) return MM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  mmk::launch_diag_exp(x_dev, y_fast_dev, y_lib_dev, n, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}
