// Learned heat-flux closure on the FP64 path (an extension of the library; the paper has no
// counterpart).  Per step, from Q^n:
//  - k_closure_features: 39 features of every cell (the 3x3 stencil of rho, u, T relative to the
//    cell times the cell Knudsen number k = eps sqrt(T) / (tau min(dx, dy)), the pressure
//    anisotropy, u / sqrt T, log10 eps, the relaxation weight omega1 and log10 k), the
//    Chapman-Enskog heat flux H_CE (closed-form third central moments of the transport part of
//    Ghat, Eq. 5-97: H111 = -3 eps p T_x / tau, H112 = -eps p T_y / tau, H122 = -eps p T_x / tau,
//    H222 = -3 eps p T_y / tau with the discrete gradient of Eq. 5-97more) and the scale
//    s = eps rho T^{3/2};
//  - the network (mm_mlp.cu) predicts y = (H - H_CE) / s;
//  - k_closure_decide: a cell takes the closure when max_m |y_m| <= threshold and it touches no
//    non-periodic boundary; its heat flux becomes H_CE + s y;
//  - k_closure_lists: work lists of the micro kernels: the y sweep runs on micro cells, the x sweep
//    on micro cells and their y neighbours (whose G* the y sweep reads); the refresh list holds
//    the cells of the micro cells' 3x3 blocks (the g^n the sweeps read) whose g^n the previous
//    step's micro update did not produce;
//  - k_closure_ghat: g^n = Ghat(Q^n) on the refresh list, before the sweeps (the asymptotic-
//    preserving limit of the relaxation, Eq. 5-98 with omega1 = 0).  Closure cells skip the micro
//    update and keep their g, which is read only after such a refresh.
// Collection of training data uses k_closure_features before and k_closure_targets after a
// plain step.
#include <algorithm>
#include <cmath>

#include "mm_body_macro.cuh"
#include "mm_body_micro.cuh"
#include "mm_body_mlp.cuh"

namespace mmk {

namespace {

constexpr int kF = MM_MLP_IN;
constexpr int kYo = MM_MLP_OUT;

// Neighbour index along one axis and whether it is the mirror image at a specular wall.
__device__ __forceinline__ int nb_index(int i, int d, int n, int bclo, int bchi, bool& mirror) {
  const int k = i + d;
  mirror = false;
  if (k >= 0 && k < n) return k;
  const int bc = k < 0 ? bclo : bchi;
  if (bc == MM_BC_PERIODIC) return (k + n) % n;
  mirror = bc == MM_BC_SPECULAR;
  return i;
}

__device__ __forceinline__ bool boundary_cell(const KGrid& g, const KParams& p, int i, int j) {
  return (i == 0 && p.bc[0] != MM_BC_PERIODIC) || (i == g.nx - 1 && p.bc[1] != MM_BC_PERIODIC) ||
         (j == 0 && p.bc[2] != MM_BC_PERIODIC) || (j == g.ny - 1 && p.bc[3] != MM_BC_PERIODIC);
}

// Features x[39] and (H_CE[4], scale) of cell c; the primitive variables of the stencil come from
// the prims kernel.
__device__ __forceinline__ void cell_features(const double* __restrict__ Q,
                                              const double* __restrict__ prim, const KGrid& g,
                                              const KParams& p, double eps, double log10_eps,
                                              double dt, int c, float* x, double aux5[5]) {
  // Differences of neighbouring FP64 fields are formed in FP64 (they cancel) and rounded once;
  // the scalings that multiply them, and the features that are not differences, are FP32: every
  // feature is within a few FP32 ulp of its FP64 value, which is all an FP32 network input can
  // carry, and the FP64 pipe (1/64 of the FP32 rate) keeps only the subtractions and H_CE.
  const int nc = g.nx * g.ny;
  const int i = c % g.nx, j = c / g.nx;
  const double rho = prim[P_RHO * nc + c];
  const double u1 = prim[P_U1 * nc + c], u2 = prim[P_U2 * nc + c];
  const double T = prim[P_T * nc + c];
  const double tau = prim[P_TAU * nc + c];
  const float rhof = (float)rho, Tf = (float)T, tauf = (float)tau, epsf = (float)eps;
  const float sTf = sqrtf(Tf);
  const float kn = epsf * sTf / (tauf * (float)fmin(g.dx, g.dy));
  const float sr = kn / rhof, su = kn / sTf, sT = kn / Tf;
  int f = 0;
  double TL = T, TR = T, TB = T, TT = T;
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj) {
    bool my;
    const int nj = nb_index(j, dj, g.ny, p.bc[2], p.bc[3], my);
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      if (di == 0 && dj == 0) continue;
      bool mx;
      const int ni = nb_index(i, di, g.nx, p.bc[0], p.bc[1], mx);
      const int n = nj * g.nx + ni;
      const double a1 = prim[P_U1 * nc + n], a2 = prim[P_U2 * nc + n];
      const double Tn = prim[P_T * nc + n];
      x[f++] = sr * (float)(prim[P_RHO * nc + n] - rho);
      x[f++] = su * (float)(mx ? -a1 - u1 : a1 - u1);
      x[f++] = su * (float)(my ? -a2 - u2 : a2 - u2);
      x[f++] = sT * (float)(Tn - T);
      if (dj == 0) (di < 0 ? TL : TR) = Tn;
      if (di == 0) (dj < 0 ? TB : TT) = Tn;
    }
  }
  const double th11 = prim[P_TH11 * nc + c], th22 = prim[P_TH22 * nc + c];
  const double P12 = Q[4 * nc + c] - rho * u1 * u2;
  const float iTf = 1.f / Tf;
  x[32] = (float)(th11 - th22) * (0.5f * iTf);
  x[33] = (float)P12 * (iTf / rhof);
  x[34] = (float)u1 / sTf;
  x[35] = (float)u2 / sTf;
  x[36] = (float)log10_eps;
  x[37] = epsf / fmaf((float)dt, tauf, epsf);
  x[38] = log10f(kn);
  // Chapman-Enskog heat flux with the discrete temperature gradient of Eq. (5-97more), FP64
  const double Tx = (0.5 * (TR + T) - 0.5 * (T + TL)) * g.idx;
  const double Ty = (0.5 * (TT + T) - 0.5 * (T + TB)) * g.idy;
  const double ep = eps * rho * T / tau;
  aux5[0] = -3.0 * ep * Tx;
  aux5[1] = -ep * Ty;
  aux5[2] = -ep * Tx;
  aux5[3] = -3.0 * ep * Ty;
  aux5[4] = eps * rho * T * sqrt(T);
}

__global__ void k_closure_features(const double* __restrict__ Q, const double* __restrict__ prim,
                                   KGrid g, KParams p, double eps, double log10_eps, double dt,
                                   float* __restrict__ X, double* __restrict__ aux) {
  const int nc = g.nx * g.ny;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  float x[kF];
  double a5[5];
  cell_features(Q, prim, g, p, eps, log10_eps, dt, c, x, a5);
  float* xo = X + (size_t)c * kF;
#pragma unroll
  for (int f = 0; f < kF; ++f) xo[f] = x[f];
#pragma unroll
  for (int m = 0; m < 5; ++m) aux[m * nc + c] = a5[m];
}

// Features, network and decision of the hybrid step in one pass over the cells (persistent
// CTAs, the network's weights staged once per CTA): the same arithmetic as k_closure_features,
// k_mlp_infer and k_closure_decide in sequence, without the feature and output arrays.
__global__ void __launch_bounds__(mlp_body::kInferThreads, 4)
    k_closure_predict(const double* __restrict__ Q, const double* __restrict__ prim,
                      const __nv_bfloat16* __restrict__ w, const float* __restrict__ norm,
                      KGrid g, KParams p, double eps, double log10_eps, double dt, float thr,
                      unsigned char* __restrict__ flags, double* __restrict__ H,
                      unsigned long long* __restrict__ nclosure) {
  using namespace mlp_body;
  extern __shared__ __align__(16) float smi[];
  float* sw = smi;
  float* sn = smi + kINP;
  float* tile = smi + kINP + 88 + (threadIdx.x >> 5) * kTile;
  stage_infer(w, norm, sw, sn);
  const int nc = g.nx * g.ny;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x; base < nc; base += gridDim.x * blockDim.x) {
    const int c = base + threadIdx.x;
    float x[kF];
    double a5[5] = {0, 0, 0, 0, 1};
    if (c < nc) {
      cell_features(Q, prim, g, p, eps, log10_eps, dt, c, x, a5);
    } else {
#pragma unroll
      for (int f = 0; f < kF; ++f) x[f] = sn[f];  // standardises to zero
    }
    float y[kOut];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if ((lane >> 4) == h) put_row(tile, lane & 15, x, sn);
      __syncwarp();
      infer16(sw, tile);
      if ((lane >> 4) == h) {
        const float* yr = tile + kTileY + (lane & 15) * 4;
#pragma unroll
        for (int o = 0; o < kOut; ++o) y[o] = yr[o];
      }
      __syncwarp();
    }
    bool cl = false;
    if (c < nc) {
      float ind = 0.f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) {
        y[o] = destandardise(y[o], sn, o);
        ind = fmaxf(ind, fabsf(y[o]));
      }
      const int i = c % g.nx, j = c / g.nx;
      cl = !boundary_cell(g, p, i, j) && ind <= thr;  // NaN fails the test: micro solve
      flags[c] = cl ? 1 : 0;
      if (cl)
        for (int m = 0; m < kOut; ++m) H[m * nc + c] = fma(a5[4], (double)y[m], a5[m]);
    }
    const unsigned b = __ballot_sync(0xffffffffu, cl);
    if (lane == 0 && b) atomicAdd(nclosure, (unsigned long long)__popc(b));
  }
}

__global__ void k_closure_targets(const double* __restrict__ H, const double* __restrict__ aux,
                                  float* __restrict__ Y, int nc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double is = 1.0 / aux[4 * nc + c];
  for (int m = 0; m < kYo; ++m) Y[(size_t)c * kYo + m] = (float)((H[m * nc + c] - aux[m * nc + c]) * is);
}

__global__ void k_closure_decide(const float* __restrict__ Y, const double* __restrict__ aux,
                                 float thr, KGrid g, KParams p, unsigned char* __restrict__ flags,
                                 double* __restrict__ H, unsigned long long* __restrict__ nclosure) {
  const int nc = g.nx * g.ny;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  bool cl = false;
  if (c < nc) {
    const int i = c % g.nx, j = c / g.nx;
    float y[kYo];
    float ind = 0.f;
    for (int m = 0; m < kYo; ++m) {
      y[m] = Y[(size_t)c * kYo + m];
      ind = fmaxf(ind, fabsf(y[m]));
    }
    cl = !boundary_cell(g, p, i, j) && ind <= thr;  // NaN fails the test: micro solve
    flags[c] = cl ? 1 : 0;
    if (cl) {
      const double s = aux[4 * nc + c];
      for (int m = 0; m < kYo; ++m) H[m * nc + c] = fma(s, (double)y[m], aux[m * nc + c]);
    }
  }
  const unsigned b = __ballot_sync(0xffffffffu, cl);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(nclosure, (unsigned long long)__popc(b));
}

// Append the cells with pred set to list (warp-aggregated; the order within the list does not
// matter: every cell's update is independent of the others').
__device__ __forceinline__ void append(bool pred, int c, int* list, int* count) {
  const unsigned full = 0xffffffffu;
  const unsigned b = __ballot_sync(full, pred);
  if (!b) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(b) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(b));
  base = __shfl_sync(full, base, leader);
  if (pred) list[base + __popc(b & ((1u << lane) - 1u))] = c;
}

// Work lists of a hybrid step.  x sweep: micro cells and their y neighbours (the y sweep reads
// their G*); y sweep: micro cells off diffuse walls; refresh: cells in the 3x3 block of a micro
// cell (the g^n the sweeps read) whose g^n was not produced by the micro update of the previous
// step (valid[c] == 0).  valid[c] then becomes this step's micro flag.
__global__ void k_closure_lists(const unsigned char* __restrict__ flags,
                                unsigned char* __restrict__ valid, KGrid g, KParams p,
                                int* __restrict__ xlist, int* __restrict__ ylist,
                                int* __restrict__ rlist, int* __restrict__ counts) {
  const int nc = g.nx * g.ny;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  bool inx = false, iny = false, inr = false;
  if (c < nc) {
    const int i = c % g.nx, j = c / g.nx;
    const bool micro = flags[c] == 0;
    bool ynb = false, blk = false;
    for (int dj = -1; dj <= 1; ++dj) {
      int nj = j + dj;
      if (nj < 0 || nj >= g.ny) {
        if (p.bc[dj < 0 ? 2 : 3] != MM_BC_PERIODIC) continue;
        nj = (nj + g.ny) % g.ny;
      }
      for (int di = -1; di <= 1; ++di) {
        int ni = i + di;
        if (ni < 0 || ni >= g.nx) {
          if (p.bc[di < 0 ? 0 : 1] != MM_BC_PERIODIC) continue;
          ni = (ni + g.nx) % g.nx;
        }
        const bool m = flags[nj * g.nx + ni] == 0;
        blk = blk || m;
        if (di == 0 && dj != 0) ynb = ynb || m;
      }
    }
    inx = micro || ynb;
    iny = micro && !micro_body::diffuse_wall_cell(g, p, i, j);
    inr = blk && valid[c] == 0;
    valid[c] = micro ? 1 : 0;
  }
  append(inx, c, xlist, counts);
  append(iny, c, ylist, counts + 1);
  append(inr, c, rlist, counts + 2);
}

// Cells whose g is not current (valid[c] == 0), to be reset to Ghat before a plain step.
__global__ void k_closure_stale(unsigned char* __restrict__ valid, int nc, int* __restrict__ rlist,
                                int* __restrict__ count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  bool st = false;
  if (c < nc) {
    st = valid[c] == 0;
    valid[c] = 1;
  }
  append(st, c, rlist, count);
}

// g^n = Ghat(Q^n) of Eq. (5-97) in the cells of a list, from the per-cell coefficients of the prims
// kernel (stored there times omega2, hence the factor 1/omega2 = (eps + dt tau) / (dt tau)):
// Ghat = (1/om2) [ -(p0 + p1 c2 + p2 c2^2 + p3 c2^3 + om2 mu / eps) e1 e2 + om2 KG / eps e^{-c.Tcal^{-1}c/2} ].
// Thread t owns v1 index k = t % nv1 and rows l = t / nv1 + m R, as in the micro kernels.
__global__ void __launch_bounds__(512, 1)
    k_closure_ghat(double* __restrict__ G, const double* __restrict__ prim, KGrid g, double dt,
                   double eps, int R, const int* __restrict__ list, const int* __restrict__ count,
                   double* __restrict__ Rm) {
  extern __shared__ double sm[];
  const int nv1 = g.nv1, nv2 = g.nv2;
  const int nc = g.nx * g.ny;
  double* e2t = sm;
  double* E1t = sm + nv2;
  double* E2t = sm + 2 * nv2;
  double* E3t = sm + 3 * nv2;
  double* g2t = sm + 4 * nv2;
  const int t = threadIdx.x;
  const int k = t % nv1, r = t / nv1;
  const bool active = r < R;
  const int n = *count;
  const size_t nv = (size_t)nv1 * nv2;
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    const int cell = list[q];
    const double u1 = prim[P_U1 * nc + cell], u2 = prim[P_U2 * nc + cell];
    const double inv2T = prim[P_INV2T * nc + cell];
    const double Ti11 = prim[P_TI11 * nc + cell], Ti12 = prim[P_TI12 * nc + cell];
    const double Ti22 = prim[P_TI22 * nc + cell];
    const double gam0 = prim[P_GAM0 * nc + cell], ome = prim[P_OME * nc + cell];
    const double dtt = dt * prim[P_TAU * nc + cell];
    const double iom2 = (eps + dtt) / dtt;
    for (int l = t; l < nv2; l += blockDim.x) {
      const double c2 = fma(l + 0.5, g.dv2, g.v2min) - u2;
      const double qq = c2 * c2;
      const double e2 = expd(-qq * inv2T);
      e2t[l] = e2;
      E1t[l] = e2 * c2;
      E2t[l] = e2 * qq;
      E3t[l] = e2 * qq * c2;
      g2t[l] = expd(-0.5 * Ti22 * qq);
    }
    const double c1 = fma(k + 0.5, g.dv1, g.v1min) - u1;
    const double c1q = c1 * c1;
    const double w01 = prim[P_W01 * nc + cell], w02 = prim[P_W02 * nc + cell];
    const double w03 = prim[P_W03 * nc + cell], w10 = prim[P_W10 * nc + cell];
    const double w11 = prim[P_W11 * nc + cell], w12 = prim[P_W12 * nc + cell];
    const double w20 = prim[P_W20 * nc + cell], w21 = prim[P_W21 * nc + cell];
    const double w30 = prim[P_W30 * nc + cell];
    const double e1 = expd(-c1q * inv2T) * iom2;
    const double A0 = -e1 * (c1 * fma(c1, fma(c1, w03, w02), w01) + ome);
    const double A1 = -e1 * fma(c1, fma(c1, w12, w11), w10);
    const double A2 = -e1 * fma(c1, w21, w20);
    const double A3 = -e1 * w30;
    const double gam1 = gam0 * iom2 * expd(-0.5 * Ti11 * c1q);
    const double c2r = fma(r + 0.5, g.dv2, g.v2min) - u2;
    double x = expd(-Ti12 * c1 * c2r);
    const double rat = expd(-Ti12 * c1 * (R * g.dv2));
    __syncthreads();
    if (active) {
      double* Go = G + (size_t)cell * nv + k;
      // with Rm (one row per pass): the row sums of the new g, as row_sums_body forms them
      double S0 = 0.0, S1 = 0.0, S2 = 0.0;
      for (int l = r; l < nv2; l += R) {
        double o = A0 * e2t[l];
        o = fma(A1, E1t[l], o);
        o = fma(A2, E2t[l], o);
        o = fma(A3, E3t[l], o);
        o = fma(gam1, g2t[l] * x, o);
        x *= rat;
        Go[l * nv1] = o;
        if (Rm) {
          const double v2 = fma(l + 0.5, g.dv2, g.v2min);
          S0 += o;
          S1 = fma(v2, o, S1);
          S2 = fma(v2 * v2, o, S2);
        }
      }
      if (Rm) micro_body::store_row_sums(Rm, cell, nv1, k, S0, S1, S2);
    }
    __syncthreads();
  }
}

}  // namespace

void launch_closure_features(const double* Q, const double* prim, const KGrid& g,
                             const KParams& p, double eps, double dt, float* X, double* aux,
                             cudaStream_t s) {
  const int nc = g.nx * g.ny;
  k_closure_features<<<(nc + 127) / 128, 128, 0, s>>>(Q, prim, g, p, eps, std::log10(eps), dt,
                                                      X, aux);
}

void launch_closure_predict(const double* Q, const double* prim, const mm_mlp* m,
                            const KGrid& g, const KParams& p, double eps, double dt, double thr,
                            unsigned char* flags, double* H, double* aux,
                            unsigned long long* nclosure, cudaStream_t s) {
  (void)aux;
  const __nv_bfloat16* w;
  const float* norm;
  mlp_device_params(m, &w, &norm);
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = mlp_body::infer_smem_bytes();
  cudaFuncSetAttribute(k_closure_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_closure_predict, mlp_body::kInferThreads,
                                                smem);
  const int nc = g.nx * g.ny;
  const int need = (nc + mlp_body::kInferThreads - 1) / mlp_body::kInferThreads;
  const int blocks = std::max(1, std::min(need, (nsm > 0 ? nsm : 1) * (per > 0 ? per : 1)));
  k_closure_predict<<<blocks, mlp_body::kInferThreads, smem, s>>>(
      Q, prim, w, norm, g, p, eps, std::log10(eps), dt, (float)thr, flags, H, nclosure);
}

void launch_closure_targets(const double* H, const double* aux, float* Y, const KGrid& g,
                            cudaStream_t s) {
  const int nc = g.nx * g.ny;
  k_closure_targets<<<(nc + 255) / 256, 256, 0, s>>>(H, aux, Y, nc);
}

void launch_closure_decide(const float* Y, const double* aux, double thr, const KGrid& g,
                           const KParams& p, unsigned char* flags, double* H,
                           unsigned long long* nclosure, cudaStream_t s) {
  const int nc = g.nx * g.ny;
  k_closure_decide<<<(nc + 255) / 256, 256, 0, s>>>(Y, aux, (float)thr, g, p, flags, H, nclosure);
}

void launch_closure_lists(const unsigned char* flags, unsigned char* valid, const KGrid& g,
                          const KParams& p, int* lists, int* counts, cudaStream_t s) {
  const int nc = g.nx * g.ny;
  cudaMemsetAsync(counts, 0, 3 * sizeof(int), s);
  k_closure_lists<<<(nc + 255) / 256, 256, 0, s>>>(flags, valid, g, p, lists, lists + nc,
                                                   lists + 2 * nc, counts);
}

void launch_closure_stale(unsigned char* valid, const KGrid& g, int* list, int* count,
                          cudaStream_t s) {
  const int nc = g.nx * g.ny;
  cudaMemsetAsync(count, 0, sizeof(int), s);
  k_closure_stale<<<(nc + 255) / 256, 256, 0, s>>>(valid, nc, list, count);
}

int closure_ghat_blocks(const MicroShape& ms) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_closure_ghat, ms.threads, ms.smem_ghat);
  return (nsm > 0 ? nsm : 1) * (per > 0 ? per : 1);
}

void launch_closure_ghat(double* G, const double* prim, const KGrid& g, double dt, double eps,
                         const MicroShape& ms, const int* list, const int* count, int blocks,
                         cudaStream_t s, double* Rm) {
  if (ms.smem_ghat > 48 * 1024)
    cudaFuncSetAttribute(k_closure_ghat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms.smem_ghat);
  k_closure_ghat<<<blocks, ms.threads, ms.smem_ghat, s>>>(G, prim, g, dt, eps, ms.R, list, count,
                                                          ms.R == 1 ? Rm : nullptr);
}

}  // namespace mmk
