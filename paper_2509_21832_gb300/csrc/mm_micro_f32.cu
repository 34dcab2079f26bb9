// FP32-g phase-space kernels of the micro step (Section 5.3 of Rossmanith & Sar, arXiv
// 2509.21832): the same split upwind transport with projection, relaxation toward Ghat and heat
// flux as mm_micro.cu, with g stored and transported in FP32.
//
// Precision split: no FP64 instruction runs here (the FP64 pipe of GB300 runs at 1/61 of FP32
// and a warp instruction costs its full issue time even with one active lane, so an FP64
// epilogue per cell would bound the kernel); per-cell coefficients come from the prims kernel,
// computed in FP64 and rounded once; each warp's velocity sums are FP32 (per-thread partial sums
// over its rows, then a pairwise butterfly); the warps' sums are combined with compensated
// (Neumaier) FP32 summation; the heat flux leaves as (hi, lo) pairs that are combined in FP64 by
// the per-cell unpack kernel.
#include <cmath>

#include "mm_internal.cuh"

namespace mmk {

namespace {

constexpr int kPartF = 128;  // floats: 32 warps x 4 partial sums
constexpr int kHeadF = 136;  // floats before the tables: partials + 8 broadcast slots

// Transposing butterfly over a warp for four floats; the warp's totals are written to
// part[warp * 4 + m] by lanes 0, 8, 16, 24.
__device__ __forceinline__ void warp_sum4f(const float v[4], float* part) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool h16 = lane & 16;
  const float s0 = h16 ? v[0] : v[2];
  const float s1 = h16 ? v[1] : v[3];
  const float k0 = (h16 ? v[2] : v[0]) + __shfl_xor_sync(full, s0, 16);
  const float k1 = (h16 ? v[3] : v[1]) + __shfl_xor_sync(full, s1, 16);
  const bool h8 = lane & 8;
  const float s = h8 ? k0 : k1;
  float kk = (h8 ? k1 : k0) + __shfl_xor_sync(full, s, 8);
  kk += __shfl_xor_sync(full, kk, 4);
  kk += __shfl_xor_sync(full, kk, 2);
  kk += __shfl_xor_sync(full, kk, 1);
  if ((lane & 7) == 0) part[warp * 4 + (lane >> 3)] = kk;
}

// Compensated (Neumaier) sum of the warps' partial sums: value ~ hi + lo.
__device__ __forceinline__ void sum_parts(const float* part, float hi[4], float lo[4]) {
  const int nw = (blockDim.x + 31) >> 5;
  for (int m = 0; m < 4; ++m) {
    float s = 0.f, c = 0.f;
    for (int w = 0; w < nw; ++w) {
      const float x = part[w * 4 + m];
      const float t = s + x;
      c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    hi[m] = s;
    lo[m] = c;
  }
}

__device__ __forceinline__ bool diffuse_wall_cell(const KGrid& g, const KParams& p, int i, int j) {
  return (i == 0 && p.bc[0] == MM_BC_DIFFUSE) || (i == g.nx - 1 && p.bc[1] == MM_BC_DIFFUSE) ||
         (j == 0 && p.bc[2] == MM_BC_DIFFUSE) || (j == g.ny - 1 && p.bc[3] == MM_BC_DIFFUSE);
}

struct UpwindF {
  int cell;
  bool mirror, zero;
};

__device__ __forceinline__ UpwindF upwind_side(const KGrid& g, const KParams& p, int i, int j,
                                               int s) {
  UpwindF u{0, false, false};
  int ni = i, nj = j;
  if (s == 0) ni = i - 1;
  if (s == 1) ni = i + 1;
  if (s == 2) nj = j - 1;
  if (s == 3) nj = j + 1;
  const bool out = ni < 0 || ni >= g.nx || nj < 0 || nj >= g.ny;
  if (out) {
    const int bc = p.bc[s];
    if (bc == MM_BC_PERIODIC) {
      ni = (ni + g.nx) % g.nx;
      nj = (nj + g.ny) % g.ny;
    } else {
      ni = i;
      nj = j;
      u.mirror = bc == MM_BC_SPECULAR;
      u.zero = bc == MM_BC_DIFFUSE;
    }
  }
  u.cell = nj * g.nx + ni;
  return u;
}

// x sweep, Eqs. (zmicrox)-(update-micro-2D-xdir)
__global__ void __launch_bounds__(512, 1) k_micro_x_f32(const float* __restrict__ Gin,
                                                        float* __restrict__ Gout,
                                                        const float* __restrict__ pf, KGrid g,
                                                        KGridF gf, KParams p, float dtidx,
                                                        int R) {
  extern __shared__ float smf[];
  const int nv1 = g.nv1, nv2 = g.nv2;
  float* part = smf;
  float* bco = smf + kPartF;
  float* c2t = smf + kHeadF;
  float* c2q = c2t + nv2;
  float* e2t = c2q + nv2;
  float* qet = e2t + nv2;

  const int nc = g.nx * g.ny;
  const int cell = blockIdx.x;
  const int i = cell % g.nx, j = cell / g.nx;
  const int t = threadIdx.x;
  const int k = t % nv1, r = t / nv1;
  const bool active = r < R;

  const float u1 = pf[F_U1 * nc + cell], u2 = pf[F_U2 * nc + cell];
  const float inv2T = pf[F_INV2T * nc + cell], iT = pf[F_IT * nc + cell];
  const float kap = pf[F_KAP * nc + cell];
  const float v1min = gf.v1min, v2min = gf.v2min, dv1 = gf.dv1, dv2 = gf.dv2;

  for (int l = t; l < nv2; l += blockDim.x) {
    const float c2 = fmaf(l + 0.5f, dv2, v2min) - u2;
    const float q = c2 * c2;
    c2t[l] = c2;
    c2q[l] = q;
    e2t[l] = expf(-q * inv2T);
  }
  const float v1 = fmaf(k + 0.5f, dv1, v1min);
  const float c1 = v1 - u1;
  const float av = fabsf(v1);
  const float sig = -av * gf.idx;
  const float lam = av * dtidx;
  const UpwindF up = upwind_side(g, p, i, j, v1 > 0.f ? 0 : 1);
  const int ku = up.mirror ? nv1 - 1 - k : k;
  const size_t nv = (size_t)nv1 * nv2;
  const float* Gc = Gin + (size_t)cell * nv + k;
  const float* Gu = Gin + (size_t)up.cell * nv + ku;
  __syncthreads();

  float D0 = 0.f, D1 = 0.f, D2 = 0.f;
  if (active) {
    for (int l = r; l < nv2; l += R) {
      const float gv = Gc[l * nv1];
      const float gu = up.zero ? 0.f : Gu[l * nv1];
      const float d = gu - gv;
      D0 += d;
      D1 = fmaf(c2t[l], d, D1);
      D2 = fmaf(c2q[l], d, D2);
    }
  }
  const float sD0 = sig * D0;
  const float S[4] = {sD0, c1 * sD0, sig * D1, fmaf(c1 * c1, sD0, sig * D2)};
  warp_sum4f(S, part);
  __syncthreads();
  if (t == 0) {
    float hi[4], lo[4];
    sum_parts(part, hi, lo);
    const float S0 = hi[0] + lo[0], S1 = hi[1] + lo[1], S2 = hi[2] + lo[2], S3 = hi[3] + lo[3];
    bco[0] = fmaf(-S3, inv2T, 2.f * S0);
    bco[1] = S1 * iT;
    bco[2] = S2 * iT;
    bco[3] = fmaf(0.25f * S3, iT * iT, -S0 * inv2T);
  }
  __syncthreads();
  const float b0 = bco[0], b1 = bco[1], b2 = bco[2], gm = bco[3];
  for (int l = t; l < nv2; l += blockDim.x) qet[l] = e2t[l] * fmaf(b2, c2t[l], gm * c2q[l]);
  const float e1 = expf(-c1 * c1 * inv2T);
  const float bk = kap * e1;
  const float ak = bk * fmaf(gm * c1, c1, fmaf(b1, c1, b0));
  __syncthreads();

  if (active) {
    float* Go = Gout + (size_t)cell * nv + k;
    for (int l = r; l < nv2; l += R) {
      const float gv = Gc[l * nv1];
      const float gu = up.zero ? 0.f : Gu[l * nv1];
      const float d = gu - gv;
      float o = fmaf(lam, d, gv);
      o = fmaf(ak, e2t[l], o);
      o = fmaf(bk, qet[l], o);
      Go[l * nv1] = o;
    }
  }
}

constexpr int kYTablesF = 13;

// y sweep + relaxation + heat flux (Eqs. zmicroy-update-micro-2D-ydir, 5-97, 5-98, 5-99) for
// cells not adjacent to a diffuse wall
__global__ void __launch_bounds__(512, 1) k_micro_y_f32(const float* __restrict__ Gs,
                                                        float* __restrict__ Gout,
                                                        float* __restrict__ Hf,
                                                        const float* __restrict__ pf, KGrid g,
                                                        KGridF gf, KParams p, float dtidy,
                                                        int R) {
  extern __shared__ float smf[];
  const int nv1 = g.nv1, nv2 = g.nv2;
  const int nc = g.nx * g.ny;
  const int cell = blockIdx.x;
  const int i = cell % g.nx, j = cell / g.nx;
  if (diffuse_wall_cell(g, p, i, j)) return;

  float* part = smf;
  float* bco = smf + kPartF;
  float* tb = smf + kHeadF;
  float* c2t = tb;
  float* c2q = tb + nv2;
  float* c2c = tb + 2 * nv2;
  float* e2t = tb + 3 * nv2;
  float* g2t = tb + 4 * nv2;
  float* v2t = tb + 5 * nv2;
  float* s0t = tb + 6 * nv2;
  float* s1t = tb + 7 * nv2;
  float* s2t = tb + 8 * nv2;
  float* wlt = tb + 9 * nv2;
  float* E1t = tb + 10 * nv2;
  float* E2t = tb + 11 * nv2;
  float* E3t = tb + 12 * nv2;

  const int t = threadIdx.x;
  const int k = t % nv1, r = t / nv1;
  const bool active = r < R;

  const float u1 = pf[F_U1 * nc + cell], u2 = pf[F_U2 * nc + cell];
  const float inv2T = pf[F_INV2T * nc + cell], iT = pf[F_IT * nc + cell];
  const float Ti11h = pf[F_TI11H * nc + cell], Ti12 = pf[F_TI12 * nc + cell];
  const float Ti22h = pf[F_TI22H * nc + cell];
  const float om1 = pf[F_OM1 * nc + cell], om1kap = pf[F_OM1KAP * nc + cell];
  const float gam0 = pf[F_GAM0 * nc + cell], ome = pf[F_OME * nc + cell];
  const float v1min = gf.v1min, v2min = gf.v2min, dv1 = gf.dv1, dv2 = gf.dv2;
  const float idy = gf.idy;

  for (int l = t; l < nv2; l += blockDim.x) {
    const float v2 = fmaf(l + 0.5f, dv2, v2min);
    const float c2 = v2 - u2;
    const float q = c2 * c2;
    const float e2 = expf(-q * inv2T);
    const float av = fabsf(v2);
    const float sg = -av * idy;
    c2t[l] = c2;
    c2q[l] = q;
    c2c[l] = q * c2;
    e2t[l] = e2;
    g2t[l] = expf(-Ti22h * q);
    v2t[l] = v2;
    s0t[l] = sg;
    s1t[l] = sg * c2;
    s2t[l] = sg * q;
    wlt[l] = om1 * (av * dtidy);
    E1t[l] = e2 * c2;
    E2t[l] = e2 * q;
    E3t[l] = e2 * q * c2;
  }

  const UpwindF ub = upwind_side(g, p, i, j, 2);
  const UpwindF ut = upwind_side(g, p, i, j, 3);
  const size_t nv = (size_t)nv1 * nv2;
  const float* Gc = Gs + (size_t)cell * nv + k;
  const float* Gb = Gs + (size_t)ub.cell * nv + k;
  const float* Gt = Gs + (size_t)ut.cell * nv + k;
  const float v1 = fmaf(k + 0.5f, dv1, v1min);
  const float c1 = v1 - u1;
  const float c1q = c1 * c1;
  __syncthreads();

  float E0 = 0.f, E1 = 0.f, E2 = 0.f;
  if (active) {
    for (int l = r; l < nv2; l += R) {
      const float gv = Gc[l * nv1];
      const bool top = v2t[l] < 0.f;
      const UpwindF& u = top ? ut : ub;
      const float* Gu = top ? Gt : Gb;
      const int lu = u.mirror ? nv2 - 1 - l : l;
      const float gu = u.zero ? 0.f : Gu[lu * nv1];
      const float d = gu - gv;
      E0 = fmaf(s0t[l], d, E0);
      E1 = fmaf(s1t[l], d, E1);
      E2 = fmaf(s2t[l], d, E2);
    }
  }
  const float S[4] = {E0, c1 * E0, E1, fmaf(c1q, E0, E2)};
  warp_sum4f(S, part);
  __syncthreads();
  if (t == 0) {
    float hi[4], lo[4];
    sum_parts(part, hi, lo);
    const float S0 = hi[0] + lo[0], S1 = hi[1] + lo[1], S2 = hi[2] + lo[2], S3 = hi[3] + lo[3];
    bco[0] = fmaf(-S3, inv2T, 2.f * S0);
    bco[1] = S1 * iT;
    bco[2] = S2 * iT;
    bco[3] = fmaf(0.25f * S3, iT * iT, -S0 * inv2T);
  }
  __syncthreads();
  const float b0 = bco[0], b1 = bco[1], b2 = bco[2], gm = bco[3];
  const float w01 = pf[F_W01 * nc + cell], w02 = pf[F_W02 * nc + cell];
  const float w03 = pf[F_W03 * nc + cell], w10 = pf[F_W10 * nc + cell];
  const float w11 = pf[F_W11 * nc + cell], w12 = pf[F_W12 * nc + cell];
  const float w20 = pf[F_W20 * nc + cell], w21 = pf[F_W21 * nc + cell];
  const float w30 = pf[F_W30 * nc + cell];
  const float C0 = om1kap * fmaf(gm, c1q, fmaf(b1, c1, b0)) - c1 * fmaf(c1, fmaf(c1, w03, w02), w01) - ome;
  const float C1 = fmaf(om1kap, b2, -fmaf(c1, fmaf(c1, w12, w11), w10));
  const float C2 = fmaf(om1kap, gm, -fmaf(c1, w21, w20));
  const float C3 = -w30;
  const float e1 = expf(-c1q * inv2T);
  const float A0 = e1 * C0, A1 = e1 * C1, A2 = e1 * C2, A3 = e1 * C3;
  const float gam1 = gam0 * expf(-Ti11h * c1q);
  const float c2r = fmaf(r + 0.5f, dv2, v2min) - u2;
  float x = expf(-Ti12 * c1 * c2r);
  const float rat = expf(-Ti12 * c1 * (R * dv2));

  float H0 = 0.f, H1 = 0.f, H2 = 0.f, H3 = 0.f;
  if (active) {
    float* Go = Gout + (size_t)cell * nv + k;
    for (int l = r; l < nv2; l += R) {
      const float gv = Gc[l * nv1];
      const bool top = v2t[l] < 0.f;
      const UpwindF& u = top ? ut : ub;
      const float* Gu = top ? Gt : Gb;
      const int lu = u.mirror ? nv2 - 1 - l : l;
      const float gu = u.zero ? 0.f : Gu[lu * nv1];
      const float d = gu - gv;
      float o = fmaf(wlt[l], d, om1 * gv);
      o = fmaf(A0, e2t[l], o);
      o = fmaf(A1, E1t[l], o);
      o = fmaf(A2, E2t[l], o);
      o = fmaf(A3, E3t[l], o);
      o = fmaf(gam1, g2t[l] * x, o);
      x *= rat;
      Go[l * nv1] = o;
      H0 += o;
      H1 = fmaf(c2t[l], o, H1);
      H2 = fmaf(c2q[l], o, H2);
      H3 = fmaf(c2c[l], o, H3);
    }
  }
  const float Hs[4] = {c1q * c1 * H0, c1q * H1, c1 * H2, H3};
  __syncthreads();  // the partial-sum slots are reused
  warp_sum4f(Hs, part);
  __syncthreads();
  if (t == 0) {
    float hi[4], lo[4];
    sum_parts(part, hi, lo);
    for (int m = 0; m < 4; ++m) {
      Hf[(2 * m) * nc + cell] = hi[m];
      Hf[(2 * m + 1) * nc + cell] = lo[m];
    }
  }
}

}  // namespace

KGridF grid_f32(const KGrid& g) {
  return KGridF{(float)g.v1min, (float)g.v2min, (float)g.dv1, (float)g.dv2, (float)g.idx,
                (float)g.idy};
}

void launch_micro_x_f32(const float* Gin, float* Gout, const float* primf, const KGrid& g,
                        const KParams& p, double dt, const MicroShape& ms, cudaStream_t s) {
  const size_t smem = sizeof(float) * (kHeadF + 4 * (size_t)g.nv2);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_micro_x_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_micro_x_f32<<<g.nx * g.ny, ms.threads, smem, s>>>(Gin, Gout, primf, g, grid_f32(g), p,
                                                      (float)(dt * g.idx), ms.R);
}

void launch_micro_y_f32(const float* Gs, float* Gout, float* Hf, const float* primf,
                        const KGrid& g, const KParams& p, double dt, const MicroShape& ms,
                        cudaStream_t s) {
  const size_t smem = sizeof(float) * (kHeadF + kYTablesF * (size_t)g.nv2);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_micro_y_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_micro_y_f32<<<g.nx * g.ny, ms.threads, smem, s>>>(Gs, Gout, Hf, primf, g, grid_f32(g), p,
                                                      (float)(dt * g.idy), ms.R);
}

}  // namespace mmk
