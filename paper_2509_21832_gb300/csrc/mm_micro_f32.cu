// FP32-g phase-space kernels of the micro step (Section 5.3 of Rossmanith & Sar, arXiv
// 2509.21832): the same split upwind transport with projection, relaxation toward Ghat and heat
// flux as mm_micro.cu, with g stored and transported in FP32.
//
// Precision split: no FP64 instruction runs in the streaming kernels (the FP64 pipe of GB300
// runs at 1/64 of FP32 and a warp instruction costs its full issue time even with one active
// lane, so an FP64 epilogue per cell would bound the kernel); per-cell coefficients come from
// the fields kernel (the ES tensor inverse, 1/T and the projector scale in FP64 rounded once,
// the relaxation weights as FP32 products of those); velocity sums are FP32 (per-lane partial
// sums over its rows, then a pairwise warp butterfly); the heat flux leaves as (hi, lo) FP32
// pairs (lo = 0 here) that the per-cell unpack kernel turns into FP64.
//
// Three kernels stream the same arithmetic, chosen on the host (pick_fused):
//  - k_micro_staged_f32 (24^2 and 16^2 meshes symmetric in v2): flat lane mapping, the four
//    warps of a CTA march four adjacent columns in step, g blocks staged by bulk copies;
//  - k_micro_flat_f32 (32^2, symmetric in v2): flat lane mapping, one warp per column, g through
//    the read-only path;
//  - k_micro_fused_f32 (any mesh with nv1 <= 32): lane = v1 index, one warp per column.
// The flat-mapped sweeps update two elements per instruction (packed f32x2 arithmetic of
// sm_100 and later).  k_wall_f32 then finishes the cells next to a diffuse wall from the G* the
// streaming kernels export.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "mm_body_macro.cuh"
#include "mm_internal.cuh"

namespace mmk {

namespace {

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


// ------------------------------------------------------------------------------------------
// Fused streaming micro step (FP32 g), one warp per cell column.
//
// A warp owns the column of cells i and a segment of rows [j0, j1) and marches upward: the x
// sweep of row j+1 goes into a three-row ring of split-step values G* in the warp's slice of
// shared memory, then the y sweep, relaxation and heat flux of row j read rows j-1, j, j+1 from
// the ring.  G* never goes to HBM: each step reads g once (the x neighbours' rows come through
// L2, shared by the adjacent columns that march in step) and writes it once.  Lane t owns the v1
// index k = t mod nv1 and the v2 rows l = t div nv1 + m R (R = 32 div nv1); every velocity sum
// is a warp butterfly whose totals all lanes receive, so the warp never waits for other warps.
// Cells next to a diffuse wall (and their y neighbours) also export G* to global memory for the
// wall kernel, which finishes them afterwards.
// ------------------------------------------------------------------------------------------
struct FusedF32 {
  const float* Gin;
  float* Gout;
  float* Gexp;  // G* export for the diffuse-wall kernel (NULL without diffuse walls)
  float* Hf;
  const float* pf;
  KGrid g;
  KGridF gf;
  KParams p;
  float dtidx, dtidy;
  int R;         // rows per pass: 32 / nv1
  int seg_rows;  // rows per segment
  int nseg;      // row segments
  int* err;      // device error word (ERR_WAIT_TIMEOUT from a bounded wait)
};

constexpr int kFusedWarps = 4;  // warps (columns) per CTA

__device__ __forceinline__ bool exports_gstar(const KGrid& g, const KParams& p, int i, int j) {
  return (p.bc[2] == MM_BC_DIFFUSE && j <= 1) || (p.bc[3] == MM_BC_DIFFUSE && j >= g.ny - 2) ||
         (p.bc[0] == MM_BC_DIFFUSE && i == 0) || (p.bc[1] == MM_BC_DIFFUSE && i == g.nx - 1);
}

// Sum four floats over the warp; every lane receives the four totals.
__device__ __forceinline__ void warp_allsum4(float v[4]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
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
  v[0] = __shfl_sync(full, kk, 0);
  v[1] = __shfl_sync(full, kk, 8);
  v[2] = __shfl_sync(full, kk, 16);
  v[3] = __shfl_sync(full, kk, 24);
}

// Per-cell FP32 coefficients of one cell, loaded by one instruction (lane f reads field f) and
// handed out by warp shuffles.
__device__ __forceinline__ float load_fields(const float* __restrict__ pf, int nc, int cell) {
  const int lane = threadIdx.x & 31;
  return lane < NPRIMF ? __ldg(pf + (size_t)lane * nc + cell) : 0.f;
}
__device__ __forceinline__ float field(float fv, int f) { return __shfl_sync(0xffffffffu, fv, f); }

// Velocity shape: compile-time for the common meshes (NV1 > 0: nv1 = NV1, nv2 = NV2, every
// active lane owns exactly NR = NV2 / R rows), runtime otherwise (NV1 = 0).
template <int NV1, int NV2>
struct VShape {
  static constexpr bool fixed = NV1 > 0;
  static constexpr int RC = NV1 > 0 ? 32 / NV1 : 1;
  static constexpr int NRC = NV1 > 0 ? NV2 / RC : 0;
  int nv1, nv2, R, nr;
  __device__ __forceinline__ VShape(const KGrid& g, int Rrt) {
    nv1 = fixed ? NV1 : g.nv1;
    nv2 = fixed ? NV2 : g.nv2;
    R = fixed ? RC : Rrt;
    nr = fixed ? NRC : (g.nv2 + Rrt - 1) / Rrt;
  }
};

// x sweep of cell (i, j) into dst (the warp's shared-memory ring slot).
template <int NV1, int NV2>
__device__ __forceinline__ void wx_sweep(const FusedF32& a, int i, int j, float* dst, float* xt) {
  const KGrid& g = a.g;
  const VShape<NV1, NV2> vs(g, a.R);
  const int nv1 = vs.nv1, nv2 = vs.nv2, R = vs.R, nc = g.nx * g.ny;
  const int cell = j * g.nx + i;
  // row tables as pairs, one shared load each: X1 = (c2, c2^2), X2 = (e2, projection term)
  float2* X1 = reinterpret_cast<float2*>(xt);
  float2* X2 = X1 + nv2;
  const int lane = threadIdx.x & 31, k = lane % nv1, r = lane / nv1;
  const bool active = r < R;
  const float fv = load_fields(a.pf, nc, cell);
  const float u1 = field(fv, F_U1), u2 = field(fv, F_U2);
  const float inv2T = field(fv, F_INV2T), iT = field(fv, F_IT), kap = field(fv, F_KAP);
  for (int l = lane; l < nv2; l += 32) {
    const float c2 = fmaf(l + 0.5f, a.gf.dv2, a.gf.v2min) - u2;
    const float q = c2 * c2;
    X1[l] = make_float2(c2, q);
    X2[l] = make_float2(expf(-q * inv2T), 0.f);
  }
  const float v1 = fmaf(k + 0.5f, a.gf.dv1, a.gf.v1min);
  const float c1 = v1 - u1;
  const float av = fabsf(v1);
  const float sig = -av * a.gf.idx;
  const float lam = av * a.dtidx;
  const UpwindF up = upwind_side(g, a.p, i, j, v1 > 0.f ? 0 : 1);
  const int ku = up.mirror ? nv1 - 1 - k : k;
  const size_t nv = (size_t)nv1 * nv2;
  const float* Gc = a.Gin + (size_t)cell * nv + k;
  const float* Gu = a.Gin + (size_t)up.cell * nv + ku;
  __syncwarp();
  // pass 1: upwind differences and their moments; dst keeps the upwind update G + lam d
  float D0 = 0.f, D1 = 0.f, D2 = 0.f;
  if (active) {
    if constexpr (VShape<NV1, NV2>::fixed) {
      constexpr int NR = VShape<NV1, NV2>::NRC;
      constexpr int RR = VShape<NV1, NV2>::RC;
      float gv[NR], gu[NR];
#pragma unroll
      for (int m = 0; m < NR; ++m) {
        const int l = r + m * RR;
        gv[m] = __ldg(Gc + l * NV1);
        gu[m] = up.zero ? 0.f : __ldg(Gu + l * NV1);
      }
#pragma unroll
      for (int m = 0; m < NR; ++m) {
        const int l = r + m * RR;
        const float d = gu[m] - gv[m];
        const float2 cq = X1[l];
        dst[l * NV1 + k] = fmaf(lam, d, gv[m]);
        D0 += d;
        D1 = fmaf(cq.x, d, D1);
        D2 = fmaf(cq.y, d, D2);
      }
    } else {
      constexpr int kChunk = 16;
      for (int l0 = r; l0 < nv2; l0 += kChunk * R) {
        float gv[kChunk], gu[kChunk];
#pragma unroll
        for (int m = 0; m < kChunk; ++m) {
          const int l = l0 + m * R;
          const bool in = l < nv2;
          gv[m] = in ? __ldg(Gc + l * nv1) : 0.f;
          gu[m] = (in && !up.zero) ? __ldg(Gu + l * nv1) : 0.f;
        }
#pragma unroll
        for (int m = 0; m < kChunk; ++m) {
          const int l = l0 + m * R;
          if (l < nv2) {
            const float d = gu[m] - gv[m];
            const float2 cq = X1[l];
            dst[l * nv1 + k] = fmaf(lam, d, gv[m]);
            D0 += d;
            D1 = fmaf(cq.x, d, D1);
            D2 = fmaf(cq.y, d, D2);
          }
        }
      }
    }
  }
  const float sD0 = sig * D0;
  float S[4] = {sD0, c1 * sD0, sig * D1, fmaf(c1 * c1, sD0, sig * D2)};
  warp_allsum4(S);
  const float b0 = fmaf(-S[3], inv2T, 2.f * S[0]);
  const float b1 = S[1] * iT, b2 = S[2] * iT;
  const float gm = fmaf(0.25f * S[3], iT * iT, -S[0] * inv2T);
  for (int l = lane; l < nv2; l += 32) {
    const float2 cq = X1[l];
    X2[l].y = X2[l].x * fmaf(b2, cq.x, gm * cq.y);
  }
  const float e1 = expf(-c1 * c1 * inv2T);
  const float bk = kap * e1;
  const float ak = bk * fmaf(gm * c1, c1, fmaf(b1, c1, b0));
  __syncwarp();
  // pass 2: G* = G - dt Z + dt Zhat, from shared memory only
  const bool exp_ = a.Gexp != nullptr && exports_gstar(g, a.p, i, j);
  if (active) {
    float* Ge = a.Gexp + (size_t)cell * nv + k;
#pragma unroll
    for (int m = 0; m < vs.nr; ++m) {
      const int l = r + m * R;
      if (!VShape<NV1, NV2>::fixed && l >= nv2) break;
      const float2 eq = X2[l];
      float o = dst[l * nv1 + k];
      o = fmaf(ak, eq.x, o);
      o = fmaf(bk, eq.y, o);
      dst[l * nv1 + k] = o;
      if (exp_) Ge[l * nv1] = o;
    }
  }
  __syncwarp();
}

// y sweep + relaxation + heat flux of cell (i, j) from the G* rows in the warp's ring.
template <int NV1, int NV2>
__device__ __forceinline__ void wy_sweep(const FusedF32& a, int i, int j, const float* rc,
                                         const float* srcb, bool mb, bool zb, const float* srct,
                                         bool mt, bool zt, float* tb) {
  const KGrid& g = a.g;
  const VShape<NV1, NV2> vs(g, a.R);
  const int nv1 = vs.nv1, nv2 = vs.nv2, R = vs.R, nc = g.nx * g.ny;
  const int cell = j * g.nx + i;
  // row tables grouped for 16-byte shared loads: TS = (s0, s1, s2) for the moments of Z*;
  // TA = (e2, e2 c2, e2 c2^2, e2 c2^3), TB = (wl, om1 - wl, g2, c2), TC = (c2^2, c2^3) for the
  // update and the heat flux
  float4* TS = reinterpret_cast<float4*>(tb);
  float4* TA = TS + nv2;
  float4* TB = TA + nv2;
  float2* TC = reinterpret_cast<float2*>(TB + nv2);
  const int lane = threadIdx.x & 31, k = lane % nv1, r = lane / nv1;
  const bool active = r < R;
  const float fv = load_fields(a.pf, nc, cell);
  const float u1 = field(fv, F_U1), u2 = field(fv, F_U2);
  const float inv2T = field(fv, F_INV2T), iT = field(fv, F_IT);
  const float Ti11h = field(fv, F_TI11H), Ti12 = field(fv, F_TI12), Ti22h = field(fv, F_TI22H);
  const float om1 = field(fv, F_OM1), om1kap = field(fv, F_OM1KAP);
  const float gam0 = field(fv, F_GAM0), ome = field(fv, F_OME);
  const float w01 = field(fv, F_W01), w02 = field(fv, F_W02), w03 = field(fv, F_W03);
  const float w10 = field(fv, F_W10), w11 = field(fv, F_W11), w12 = field(fv, F_W12);
  const float w20 = field(fv, F_W20), w21 = field(fv, F_W21), w30 = field(fv, F_W30);
  // tables; nneg = rows with v2 < 0 (v2 increases with l): the upwind side of a row is an
  // integer comparison
  int nneg = 0;
  for (int l0 = 0; l0 < nv2; l0 += 32) {
    const int l = l0 + lane;
    bool neg = false;
    if (l < nv2) {
      const float v2 = fmaf(l + 0.5f, a.gf.dv2, a.gf.v2min);
      const float c2 = v2 - u2;
      const float q = c2 * c2;
      const float e2 = expf(-q * inv2T);
      const float av = fabsf(v2);
      const float sg = -av * a.gf.idy;
      const float wl = om1 * (av * a.dtidy);
      TS[l] = make_float4(sg, sg * c2, sg * q, 0.f);
      TA[l] = make_float4(e2, e2 * c2, e2 * q, e2 * q * c2);
      TB[l] = make_float4(wl, om1 - wl, expf(-Ti22h * q), c2);
      TC[l] = make_float2(q, q * c2);
      neg = v2 < 0.f;
    }
    nneg += __popc(__ballot_sync(0xffffffffu, neg));
  }
  const float v1 = fmaf(k + 0.5f, a.gf.dv1, a.gf.v1min);
  const float c1 = v1 - u1;
  const float c1q = c1 * c1;
  __syncwarp();
  float E0 = 0.f, E1 = 0.f, E2 = 0.f;
  if (active) {
#pragma unroll
    for (int m = 0; m < vs.nr; ++m) {
      const int l = r + m * R;
      if (!VShape<NV1, NV2>::fixed && l >= nv2) break;
      const float gv = rc[l * nv1 + k];
      const bool top = l < nneg;
      const float* src = top ? srct : srcb;
      const int lu = (top ? mt : mb) ? nv2 - 1 - l : l;
      const float gu = (top ? zt : zb) ? 0.f : src[lu * nv1 + k];
      const float d = gu - gv;
      const float4 ts = TS[l];
      E0 = fmaf(ts.x, d, E0);
      E1 = fmaf(ts.y, d, E1);
      E2 = fmaf(ts.z, d, E2);
    }
  }
  float S[4] = {E0, c1 * E0, E1, fmaf(c1q, E0, E2)};
  warp_allsum4(S);
  const float b0 = fmaf(-S[3], inv2T, 2.f * S[0]);
  const float b1 = S[1] * iT, b2 = S[2] * iT;
  const float gm = fmaf(0.25f * S[3], iT * iT, -S[0] * inv2T);
  const float C0 = om1kap * fmaf(gm, c1q, fmaf(b1, c1, b0)) - c1 * fmaf(c1, fmaf(c1, w03, w02), w01) - ome;
  const float C1 = fmaf(om1kap, b2, -fmaf(c1, fmaf(c1, w12, w11), w10));
  const float C2 = fmaf(om1kap, gm, -fmaf(c1, w21, w20));
  const float C3 = -w30;
  const float e1 = expf(-c1q * inv2T);
  const float A0 = e1 * C0, A1 = e1 * C1, A2 = e1 * C2, A3 = e1 * C3;
  const float c2r = fmaf(r + 0.5f, a.gf.dv2, a.gf.v2min) - u2;
  // gam0 exp(-Ti11 c1^2 / 2) times the cross factor exp(-Ti12 c1 c2) of row l
  float x = gam0 * expf(-Ti11h * c1q - Ti12 * c1 * c2r);
  const float rat = expf(-Ti12 * c1 * (R * a.gf.dv2));
  float H0 = 0.f, H1 = 0.f, H2 = 0.f, H3 = 0.f;
  if (active) {
    const size_t nv = (size_t)nv1 * nv2;
    float* Go = a.Gout + (size_t)cell * nv + k;
#pragma unroll
    for (int m = 0; m < vs.nr; ++m) {
      const int l = r + m * R;
      if (!VShape<NV1, NV2>::fixed && l >= nv2) break;
      const float gv = rc[l * nv1 + k];
      const bool top = l < nneg;
      const float* src = top ? srct : srcb;
      const int lu = (top ? mt : mb) ? nv2 - 1 - l : l;
      const float gu = (top ? zt : zb) ? 0.f : src[lu * nv1 + k];
      const float4 ta = TA[l];
      const float4 tb4 = TB[l];
      const float2 tc = TC[l];
      float o = fmaf(tb4.x, gu, tb4.y * gv);
      o = fmaf(A0, ta.x, o);
      o = fmaf(A1, ta.y, o);
      o = fmaf(A2, ta.z, o);
      o = fmaf(A3, ta.w, o);
      o = fmaf(tb4.z, x, o);
      x *= rat;
      Go[l * nv1] = o;
      H0 += o;
      H1 = fmaf(tb4.w, o, H1);
      H2 = fmaf(tc.x, o, H2);
      H3 = fmaf(tc.y, o, H3);
    }
  }
  float Hs[4] = {c1q * c1 * H0, c1q * H1, c1 * H2, H3};
  warp_allsum4(Hs);
  if (lane < 8) a.Hf[lane * nc + cell] = (lane & 1) ? 0.f : Hs[lane >> 1];
  __syncwarp();
}

template <int NV1, int NV2>
__global__ void __launch_bounds__(32 * kFusedWarps, 4) k_micro_fused_f32(FusedF32 a) {
  extern __shared__ float smf[];
  const KGrid& g = a.g;
  const int nv = g.nv1 * g.nv2;
  const int w = threadIdx.x >> 5;
  const int ring_f = (3 * nv + 3) / 4 * 4;
  const int per_warp = ring_f + 18 * g.nv2 + (g.nv2 & 1) * 2;
  float* ring = smf + (size_t)w * per_warp;
  float* xt = ring + ring_f;
  float* yt = xt + 4 * g.nv2;
  const int gw = blockIdx.x * kFusedWarps + w;
  if (gw >= g.nx * a.nseg) return;  // whole warp leaves; no CTA-wide barrier is used below
  const int i = gw % g.nx;
  const int seg = gw / g.nx;
  const int j0 = seg * a.seg_rows;
  const int j1 = min(g.ny, j0 + a.seg_rows);
  if (j0 >= j1) return;
  const bool pery = a.p.bc[2] == MM_BC_PERIODIC;
  // position p = j - j0 + 1 of a row in the march; its G* lives in ring slot p % 3
  auto slot = [&](int pos) { return ring + (size_t)(pos % 3) * nv; };
  if (j0 > 0 || pery) wx_sweep<NV1, NV2>(a, i, j0 > 0 ? j0 - 1 : g.ny - 1, slot(0), xt);
  wx_sweep<NV1, NV2>(a, i, j0, slot(1), xt);
  for (int j = j0; j < j1; ++j) {
    const int pos = j - j0 + 1;
    if (j + 1 < g.ny || pery) wx_sweep<NV1, NV2>(a, i, j + 1 < g.ny ? j + 1 : 0, slot(pos + 1), xt);
    if (diffuse_wall_cell(g, a.p, i, j)) continue;  // finished by the wall kernel
    const float* rc = slot(pos);
    const bool hasb = j > 0 || pery, hast = j < g.ny - 1 || pery;
    const float* srcb = hasb ? slot(pos + 2) : rc;  // slot(pos - 1)
    const float* srct = hast ? slot(pos + 1) : rc;
    const bool mb = !hasb && a.p.bc[2] == MM_BC_SPECULAR;
    const bool zb = !hasb && a.p.bc[2] == MM_BC_DIFFUSE;
    const bool mt = !hast && a.p.bc[3] == MM_BC_SPECULAR;
    const bool zt = !hast && a.p.bc[3] == MM_BC_DIFFUSE;
    wy_sweep<NV1, NV2>(a, i, j, rc, srcb, mb, zb, srct, mt, zt, yt);
  }
}

// ------------------------------------------------------------------------------------------
// Flat-mapped variant for the compile-time meshes (nv a multiple of 32, v2 mesh symmetric about
// zero).  The same march, ring and arithmetic, but lane L owns the flat velocity indices
// q = L + 32 m, m < nv / 32, so every lane is busy whatever nv1 is: with nv1 = 24 a lane owns
// P = 3 columns k_s = (L + 32 s) mod nv1 and, in each, every ST = 4th row from
// l_s = (L + 32 s) div nv1.  Each phase-space access is a contiguous 128-byte warp row; the rows
// with v2 < 0 (upwind from above) are exactly the first half, so the upwind source of every
// element is fixed at compile time; a specular y wall is served by a mirrored copy of the cell's
// G* in the ring slot the missing neighbour would use; a diffuse x wall reads a zero row.  The
// upwind differences stay in registers between the two passes of each sweep.
// ------------------------------------------------------------------------------------------
__device__ __align__(16) float kZeroRowF[1024];

// Bulk prefetch of bytes (a multiple of 16) at a 16-byte aligned global address into L2.
__device__ __forceinline__ void l2_prefetch_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}  // zero upwind values behind a diffuse wall (nv <= 1024)

constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

// The flat-mapped sweeps read a cell's fields from shared memory as float4 groups in this order.
static_assert(F_U1 == 0 && F_U2 == 1 && F_INV2T == 2 && F_IT == 3 && F_KAP == 4 && F_OM1 == 5 &&
                  F_OM1KAP == 6 && F_GAM0 == 7 && F_OME == 8 && F_TI11H == 9 && F_TI12 == 10 &&
                  F_TI22H == 11 && F_W01 == 12 && F_W02 == 13 && F_W03 == 14 && F_W10 == 15 &&
                  F_W11 == 16 && F_W12 == 17 && F_W20 == 18 && F_W21 == 19 && F_W30 == 20 &&
                  NPRIMF == 21,
              "field order");
constexpr int kFieldSlot = 24;  // floats per cell's fields in shared memory (16-byte multiple)

template <int NV1, int NV2>
struct FlatShape {
  static constexpr int NV = NV1 * NV2;
  static constexpr int M = NV / 32;                 // elements per lane
  static constexpr int P = NV1 / cgcd(NV1, 32);     // v1 columns per lane
  static constexpr int ST = 32 / cgcd(NV1, 32);     // row stride within a column
  static constexpr int TOP = NV2 / (2 * ST);        // visits t < TOP are rows with v2 < 0
  static constexpr int PER_WARP = 3 * NV + 14 * NV2 + kFieldSlot;  // ring, tables, fields
  static_assert(NV % 32 == 0 && M % P == 0 && (M / P) * ST == NV2, "flat shape");
  static_assert((NV2 / 2) % ST == 0 && NV <= 1024 && NV2 % 2 == 0, "flat shape");
};

// Packed FP32 pairs: a lane updates the elements of visits t = 2u and 2u + 1 of one v1 column
// (rows a = l0 + 2 ST u and b = a + ST) with one f32x2 instruction.  Their row factors share a
// table slot, l0 + ST u, so that one shared load brings both.
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 sub2(float2 x, float2 y) {
  return __fadd2_rn(x, make_float2(-y.x, -y.y));
}

template <int NV1, int NV2>
__device__ __forceinline__ int pair_slot(int l, int& half) {
  constexpr int ST = FlatShape<NV1, NV2>::ST;
  const int r = l % (2 * ST);
  half = r >= ST ? 1 : 0;
  return r - half * ST + ST * (l / (2 * ST));
}

// x sweep of cell (i, j) into the ring slot dst (flat mapping).  Gc is the cell's g block, Gl and
// Gr the blocks upwind on the left and right (the cell's own block for extrapolation and specular
// sides, mirrored in v1 when mirl / mirr, a zero row behind a diffuse side): global memory read
// through the read-only path, or the shared-memory stage (STAGED).
template <int NV1, int NV2, bool STAGED>
__device__ __forceinline__ void fx_sweep(const FusedF32& a, int i, int j, float* dst, float* xt,
                                         const float* Gcb, const float* Gl, const float* Gr,
                                         bool mirl, bool mirr, const float* fs) {
  using S = FlatShape<NV1, NV2>;
  constexpr int P = S::P, NU = S::M / S::P / 2, ST = S::ST;
  const KGrid& g = a.g;
  const int cell = j * g.nx + i;
  const int lane = threadIdx.x & 31;
  // per row pair: {c2_a, c2_b, c2_a^2, c2_b^2}, {e2_a, e2_b, projection term a, b}
  float4* XP = reinterpret_cast<float4*>(xt);
  const float4 f0 = *reinterpret_cast<const float4*>(fs);  // (u1, u2, 1/2T, 1/T)
  const float u1 = f0.x, u2 = f0.y, inv2T = f0.z, iT = f0.w, kap = fs[F_KAP];
  for (int l = lane; l < NV2; l += 32) {
    int h;
    const int p = pair_slot<NV1, NV2>(l, h);
    const float c2 = fmaf(l + 0.5f, a.gf.dv2, a.gf.v2min) - u2;
    const float q = c2 * c2;
    float* X = xt + 8 * p;
    X[h] = c2;
    X[2 + h] = q;
    X[4 + h] = expf(-q * inv2T);
  }
  float c1[P], sig[P], lam[P];
  const float* Gu[P];
  int l0[P], kc[P];
#pragma unroll
  for (int s = 0; s < P; ++s) {
    const int q0 = lane + 32 * s, k = q0 % NV1;
    l0[s] = q0 / NV1;
    kc[s] = k;
    const float v1 = fmaf(k + 0.5f, a.gf.dv1, a.gf.v1min);
    c1[s] = v1 - u1;
    const float av = fabsf(v1);
    sig[s] = -av * a.gf.idx;
    lam[s] = av * a.dtidx;
    const bool left = v1 > 0.f;
    Gu[s] = (left ? Gl : Gr) + q0 + ((left ? mirl : mirr) ? NV1 - 1 - 2 * k : 0);
  }
  const float* Gc = Gcb + lane;
  auto ld = [](const float* q) { return STAGED ? *q : __ldg(q); };
  __syncwarp();
  // pass 1: upwind differences, their moments and the upwind update (kept in registers)
  float2 ue[P][NU];
  float2 D0[P], D1[P], D2[P];
#pragma unroll
  for (int s = 0; s < P; ++s) D0[s] = D1[s] = D2[s] = f2(0.f);
  {
    float2 gv[P][NU], gu[P][NU];
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
      for (int s = 0; s < P; ++s) {
        const int m = s + P * 2 * u;
        gv[s][u] = f2(ld(Gc + 32 * m), ld(Gc + 32 * (m + P)));
        gu[s][u] = f2(ld(Gu[s] + 32 * P * (2 * u)), ld(Gu[s] + 32 * P * (2 * u + 1)));
      }
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
      for (int s = 0; s < P; ++s) {
        const float2 d = sub2(gu[s][u], gv[s][u]);
        const float4 X = XP[2 * (l0[s] + ST * u)];
        ue[s][u] = __ffma2_rn(f2(lam[s]), d, gv[s][u]);
        D0[s] = __fadd2_rn(D0[s], d);
        D1[s] = __ffma2_rn(f2(X.x, X.y), d, D1[s]);
        D2[s] = __ffma2_rn(f2(X.z, X.w), d, D2[s]);
      }
  }
  float Sx[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int s = 0; s < P; ++s) {
    const float sD0 = sig[s] * (D0[s].x + D0[s].y);
    Sx[0] += sD0;
    Sx[1] = fmaf(c1[s], sD0, Sx[1]);
    Sx[2] = fmaf(sig[s], D1[s].x + D1[s].y, Sx[2]);
    Sx[3] += fmaf(c1[s] * c1[s], sD0, sig[s] * (D2[s].x + D2[s].y));
  }
  warp_allsum4(Sx);
  const float b0 = fmaf(-Sx[3], inv2T, 2.f * Sx[0]);
  const float b1 = Sx[1] * iT, b2 = Sx[2] * iT;
  const float gm = fmaf(0.25f * Sx[3], iT * iT, -Sx[0] * inv2T);
  for (int p = lane; p < NV2 / 2; p += 32) {
    const float4 X = XP[2 * p];
    float4 E = XP[2 * p + 1];
    E.z = E.x * fmaf(b2, X.x, gm * X.z);
    E.w = E.y * fmaf(b2, X.y, gm * X.w);
    XP[2 * p + 1] = E;
  }
  // kap e1 of each column: with several columns per lane, lane k evaluates column k's and the
  // owners fetch it by shuffle
  float ak[P], bk[P];
  if constexpr (P == 1) {
    bk[0] = kap * expf(-c1[0] * c1[0] * inv2T);
  } else {
    const float ck = fmaf((lane < NV1 ? lane : 0) + 0.5f, a.gf.dv1, a.gf.v1min) - u1;
    const float bown = kap * expf(-ck * ck * inv2T);
#pragma unroll
    for (int s = 0; s < P; ++s) bk[s] = __shfl_sync(0xffffffffu, bown, kc[s]);
  }
#pragma unroll
  for (int s = 0; s < P; ++s) ak[s] = bk[s] * fmaf(gm * c1[s], c1[s], fmaf(b1, c1[s], b0));
  __syncwarp();
  // pass 2: G* = G - dt Z + dt Zhat
#pragma unroll
  for (int u = 0; u < NU; ++u)
#pragma unroll
    for (int s = 0; s < P; ++s) {
      const float4 E = XP[2 * (l0[s] + ST * u) + 1];
      float2 o = __ffma2_rn(f2(ak[s]), f2(E.x, E.y), ue[s][u]);
      o = __ffma2_rn(f2(bk[s]), f2(E.z, E.w), o);
      const int m = s + P * 2 * u;
      dst[lane + 32 * m] = o.x;
      dst[lane + 32 * (m + P)] = o.y;
    }
  if (a.Gexp != nullptr && exports_gstar(g, a.p, i, j)) {
    float* Ge = a.Gexp + (size_t)cell * S::NV + lane;
#pragma unroll
    for (int m = 0; m < S::M; ++m) Ge[32 * m] = dst[lane + 32 * m];
  }
  __syncwarp();
}

// y sweep + relaxation + heat flux of cell (i, j) from the ring rows below (rb), at (rc) and
// above (rt) the cell (flat mapping).
template <int NV1, int NV2>
__device__ __forceinline__ void fy_sweep(const FusedF32& a, int i, int j, const float* rb,
                                         const float* rc, const float* rt, float* tb,
                                         const float* fs) {
  using S = FlatShape<NV1, NV2>;
  constexpr int P = S::P, NU = S::M / S::P / 2, ST = S::ST;
  const KGrid& g = a.g;
  const int nc = g.nx * g.ny, cell = j * g.nx + i;
  const int lane = threadIdx.x & 31;
  // per row pair (five float4): {s0_a, s0_b, s0 c2_a, s0 c2_b}, {s0 c2^2_a, s0 c2^2_b, -, -}
  // for the moments of Z*; {wl_a, wl_b, e2_a, e2_b}, {c2_a, c2_b, g2_a, g2_b},
  // {c2^2_a, c2^2_b, c2^3_a, c2^3_b} for the update and the heat flux
  const float4* Y = reinterpret_cast<const float4*>(tb);
  const float4* F4 = reinterpret_cast<const float4*>(fs);
  const float4 fa = F4[0], fb = F4[1], fc = F4[2], fd = F4[3], fe = F4[4];
  const float u1 = fa.x, u2 = fa.y, inv2T = fa.z, iT = fa.w;
  const float om1 = fb.y, om1kap = fb.z, gam0 = fb.w;
  const float ome = fc.x, Ti11h = fc.y, Ti12 = fc.z, Ti22h = fc.w;
  const float w01 = fd.x, w02 = fd.y, w03 = fd.z, w10 = fd.w;
  const float w11 = fe.x, w12 = fe.y, w20 = fe.z, w21 = fe.w, w30 = fs[F_W30];
  for (int l = lane; l < NV2; l += 32) {
    int h;
    const int p = pair_slot<NV1, NV2>(l, h);
    const float v2 = fmaf(l + 0.5f, a.gf.dv2, a.gf.v2min);
    const float c2 = v2 - u2;
    const float q = c2 * c2;
    const float av = fabsf(v2);
    const float sg = -av * a.gf.idy;
    float* T = tb + 20 * p;
    T[h] = sg;
    T[2 + h] = sg * c2;
    T[4 + h] = sg * q;
    T[8 + h] = om1 * (av * a.dtidy);
    T[10 + h] = expf(-q * inv2T);
    T[12 + h] = c2;
    T[14 + h] = expf(-Ti22h * q);
    T[16 + h] = q;
    T[18 + h] = q * c2;
  }
  float c1[P], c1q[P];
  int l0[P], kc[P];
#pragma unroll
  for (int s = 0; s < P; ++s) {
    const int q0 = lane + 32 * s, k = q0 % NV1;
    l0[s] = q0 / NV1;
    kc[s] = k;
    c1[s] = fmaf(k + 0.5f, a.gf.dv1, a.gf.v1min) - u1;
    c1q[s] = c1[s] * c1[s];
  }
  __syncwarp();
  // pass 1: upwind differences and the moments of Z*; G* and the differences stay in registers
  float2 gvr[P][NU], dr[P][NU];
  float2 E0[P], E1[P], E2[P];
#pragma unroll
  for (int s = 0; s < P; ++s) E0[s] = E1[s] = E2[s] = f2(0.f);
#pragma unroll
  for (int u = 0; u < NU; ++u)
#pragma unroll
    for (int s = 0; s < P; ++s) {
      const int m = s + P * 2 * u;
      const float2 gv = f2(rc[lane + 32 * m], rc[lane + 32 * (m + P)]);
      const float2 gu = f2((2 * u < S::TOP ? rt : rb)[lane + 32 * m],
                           (2 * u + 1 < S::TOP ? rt : rb)[lane + 32 * (m + P)]);
      const float2 d = sub2(gu, gv);
      gvr[s][u] = gv;
      dr[s][u] = d;
      const int p = l0[s] + ST * u;
      const float4 A = Y[5 * p];
      const float4 B = Y[5 * p + 1];
      E0[s] = __ffma2_rn(f2(A.x, A.y), d, E0[s]);
      E1[s] = __ffma2_rn(f2(A.z, A.w), d, E1[s]);
      E2[s] = __ffma2_rn(f2(B.x, B.y), d, E2[s]);
    }
  float Sy[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int s = 0; s < P; ++s) {
    const float e0 = E0[s].x + E0[s].y;
    Sy[0] += e0;
    Sy[1] = fmaf(c1[s], e0, Sy[1]);
    Sy[2] += E1[s].x + E1[s].y;
    Sy[3] += fmaf(c1q[s], e0, E2[s].x + E2[s].y);
  }
  warp_allsum4(Sy);
  const float b0 = fmaf(-Sy[3], inv2T, 2.f * Sy[0]);
  const float b1 = Sy[1] * iT, b2 = Sy[2] * iT;
  const float gm = fmaf(0.25f * Sy[3], iT * iT, -Sy[0] * inv2T);
  // per column: the polynomial coefficients of Ghat in c2 (times e1) and the ES Gaussian's
  // cross factor with its row ratio
  float A0[P], A1[P], A2[P], A3[P], x[P], rat[P];
  if constexpr (P == 1) {
    const float c = c1[0], cq = c1q[0];
    const float C0 = om1kap * fmaf(gm, cq, fmaf(b1, c, b0)) - c * fmaf(c, fmaf(c, w03, w02), w01) - ome;
    const float C1 = fmaf(om1kap, b2, -fmaf(c, fmaf(c, w12, w11), w10));
    const float C2 = fmaf(om1kap, gm, -fmaf(c, w21, w20));
    const float e1 = expf(-cq * inv2T);
    A0[0] = e1 * C0;
    A1[0] = e1 * C1;
    A2[0] = e1 * C2;
    A3[0] = -e1 * w30;
    const float c2r = fmaf(l0[0] + 0.5f, a.gf.dv2, a.gf.v2min) - u2;
    x[0] = gam0 * expf(-Ti11h * cq - Ti12 * c * c2r);
    rat[0] = expf(-Ti12 * c * (ST * a.gf.dv2));
  } else {
    // lane k evaluates column k's coefficients, the Gaussian factor at row 0 and the ratio r of
    // the cross factor between adjacent rows; the owners of column k fetch them by shuffle and
    // advance the Gaussian factor to their first row l0 by r^l0 (l0 < ST, a power of two)
    const float c = fmaf((lane < NV1 ? lane : 0) + 0.5f, a.gf.dv1, a.gf.v1min) - u1;
    const float cq = c * c;
    const float C0 = om1kap * fmaf(gm, cq, fmaf(b1, c, b0)) - c * fmaf(c, fmaf(c, w03, w02), w01) - ome;
    const float C1 = fmaf(om1kap, b2, -fmaf(c, fmaf(c, w12, w11), w10));
    const float C2 = fmaf(om1kap, gm, -fmaf(c, w21, w20));
    const float e1 = expf(-cq * inv2T);
    const float a0 = e1 * C0, a1 = e1 * C1, a2 = e1 * C2, a3 = -e1 * w30;
    const float c2z = fmaf(0.5f, a.gf.dv2, a.gf.v2min) - u2;
    const float x0 = gam0 * expf(-Ti11h * cq - Ti12 * c * c2z);
    const float r1 = expf(-Ti12 * c * a.gf.dv2);
    constexpr unsigned full = 0xffffffffu;
#pragma unroll
    for (int s = 0; s < P; ++s) {
      A0[s] = __shfl_sync(full, a0, kc[s]);
      A1[s] = __shfl_sync(full, a1, kc[s]);
      A2[s] = __shfl_sync(full, a2, kc[s]);
      A3[s] = __shfl_sync(full, a3, kc[s]);
      float r = __shfl_sync(full, r1, kc[s]);
      float xs = __shfl_sync(full, x0, kc[s]);
#pragma unroll
      for (int b = 1; b < ST; b <<= 1) {
        if (l0[s] & b) xs *= r;
        r *= r;
      }
      x[s] = xs;
      rat[s] = r;  // r1^ST
    }
  }
  // pass 2: G^{n+1} = om1 G* + wl (G*_up - G*) + Ghat + gamma exp(...), and the heat flux sums
  float2 H0[P], H1[P], H2[P], H3[P], xp[P];
  float rat2[P];
#pragma unroll
  for (int s = 0; s < P; ++s) {
    H0[s] = H1[s] = H2[s] = H3[s] = f2(0.f);
    xp[s] = f2(x[s], x[s] * rat[s]);  // the cross factor at visits 2u and 2u + 1
    rat2[s] = rat[s] * rat[s];
  }
  float* Go = a.Gout + (size_t)cell * S::NV + lane;
#pragma unroll
  for (int u = 0; u < NU; ++u)
#pragma unroll
    for (int s = 0; s < P; ++s) {
      const int p = l0[s] + ST * u;
      const float4 C = Y[5 * p + 2];
      const float4 D = Y[5 * p + 3];
      const float4 F = Y[5 * p + 4];
      float2 o = __ffma2_rn(f2(C.x, C.y), dr[s][u], __fmul2_rn(f2(om1), gvr[s][u]));
      const float2 c2p = f2(D.x, D.y);
      float2 pc = __ffma2_rn(f2(A3[s]), c2p, f2(A2[s]));
      pc = __ffma2_rn(pc, c2p, f2(A1[s]));
      pc = __ffma2_rn(pc, c2p, f2(A0[s]));
      o = __ffma2_rn(f2(C.z, C.w), pc, o);
      o = __ffma2_rn(f2(D.z, D.w), xp[s], o);
      xp[s] = __fmul2_rn(xp[s], f2(rat2[s]));
      const int m = s + P * 2 * u;
      Go[32 * m] = o.x;
      Go[32 * (m + P)] = o.y;
      H0[s] = __fadd2_rn(H0[s], o);
      H1[s] = __ffma2_rn(c2p, o, H1[s]);
      H2[s] = __ffma2_rn(f2(F.x, F.y), o, H2[s]);
      H3[s] = __ffma2_rn(f2(F.z, F.w), o, H3[s]);
    }
  float Hs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int s = 0; s < P; ++s) {
    Hs[0] = fmaf(c1q[s] * c1[s], H0[s].x + H0[s].y, Hs[0]);
    Hs[1] = fmaf(c1q[s], H1[s].x + H1[s].y, Hs[1]);
    Hs[2] = fmaf(c1[s], H2[s].x + H2[s].y, Hs[2]);
    Hs[3] += H3[s].x + H3[s].y;
  }
  warp_allsum4(Hs);
  if (lane < 8) a.Hf[lane * nc + cell] = (lane & 1) ? 0.f : Hs[lane >> 1];
  __syncwarp();
}

// dst[(k, l)] = src[(k, nv2 - 1 - l)]: the specular image of a cell's G* rows.
template <int NV1, int NV2>
__device__ __forceinline__ void mirror_rows(const float* src, float* dst) {
  using S = FlatShape<NV1, NV2>;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < S::M; ++m) {
    const int q = lane + 32 * m, l = q / NV1, k = q % NV1;
    dst[q] = src[(NV2 - 1 - l) * NV1 + k];
  }
  __syncwarp();
}

template <int NV1, int NV2>
__global__ void __launch_bounds__(32 * kFusedWarps, 4) k_micro_flat_f32(FusedF32 a) {
  using S = FlatShape<NV1, NV2>;
  extern __shared__ __align__(16) float smf[];
  const KGrid& g = a.g;
  const int w = threadIdx.x >> 5;
  float* ring = smf + (size_t)w * S::PER_WARP;
  float* xt = ring + 3 * S::NV;
  float* yt = xt + 4 * NV2;
  float* fld = yt + 10 * NV2;
  const int gw = blockIdx.x * kFusedWarps + w;
  if (gw >= g.nx * a.nseg) return;  // whole warp leaves; no CTA-wide barrier is used below
  const int i = gw % g.nx;
  const int seg = gw / g.nx;
  const int j0 = seg * a.seg_rows;
  const int j1 = min(g.ny, j0 + a.seg_rows);
  if (j0 >= j1) return;
  const bool pery = a.p.bc[2] == MM_BC_PERIODIC;
  auto slot = [&](int pos) { return ring + (size_t)(pos % 3) * S::NV; };
  // the g block of the cell two rows ahead goes to L2 while this row is swept, so that the x
  // sweep's loads of the next-but-one iteration wait on L2 rather than on HBM
  auto prefetch = [&](int jj) {
    if ((threadIdx.x & 31) == 0 && jj < g.ny)
      l2_prefetch_bulk(a.Gin + (size_t)(jj * g.nx + i) * S::NV, (unsigned)(S::NV * sizeof(float)));
  };
  // a cell's fields into the warp's shared-memory slot (lane f reads field f); the previous
  // sweep ended with a warp barrier, so nobody reads the slot any more
  auto fields_of = [&](int cell) {
    const float f = load_fields(a.pf, g.nx * g.ny, cell);
    if ((threadIdx.x & 31) < NPRIMF) fld[threadIdx.x & 31] = f;
    __syncwarp();
    return fld;
  };
  auto xsweep = [&](int jj, float* dst) {
    const UpwindF ul = upwind_side(g, a.p, i, jj, 0), ur = upwind_side(g, a.p, i, jj, 1);
    const float* Gl = ul.zero ? kZeroRowF : a.Gin + (size_t)ul.cell * S::NV;
    const float* Gr = ur.zero ? kZeroRowF : a.Gin + (size_t)ur.cell * S::NV;
    fx_sweep<NV1, NV2, false>(a, i, jj, dst, xt, a.Gin + (size_t)(jj * g.nx + i) * S::NV, Gl, Gr,
                              ul.mirror, ur.mirror, fields_of(jj * g.nx + i));
  };
  prefetch(j0 + 1);
  if (j0 > 0 || pery) xsweep(j0 > 0 ? j0 - 1 : g.ny - 1, slot(0));
  xsweep(j0, slot(1));
  for (int j = j0; j < j1; ++j) {
    const int pos = j - j0 + 1;
    prefetch(j + 2);
    if (j + 1 < g.ny || pery) xsweep(j + 1 < g.ny ? j + 1 : 0, slot(pos + 1));
    if (diffuse_wall_cell(g, a.p, i, j)) continue;  // finished by the wall kernel
    const float* rc = slot(pos);
    const bool hasb = j > 0 || pery, hast = j < g.ny - 1 || pery;
    // a missing neighbour's slot is free: it takes the specular image of the cell's rows
    const float* rb = rc;
    if (hasb) rb = slot(pos + 2);
    else if (a.p.bc[2] == MM_BC_SPECULAR) { mirror_rows<NV1, NV2>(rc, slot(pos + 2)); rb = slot(pos + 2); }
    const float* rt = rc;
    if (hast) rt = slot(pos + 1);
    else if (a.p.bc[3] == MM_BC_SPECULAR) { mirror_rows<NV1, NV2>(rc, slot(pos + 1)); rt = slot(pos + 1); }
    fy_sweep<NV1, NV2>(a, i, j, rb, rc, rt, yt, fields_of(j * g.nx + i));
  }
}

// ------------------------------------------------------------------------------------------
// Staged variant: the warps of a CTA sweep W adjacent columns in step, and the g blocks that the
// x sweeps of the next-but-one row read (the W cells and one halo cell on each side) arrive in a
// shared-memory stage by bulk asynchronous copies while the current row is swept in y.  One
// thread issues the copies and an mbarrier counts their bytes; every wait on it is bounded and a
// wait that runs out sets ERR_WAIT_TIMEOUT and ends the CTA.
// ------------------------------------------------------------------------------------------
constexpr int kWaitSpins = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  int spins = kWaitSpins) {
  for (int it = 0; it < spins; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Diagnostic of the bounded wait: one warp arms an mbarrier for 16 bytes and, when copy != 0,
// issues the 16-byte bulk copy that completes it; otherwise nothing ever completes the phase and
// the wait must run out after spins attempts.  *timed_out receives 1 if it did.
__global__ void k_diag_bounded_wait(int copy, int spins, int* __restrict__ timed_out) {
  __shared__ __align__(16) float buf[4];
  __shared__ __align__(8) unsigned long long mb;
  const uint32_t bar = smem_addr(&mb);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(16u)
                 : "memory");
    if (copy)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, "
          "[%2];" ::"r"(smem_addr(buf)),
          "l"(kZeroRowF), "r"(bar)
          : "memory");
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, 0u, spins));
  if (threadIdx.x == 0) *timed_out = ok ? 0 : 1;
}

template <int NV1, int NV2>
struct StagedShape {
  using S = FlatShape<NV1, NV2>;
  static constexpr int W = kFusedWarps;
  static constexpr int STAGE = (W + 2) * S::NV;  // floats: the g blocks of columns i0-1 .. i0+W
  static constexpr int RING = 3 * S::NV;          // per warp
  // per warp: the x sweep's tables (4 NV2 floats) and the y sweep's (10 NV2) share one area; a
  // warp's sweeps run one after the other with a warp barrier between them
  static constexpr int TABLES = 10 * NV2;
  static constexpr int FIELDS = 3 * kFieldSlot;  // per warp: fields of three x-swept rows
  // stage buffers (rows in flight): one; two leave room for 3 CTAs per SM only and measured
  // slower (2.02 against 1.86 ms at 1024^2 x 24^2)
  static constexpr int NSTAGE = 1;
  // + a full and an empty mbarrier per stage buffer and the abort flag
  static constexpr int FLOATS = NSTAGE * STAGE + W * (RING + TABLES + FIELDS) + 4 * NSTAGE + 2;
};

// Source of stage slot sigma (column c = i0 - 1 + sigma) for row jj: the column's block; beyond
// a side the block the x sweep treats as upwind there (periodic partner, the edge cell itself for
// extrapolation and specular sides, the zero row for a diffuse side); NULL past the right halo.
__device__ __forceinline__ const float* stage_source(const FusedF32& a, int c, int jj, int nv) {
  const KGrid& g = a.g;
  if (c < -1 || c > g.nx) return nullptr;
  if (c == -1 || c == g.nx) {
    const int side = c < 0 ? 0 : 1;
    const int bc = a.p.bc[side];
    if (bc == MM_BC_DIFFUSE) return kZeroRowF;
    if (bc == MM_BC_PERIODIC) c = side == 0 ? g.nx - 1 : 0;
    else c = side == 0 ? 0 : g.nx - 1;
  }
  return a.Gin + (size_t)(jj * g.nx + c) * nv;
}

// Compiled for 4 CTAs per SM (128 registers): measured faster than 3 (no spills, 12 warps).
template <int NV1, int NV2>
__global__ void __launch_bounds__(32 * kFusedWarps, 4) k_micro_staged_f32(FusedF32 a) {
  using S = FlatShape<NV1, NV2>;
  using T = StagedShape<NV1, NV2>;
  constexpr int W = T::W;
  extern __shared__ __align__(16) float smf[];
  const KGrid& g = a.g;
  const int w = threadIdx.x >> 5;
  constexpr int NS = T::NSTAGE;
  float* stage0 = smf;
  float* ring = smf + NS * T::STAGE + w * (T::RING + T::TABLES);
  float* xt = ring + T::RING;
  float* yt = xt;
  // full: the stage holds the next row (the bulk copies' bytes have landed); empty: every warp
  // has finished reading the stage, so that it may be refilled
  // per-cell fields of the x-swept rows in three slots like the G* ring (a row's fields serve
  // its x sweep and, one iteration later, its y sweep), fetched two rows ahead by cp.async
  float* fld = smf + NS * T::STAGE + W * (T::RING + T::TABLES) + w * T::FIELDS;
  float* bars = smf + NS * T::STAGE + W * (T::RING + T::TABLES + T::FIELDS);
  auto bar_full = [&](int b) { return smem_addr(bars + 4 * b); };
  auto bar_empty = [&](int b) { return smem_addr(bars + 4 * b + 2); };
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 4 * NS);
  const int ncx = (g.nx + W - 1) / W;
  const int cx = blockIdx.x % ncx, seg = blockIdx.x / ncx;
  const int i0 = cx * W, i = i0 + w;
  const bool col = i < g.nx;  // warps past the last column only read nothing from the stage
  const int j0 = seg * a.seg_rows;
  const int j1 = min(g.ny, j0 + a.seg_rows);
  if (j0 >= j1) return;  // uniform over the CTA
  const bool pery = a.p.bc[2] == MM_BC_PERIODIC;
  const bool mirl = i == 0 && a.p.bc[0] == MM_BC_SPECULAR;
  const bool mirr = i == g.nx - 1 && a.p.bc[1] == MM_BC_SPECULAR;
  const int lane = threadIdx.x & 31;
  auto slot = [&](int pos) { return ring + (size_t)(pos % 3) * S::NV; };

  if (threadIdx.x == 0) {
    for (int b = 0; b < NS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_full(b)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_empty(b)), "r"(W)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  __syncthreads();
  // bulk copies of row jj's blocks into the stage (thread 0)
  auto issue = [&](int jj, int b) {
    float* stage = stage0 + b * T::STAGE;
    const uint32_t bar = bar_full(b);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const float* src[W + 2];
    unsigned bytes = 0;
#pragma unroll
    for (int sg = 0; sg < W + 2; ++sg) {
      src[sg] = stage_source(a, i0 - 1 + sg, jj, S::NV);
      if (src[sg]) bytes += S::NV * sizeof(float);
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
#pragma unroll
    for (int sg = 0; sg < W + 2; ++sg)
      if (src[sg])
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(smem_addr(stage + sg * S::NV)),
            "l"(src[sg]), "r"((unsigned)(S::NV * sizeof(float))), "r"(bar)
            : "memory");
  };
  // the x sweeps of this segment, in order: the halo row below (if any), j0, then j0+1 .. j1
  // (wrapping for periodic y; the last one only if it exists)
  const bool halo = j0 > 0 || pery;
  const int jlast = (j1 < g.ny || pery) ? j1 : j1 - 1;  // last x-swept row (before wrapping)
  const int nx_rows = (halo ? 1 : 0) + (jlast - j0 + 1);
  auto xrow = [&](int n) {  // the n-th x-swept row
    int jj = (halo ? j0 - 1 : j0) + n;
    if (jj < 0) jj += g.ny;
    if (jj >= g.ny) jj -= g.ny;
    return jj;
  };
  // x-swept row n uses stage buffer n % NS, in that buffer's phase (n / NS) & 1
  unsigned pending = 0;  // thread 0: bit b set while a copy into buffer b has not been awaited
  if (threadIdx.x == 0)
    for (int b = 0; b < NS && b < nx_rows; ++b) {
      issue(xrow(b), b);
      pending |= 1u << b;
    }
  // fields of ring position pos (x-swept row number pos - fpos0): lane f copies field f
  const int fpos0 = halo ? 0 : 1;
  auto fslot = [&](int pos) { return fld + (pos % 3) * kFieldSlot; };
  auto fetch = [&](int pos) {
    const int xn = pos - fpos0;
    if (col && xn >= 0 && xn < nx_rows && lane < NPRIMF) {
      const float* src = a.pf + (size_t)lane * g.nx * g.ny + (size_t)xrow(xn) * g.nx + i;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(fslot(pos) + lane)),
                   "l"(src)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto fields_landed = [&]() {  // every fetch but the newest has landed, for every lane
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();
  };
  fetch(0);
  fetch(1);
  fetch(2);
  fields_landed();
  // Give up after a wait ran out (here or in another warp): thread 0 first lets its copies land
  // (bounded again), so that no bulk copy writes into the shared memory of a finished CTA; at x
  // row n the copies not yet awaited are those of rows n .. n + NS - 1.
  auto give_up = [&](int n) {
    if (lane == 0) {
      atomicOr(a.err, ERR_WAIT_TIMEOUT);
      *abort_flag = 1;
    }
    if (threadIdx.x == 0)
      for (int r = n; r < n + NS; ++r)
        if (pending & (1u << (r % NS))) mbar_wait_bounded(bar_full(r % NS), (r / NS) & 1u);
    asm volatile("cp.async.wait_all;" ::: "memory");
    return false;
  };
  // x sweep number n into ring position pos; the warp then releases the stage, and thread 0
  // refills it with the next row as soon as every warp has released it (the other warps go on
  // to their y sweeps meanwhile)
  auto xstep = [&](int n, int pos) -> bool {
    if (*abort_flag) return give_up(n);
    const int jj = xrow(n);
    const int b = n % NS;
    const uint32_t ph = (n / NS) & 1u;
    float* stage = stage0 + b * T::STAGE;
    // the sweep's warp shuffles need every lane: a warp sweeps only if all its lanes saw the copy
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar_full(b), ph));
    if (!ok) return give_up(n);
    if (threadIdx.x == 0) pending &= ~(1u << b);
    if (col)
      fx_sweep<NV1, NV2, true>(a, i, jj, slot(pos), xt, stage + (w + 1) * S::NV,
                               stage + w * S::NV, stage + (w + 2) * S::NV, mirl, mirr,
                               fslot(pos));
    __syncwarp();
    if (lane == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_empty(b)) : "memory");
    if (threadIdx.x == 0) {
      const bool free = mbar_wait_bounded(bar_empty(b), ph);
      if (free && n + NS < nx_rows) {
        issue(xrow(n + NS), b);
        pending |= 1u << b;
      }
      if (!free) {
        atomicOr(a.err, ERR_WAIT_TIMEOUT);
        *abort_flag = 1;
      }
    }
    __syncwarp();
    return true;
  };
  int n = 0;
  if (halo && !xstep(n++, 0)) return;
  if (!xstep(n++, 1)) return;
  for (int j = j0; j < j1; ++j) {
    const int pos = j - j0 + 1;
    fetch(pos + 2);    // for the next iteration's x sweep, into the slot of row j - 1
    fields_landed();   // row j + 1's, for this iteration's x sweep
    if (j + 1 < g.ny || pery)
      if (!xstep(n++, pos + 1)) return;
    if (!col || diffuse_wall_cell(g, a.p, i, j)) continue;  // wall cells: the wall kernel
    const float* rc = slot(pos);
    const bool hasb = j > 0 || pery, hast = j < g.ny - 1 || pery;
    const float* rb = rc;
    if (hasb) rb = slot(pos + 2);
    else if (a.p.bc[2] == MM_BC_SPECULAR) { mirror_rows<NV1, NV2>(rc, slot(pos + 2)); rb = slot(pos + 2); }
    const float* rt = rc;
    if (hast) rt = slot(pos + 1);
    else if (a.p.bc[3] == MM_BC_SPECULAR) { mirror_rows<NV1, NV2>(rc, slot(pos + 1)); rt = slot(pos + 1); }
    fy_sweep<NV1, NV2>(a, i, j, rb, rc, rt, yt, fslot(pos));
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// The kernel for a velocity mesh and its shared memory per CTA.  Flat-mapped kernels for the
// 32^2, 24^2 and 16^2 meshes when the v2 mesh is symmetric (the rows with v2 < 0, evaluated in
// FP32 as on the device, are exactly the first half); otherwise the column-mapped kernel
// (compile-time shape where it has one).
struct FusedPick {
  void (*kern)(FusedF32);
  size_t smem;
};

static bool v2_symmetric_f32(const KGrid& g) {
  const float dv2 = (float)g.dv2, v2min = (float)g.v2min;  // as rounded for the FP32 kernels
  if (g.nv2 % 2) return false;
  int nneg = 0;
  for (int l = 0; l < g.nv2; ++l) nneg += std::fmaf(l + 0.5f, dv2, v2min) < 0.f ? 1 : 0;
  return nneg == g.nv2 / 2;
}

// Shared memory per CTA of the column-mapped kernel: per warp a three-row ring of G* (rounded up
// to 16 bytes), the x-sweep tables (2 float2 per row) and the y-sweep tables (3 float4 + 1 float2
// per row), the whole padded to a multiple of 16 bytes so that every warp's float4 tables stay
// aligned.
static size_t column_smem(const KGrid& g) {
  const size_t nv = (size_t)g.nv1 * g.nv2;
  const size_t per_warp = (3 * nv + 3) / 4 * 4 + 18 * (size_t)g.nv2 + (g.nv2 & 1) * 2;
  return sizeof(float) * kFusedWarps * per_warp;
}

template <int NV1, int NV2>
static FusedPick flat_pick() {
  return FusedPick{k_micro_flat_f32<NV1, NV2>,
                   sizeof(float) * kFusedWarps * (size_t)FlatShape<NV1, NV2>::PER_WARP};
}

template <int NV1, int NV2>
static FusedPick staged_pick() {
  return FusedPick{k_micro_staged_f32<NV1, NV2>,
                   sizeof(float) * (size_t)StagedShape<NV1, NV2>::FLOATS};
}

static FusedPick pick_fused(const KGrid& g) {
  const bool sym = v2_symmetric_f32(g);
  if (sym && g.nv1 == 32 && g.nv2 == 32) return flat_pick<32, 32>();
  if (sym && g.nv1 == 24 && g.nv2 == 24) return staged_pick<24, 24>();
  if (sym && g.nv1 == 16 && g.nv2 == 16) return staged_pick<16, 16>();
  const size_t smem = column_smem(g);
  if (g.nv1 == 32 && g.nv2 == 32) return FusedPick{k_micro_fused_f32<32, 32>, smem};
  if (g.nv1 == 24 && g.nv2 == 24) return FusedPick{k_micro_fused_f32<24, 24>, smem};
  if (g.nv1 == 16 && g.nv2 == 16) return FusedPick{k_micro_fused_f32<16, 16>, smem};
  return FusedPick{k_micro_fused_f32<0, 0>, smem};
}


// ------------------------------------------------------------------------------------------
// Diffuse-wall cells of the FP32-g step (Section 6.3): the y sweep, the relaxation toward the
// wall form of Ghat, -(1/tau)(I - Pi_M)[upwind v.grad M] with ghost wall Maxwellians (plus
// (G - M)/eps when kept), and the heat flux, from the G* the streaming kernel exported.  One CTA
// per wall cell.  The per-cell quantities (wall densities with their error functions, the
// Maxwellian prefactors) are FP64, rounded once; the per-velocity arithmetic is FP32, as in the
// streaming kernel, since FP64 runs at 1/64 of the FP32 rate on this GPU.
// ------------------------------------------------------------------------------------------
constexpr int kWallThreadsF = 128;

// Sum N floats over the CTA (kWallThreadsF threads, fixed order); every thread gets the totals.
template <int N>
__device__ __forceinline__ void cta_sum(float (&v)[N], float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < N; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
  if (lane == 0)
#pragma unroll
    for (int m = 0; m < N; ++m) red[w * N + m] = v[m];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < N; ++m) {
    float s = red[m];
    for (int q = 1; q < kWallThreadsF / 32; ++q) s += red[q * N + m];
    v[m] = s;
  }
  __syncthreads();
}

// Eq. (twodim_wall_densities_1): the ghost density factor of a diffuse wall for the normal
// velocity ua and normal temperature Taa of the cell, wall temperature Tw.
__device__ __forceinline__ double wall_density_factor(double ua, double Taa, double Tw,
                                                      double sgn) {
  constexpr double kPiD = 3.14159265358979323846;
  return sqrt(Taa / Tw) * exp(-ua * ua / (2.0 * Taa)) +
         ua * sqrt(kPiD / (2.0 * Tw)) * (erf(ua / sqrt(2.0 * Taa)) + sgn);
}

__global__ void __launch_bounds__(kWallThreadsF) k_wall_f32(const float* __restrict__ Gs,
                                                            float* __restrict__ Gout,
                                                            double* __restrict__ Hout,
                                                            const double* __restrict__ Q,
                                                            const double* __restrict__ prim,
                                                            const int* __restrict__ wall_cells,
                                                            KGrid g, KParams p, double dt,
                                                            double eps, int* __restrict__ err) {
  extern __shared__ __align__(16) float sw[];
  const int nv1 = g.nv1, nv2 = g.nv2, nv = nv1 * nv2;
  float* Xt = sw;              // [5][nv1]: v1 factors of the four side Maxwellians and the cell's
  float* Yt = Xt + 5 * nv1;    // [5][nv2]: v2 factors
  float* Et = Yt + 5 * nv2;    // [nv2]: row factor of the ES Gaussian
  float* red = Et + nv2;       // reduction scratch
  __shared__ float sf[5][4];   // (u1, u2, 1 / (2 T), rho / (2 pi T)) of the five Maxwellians
  __shared__ float cs[13];     // per-cell scalars, rounded once
  __shared__ int kind[4];      // 0 neighbour / periodic, 1 extrapolation, 2 specular, 3 diffuse
  const int cell = wall_cells[blockIdx.x];
  const int nc = g.nx * g.ny, i = cell % g.nx, j = cell / g.nx, t = threadIdx.x;
  constexpr double kInv2Pi = 0.15915494309189533577;  // 1 / (2 pi)
  // FP64 work of the cell on the first warp only: lanes 0..3 the four sides' Maxwellians (the
  // neighbour's, or the wall's with its density factor), lane 4 the cell's, lane 0 the scalars
  if (t < 32) {
    // the cell's moments; (u1, u2, T) of every cell from the fields kernel
    const double rho = Q[cell], u1 = prim[P_U1 * nc + cell];
    const double u2 = prim[P_U2 * nc + cell], T = prim[P_T * nc + cell];
    const double ir = 1.0 / rho;
    const double P11 = Q[3 * nc + cell] - rho * u1 * u1;
    const double P12 = Q[4 * nc + cell] - rho * u1 * u2;
    const double P22 = Q[5 * nc + cell] - rho * u2 * u2;
    double q0 = u1, q1 = u2, q2 = T, q3 = rho;
    int kd = 0;
    if (t < 4) {
      const int s = t;
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
        q0 = prim[P_U1 * nc + c];
        q1 = prim[P_U2 * nc + c];
        q2 = prim[P_T * nc + c];
        q3 = Q[c];
      } else if (p.bc[s] == MM_BC_EXTRAP) {
        kd = 1;
      } else if (p.bc[s] == MM_BC_SPECULAR) {
        kd = 2;
      } else {
        kd = 3;
        const double Tw = p.wall_T[s], U = p.wall_U[s];
        const double sgn = (s == 0 || s == 2) ? -1.0 : 1.0;
        q3 = s < 2 ? rho * wall_density_factor(u1, P11 * ir, Tw, sgn)
                   : rho * wall_density_factor(u2, P22 * ir, Tw, sgn);
        q0 = s < 2 ? 0.0 : U;
        q1 = s < 2 ? U : 0.0;
        q2 = Tw;
      }
      kind[s] = kd;
    }
    if (t < 5) {
      const double iq = 1.0 / q2;
      sf[t][0] = (float)q0;
      sf[t][1] = (float)q1;
      sf[t][2] = (float)(0.5 * iq);
      sf[t][3] = (float)(q3 * iq * kInv2Pi);
    }
    if (t == 0) {
      // tau, and the inverse and normalisation of the ES tensor (Eq. 2-19)
      const double tau = macro_body::tau_of(p, rho, T);
      const double nu = p.nu;
      const double s11 = (1.0 - nu) * T + nu * (P11 * ir), s12 = nu * (P12 * ir);
      const double s22 = (1.0 - nu) * T + nu * (P22 * ir);
      const double det = s11 * s22 - s12 * s12, idet = 1.0 / det;
      const double r = 1.0 / (eps + dt * tau), iT = 1.0 / T;
      cs[0] = (float)(eps * r);       // om1
      cs[1] = (float)(dt * tau * r);  // om2
      cs[2] = (float)(1.0 / tau);
      cs[3] = (float)(1.0 / eps);
      cs[4] = (float)(0.5 * iT);
      cs[5] = (float)iT;
      cs[6] = (float)(g.dv1 * g.dv2 * kInv2Pi * iT);  // kap
      cs[7] = (float)(rho * kInv2Pi * rsqrt(det));  // KG
      cs[8] = (float)(s22 * idet);                   // Ti11
      cs[9] = (float)(-s12 * idet);                  // Ti12
      cs[10] = (float)(s11 * idet);                  // Ti22
      cs[11] = (float)u1;
      cs[12] = (float)u2;
    }
  }
  __syncthreads();
  const float v1min = (float)g.v1min, dv1 = (float)g.dv1;
  const float v2min = (float)g.v2min, dv2 = (float)g.dv2;
  for (int e = t; e < 5 * nv1; e += kWallThreadsF) {
    const int q = e / nv1;
    const float d = fmaf(e % nv1 + 0.5f, dv1, v1min) - sf[q][0];
    Xt[e] = expf(-d * d * sf[q][2]);
  }
  for (int e = t; e < 5 * nv2; e += kWallThreadsF) {
    const int q = e / nv2;
    const float d = fmaf(e % nv2 + 0.5f, dv2, v2min) - sf[q][1];
    Yt[e] = expf(-d * d * sf[q][2]);
  }
  const float om1 = cs[0], om2 = cs[1], itau = cs[2], ieps = cs[3];
  const float inv2T = cs[4], iT = cs[5], kap = cs[6], KG = cs[7];
  const float Ti11 = cs[8], Ti12 = cs[9], Ti22 = cs[10], u1f = cs[11], u2f = cs[12];
  if (p.keep_es)
    for (int l = t; l < nv2; l += kWallThreadsF) {
      const float c2 = fmaf(l + 0.5f, dv2, v2min) - u2f;
      Et[l] = expf(-0.5f * Ti22 * c2 * c2);
    }
  __syncthreads();

  const float idx = (float)g.idx, idy = (float)g.idy;
  int kd[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) kd[s] = kind[s];
  const float pf4 = sf[4][3];
  // the Maxwellian of side s at (k, l), for the upwind v.grad M (m0: the cell's own)
  auto side_m = [&](int s, float m0, int k, int l) -> float {
    if (kd[s] == 1) return m0;
    if (kd[s] == 2)
      return s < 2 ? pf4 * Xt[4 * nv1 + nv1 - 1 - k] * Yt[4 * nv2 + l]
                   : pf4 * Xt[4 * nv1 + k] * Yt[4 * nv2 + nv2 - 1 - l];
    return sf[s][3] * Xt[s * nv1 + k] * Yt[s * nv2 + l];
  };
  auto mup = [&](int k, int l, float v1, float v2, float m0) -> float {
    float z = 0.f;
    if (v1 > 0.f) z += v1 * ((m0 - side_m(0, m0, k, l)) * idx);
    if (v1 < 0.f) z += v1 * ((side_m(1, m0, k, l) - m0) * idx);
    if (v2 > 0.f) z += v2 * ((m0 - side_m(2, m0, k, l)) * idy);
    if (v2 < 0.f) z += v2 * ((side_m(3, m0, k, l) - m0) * idy);
    return z;
  };
  const UpwindF ub = upwind_side(g, p, i, j, 2), ut = upwind_side(g, p, i, j, 3);
  const float* Gc = Gs + (size_t)cell * nv;
  const float* Gb = Gs + (size_t)ub.cell * nv;
  const float* Gt = Gs + (size_t)ut.cell * nv;
  // G*, its upwind y difference term z = -|v2| (G*_up - G*) / dy and the cell's Maxwellian at
  // element e = l nv1 + k
  auto element = [&](int e, int& k, int& l, float& v1, float& v2, float& gv, float& z,
                     float& ml) {
    k = e % nv1;
    l = e / nv1;
    v1 = fmaf(k + 0.5f, dv1, v1min);
    v2 = fmaf(l + 0.5f, dv2, v2min);
    gv = Gc[e];
    const bool top = v2 < 0.f;
    const UpwindF& u = top ? ut : ub;
    const int lu = u.mirror ? nv2 - 1 - l : l;
    const float gu = u.zero ? 0.f : (top ? Gt : Gb)[lu * nv1 + k];
    z = -fabsf(v2) * idy * (gu - gv);
    ml = Xt[4 * nv1 + k] * Yt[4 * nv2 + l];  // M / (rho / (2 pi T))
  };
  // pass 1: moments (1, c1, c2, |c|^2) of Z* and of the upwind v.grad M
  float S[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int e = t; e < nv; e += kWallThreadsF) {
    int k, l;
    float v1, v2, gv, z, ml;
    element(e, k, l, v1, v2, gv, z, ml);
    const float c1 = v1 - u1f, c2 = v2 - u2f, cc = fmaf(c1, c1, c2 * c2);
    const float mz = mup(k, l, v1, v2, pf4 * ml);
    S[0] += z;
    S[1] = fmaf(c1, z, S[1]);
    S[2] = fmaf(c2, z, S[2]);
    S[3] = fmaf(cc, z, S[3]);
    S[4] += mz;
    S[5] = fmaf(c1, mz, S[5]);
    S[6] = fmaf(c2, mz, S[6]);
    S[7] = fmaf(cc, mz, S[7]);
  }
  cta_sum<8>(S, red);
  // projection polynomials kap (b0 + b1 c1 + b2 c2 + gm |c|^2) of Z* (S[0..3]) and of v.grad M
  // (S[4..7])
  float B[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float* m4 = S + 4 * q;
    B[q][0] = kap * fmaf(-m4[3], inv2T, 2.f * m4[0]);
    B[q][1] = kap * (m4[1] * iT);
    B[q][2] = kap * (m4[2] * iT);
    B[q][3] = kap * fmaf(0.25f * m4[3], iT * iT, -m4[0] * inv2T);
  }
  const float dtf = (float)dt;
  // pass 2: G^{n+1} = om1 G** + om2 Ghat with G** = G* + dt (Pi_M Z* - Z*), and the heat flux
  float Hs[4] = {0.f, 0.f, 0.f, 0.f};
  float* Go = Gout + (size_t)cell * nv;
  for (int e = t; e < nv; e += kWallThreadsF) {
    int k, l;
    float v1, v2, gv, z, ml;
    element(e, k, l, v1, v2, gv, z, ml);
    const float c1 = v1 - u1f, c2 = v2 - u2f;
    const float c1q = c1 * c1, cq = fmaf(c2, c2, c1q);
    const float ps = fmaf(B[0][3], cq, fmaf(B[0][2], c2, fmaf(B[0][1], c1, B[0][0])));
    const float pw = fmaf(B[1][3], cq, fmaf(B[1][2], c2, fmaf(B[1][1], c1, B[1][0])));
    const float m = pf4 * ml;
    const float gs2 = fmaf(dtf, fmaf(ps, ml, -z), gv);
    float gh = -itau * (mup(k, l, v1, v2, m) - pw * ml);
    if (p.keep_es)
      gh = fmaf(fmaf(KG * expf(fmaf(-0.5f * Ti11, c1q, -Ti12 * c1 * c2)), Et[l], -m), ieps, gh);
    const float o = fmaf(om1, gs2, om2 * gh);
    Go[e] = o;
    Hs[0] = fmaf(c1q * c1, o, Hs[0]);
    Hs[1] = fmaf(c1q * c2, o, Hs[1]);
    Hs[2] = fmaf(c1 * (c2 * c2), o, Hs[2]);
    Hs[3] = fmaf(c2 * (c2 * c2), o, Hs[3]);
  }
  cta_sum<4>(Hs, red);
  if (t == 0) {
    const double f = eps * g.dv1 * g.dv2;
    bool ok = true;
    for (int m = 0; m < 4; ++m) {
      Hout[m * nc + cell] = f * (double)Hs[m];
      ok = ok && isfinite(Hs[m]);
    }
    if (!ok) atomicOr(err, ERR_NONFINITE_G);
  }
}

}  // namespace

size_t fused_smem_f32(const KGrid& g) { return pick_fused(g).smem; }

size_t wall_smem_f32(const KGrid& g) {
  return sizeof(float) * (5 * (size_t)g.nv1 + 6 * (size_t)g.nv2 + 8 * (kWallThreadsF / 32));
}

void launch_wall_f32(const float* Gs, float* Gout, double* H, const double* Q,
                     const double* prim, const int* wall_cells, int n_wall, const KGrid& g,
                     const KParams& p, double dt, double eps, int* err, cudaStream_t s) {
  if (n_wall <= 0) return;
  k_wall_f32<<<n_wall, kWallThreadsF, wall_smem_f32(g), s>>>(Gs, Gout, H, Q, prim, wall_cells, g,
                                                            p, dt, eps, err);
}

KGridF grid_f32(const KGrid& g) {
  return KGridF{(float)g.v1min, (float)g.v2min, (float)g.dv1, (float)g.dv2, (float)g.idx,
                (float)g.idy};
}

int fused_segments_f32(const KGrid& g, const MicroShape& ms) {
  (void)ms;
  const FusedPick f = pick_fused(g);
  int per_sm = 0;
  if (f.smem > 48 * 1024)
    cudaFuncSetAttribute(f.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f.kern, 32 * kFusedWarps, f.smem);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long resident = (long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1) * kFusedWarps;
  // about four resident waves of columns (three and four measured best of 2 ... 8), but at
  // least 16 rows per segment
  long nseg = (4 * resident + g.nx - 1) / g.nx;
  const long max_seg = g.ny / 16 > 1 ? g.ny / 16 : 1;
  if (nseg > max_seg) nseg = max_seg;
  if (nseg < 1) nseg = 1;
  return (int)nseg;
}

void launch_micro_fused_f32(const float* Gin, float* Gout, float* Gexp, float* Hf,
                            const float* primf, const KGrid& g, const KParams& p, double dt,
                            const MicroShape& ms, int nseg, int* err, cudaStream_t s) {
  (void)ms;
  const FusedPick f = pick_fused(g);
  FusedF32 a;
  a.err = err;
  a.Gin = Gin;
  a.Gout = Gout;
  a.Gexp = Gexp;
  a.Hf = Hf;
  a.pf = primf;
  a.g = g;
  a.gf = grid_f32(g);
  a.p = p;
  a.dtidx = (float)(dt * g.idx);
  a.dtidy = (float)(dt * g.idy);
  a.R = 32 / g.nv1;
  a.seg_rows = (g.ny + nseg - 1) / nseg;
  a.nseg = nseg;
  // one warp per column and segment; the staged kernels give a CTA kFusedWarps adjacent columns
  const int warps = ((g.nx + kFusedWarps - 1) / kFusedWarps) * kFusedWarps * a.nseg;
  if (f.smem > 48 * 1024)
    cudaFuncSetAttribute(f.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.smem);
  f.kern<<<(warps + kFusedWarps - 1) / kFusedWarps, 32 * kFusedWarps, f.smem, s>>>(a);
}

}  // namespace mmk

extern "C" mm_status mm_diag_bounded_wait(int copy, int spins, void* cuda_stream) {
  if (spins < 1) return MM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* d = nullptr;
  int h = -1;
  cudaError_t e = cudaMalloc((void**)&d, sizeof(int));
  if (e == cudaSuccess) {
    mmk::k_diag_bounded_wait<<<1, 32, 0, s>>>(copy, spins, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
  }
  if (e != cudaSuccess) return MM_ERR_CUDA;
  return h ? MM_ERR_TIMEOUT : MM_OK;
}
