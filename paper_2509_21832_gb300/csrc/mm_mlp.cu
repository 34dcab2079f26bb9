// Learned heat-flux closure: a small MLP (39 -> 64 -> 64 -> 4, GELU) with BF16 weights and FP32
// accumulation, trained and evaluated by these kernels.  The network maps local macro features
// of a cell to the dimensionless non-Navier-Stokes part of the heat-flux tensor of Eq. (5-99):
// H = H_CE + eps rho T^{3/2} y, where H_CE is the Chapman-Enskog value, i.e. the moments of the
// transport part of Ghat (Eq. 5-97) for a Gaussian: H111 = -3 eps p Tx / tau, H112 = -eps p Ty /
// tau, H122 = -eps p Tx / tau, H222 = -3 eps p Ty / tau (p = rho T).
//
// Kernels: inference (tensor cores, split-TF32 activations), training forward/backward and
// weight gradients on the tensor cores with BF16 operands and FP32 accumulation (fixed-order
// reductions: deterministic), and Adam on FP32 master weights that refreshes the BF16 copies.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mm_body_mlp.cuh"

using namespace mmk;
using namespace mmk::mlp_body;

namespace {

// Inference, 32 samples per warp pass (two m16 tiles); weights staged once per CTA.
__global__ void __launch_bounds__(kInferThreads, 4) k_mlp_infer(const __nv_bfloat16* __restrict__ w,
                                                             const float* __restrict__ norm,
                                                             const float* __restrict__ X,
                                                             float* __restrict__ Y, int n) {
  extern __shared__ __align__(16) float smi[];
  float* sw = smi;
  float* sn = smi + kINP;
  float* tile = smi + kINP + 88 + (threadIdx.x >> 5) * kTile;
  stage_infer(w, norm, sw, sn);
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * kInferThreads; base < n; base += gridDim.x * kInferThreads) {
    const int s = base + threadIdx.x;  // this lane's sample
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) x[i] = s < n ? X[(size_t)s * kIn + i] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if ((lane >> 4) == h) put_row(tile, lane & 15, x, sn);
      __syncwarp();
      infer16(sw, tile);
      if ((lane >> 4) == h && s < n) {
        const float* yr = tile + kTileY + (lane & 15) * 4;
        float4 o;
        o.x = destandardise(yr[0], sn, 0);
        o.y = destandardise(yr[1], sn, 1);
        o.z = destandardise(yr[2], sn, 2);
        o.w = destandardise(yr[3], sn, 3);
        reinterpret_cast<float4*>(Y)[s] = o;
      }
      __syncwarp();
    }
  }
}

// ---- training on the tensor cores -------------------------------------------------------------
// Forward and backward of the loss L = (1/n) sum_s sum_o (y_so - t'_so)^2 (targets standardised
// like the outputs) as tile contractions: mma.sync m16n8k16 with BF16 operands and FP32
// accumulation.  A warp takes 16 samples: the layer products [16 x K] x [K x N] run with the
// activations (and, backwards, the pre-activation gradients) as the A operand, rounded to BF16,
// and the BF16 weights as the B operand from shared memory; a layer's FP32 accumulators, after
// GELU and rounding, are the next layer's A fragments register for register.  The operands of
// the weight gradients (the layer inputs with a column of ones appended for the bias, and the
// pre-activation gradients, both BF16) go to global memory feature-major; a second kernel forms
// dL/dW = D^T [A | 1] per chunk of 128 samples on the tensor cores, and a third sums the chunks
// in a fixed order (deterministic).
constexpr int kTrainThreads = 128;  // 4 warps, 16 samples each per pass
constexpr int kChunk = 128;         // samples per weight-gradient partial
// rows of the feature-major operand arrays: layer input + ones row, padded to whole n-tiles
constexpr int kR0 = 48, kR1 = 72, kRD3 = 16;  // A0t rows (39 + 1 + pad), A1t/A2t rows, D3t rows
// shared layouts of the weights (BF16, row strides that spread a fragment's 8 rows over banks)
constexpr int kSW1 = 56, kSW2 = 72, kSW3 = 72, kSW3T = 24;

struct TrainWork {
  __nv_bfloat16 *A0t, *A1t, *A2t, *D1t, *D2t, *D3t;  // feature-major [rows][np]
  float* part;                                      // weight-gradient partials [nchunk][kNP]
  float* tile_loss;                                 // [np / 16]
  int np;
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__global__ void __launch_bounds__(kTrainThreads) k_mlp_train(
    const __nv_bfloat16* __restrict__ w, const float* __restrict__ norm,
    const float* __restrict__ X, const float* __restrict__ T, int n, TrainWork wk) {
  __shared__ __align__(16) __nv_bfloat16 sW1[kH * kSW1];
  __shared__ __align__(16) __nv_bfloat16 sW2[kH * kSW2];
  __shared__ __align__(16) __nv_bfloat16 sW2t[kH * kSW2];
  __shared__ __align__(16) __nv_bfloat16 sW3[8 * kSW3];
  __shared__ __align__(16) __nv_bfloat16 sW3t[kH * kSW3T];
  __shared__ float sb[2 * kH + kOut];
  __shared__ float sn[2 * kIn + 2 * kOut];
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int q = threadIdx.x; q < kH * kSW1; q += blockDim.x) {
    const int o = q / kSW1, i = q % kSW1;
    sW1[q] = i < kIn ? w[kW1 + o * kIn + i] : zero;
  }
  for (int q = threadIdx.x; q < kH * kSW2; q += blockDim.x) {
    const int o = q / kSW2, i = q % kSW2;
    sW2[q] = i < kH ? w[kW2 + o * kH + i] : zero;   // [o][j]
    sW2t[q] = i < kH ? w[kW2 + i * kH + o] : zero;  // [j][o]
  }
  for (int q = threadIdx.x; q < 8 * kSW3; q += blockDim.x) {
    const int o = q / kSW3, j = q % kSW3;
    sW3[q] = (o < kOut && j < kH) ? w[kW3 + o * kH + j] : zero;
  }
  for (int q = threadIdx.x; q < kH * kSW3T; q += blockDim.x) {
    const int j = q / kSW3T, o = q % kSW3T;
    sW3t[q] = o < kOut ? w[kW3 + o * kH + j] : zero;
  }
  for (int q = threadIdx.x; q < kH; q += blockDim.x) {
    sb[q] = __bfloat162float(w[kB1 + q]);
    sb[kH + q] = __bfloat162float(w[kB2 + q]);
  }
  if (threadIdx.x < kOut) sb[2 * kH + threadIdx.x] = __bfloat162float(w[kB3 + threadIdx.x]);
  for (int q = threadIdx.x; q < 2 * kIn + 2 * kOut; q += blockDim.x) sn[q] = norm[q];
  __syncthreads();

  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const int np = wk.np;
  const int ntiles = np / 16;
  const float inv_n = 1.f / n;
  for (int tile = blockIdx.x * (kTrainThreads / 32) + (threadIdx.x >> 5); tile < ntiles;
       tile += gridDim.x * (kTrainThreads / 32)) {
    const int s0 = tile * 16;
    const int sa = s0 + gq, sb8 = s0 + gq + 8;  // the two samples (rows) this lane holds
    const bool va = sa < n, vb = sb8 < n;
    auto put = [&](__nv_bfloat16* At, int row, int s, float v) {
      At[(size_t)row * np + s] = __float2bfloat16_rn(v);
    };
    // ---- layer 1: x' (standardised, BF16) x W1^T + b1 ----
    uint32_t A0[3][4];
#pragma unroll
    for (int kt = 0; kt < 3; ++kt) {
      float v[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const int col = 16 * kt + 2 * tq + (h & 1) + ((h & 4) ? 8 : 0);
        const int s = (h & 2) ? sb8 : sa;
        const bool ok = ((h & 2) ? vb : va) && col < kIn;
        v[h] = ok ? (X[(size_t)s * kIn + col] - sn[col]) * sn[kIn + col] : 0.f;
        // the weight-gradient operand: x' rows, and the ones row for the bias
        const float out = col < kIn ? v[h] : (col == kIn && ((h & 2) ? vb : va) ? 1.f : 0.f);
        put(wk.A0t, col, s, out);
      }
      A0[kt][0] = pack2(v[0], v[1]);
      A0[kt][1] = pack2(v[2], v[3]);
      A0[kt][2] = pack2(v[4], v[5]);
      A0[kt][3] = pack2(v[6], v[7]);
    }
    float acc[8][4];
    float gg1[8][4];
    uint32_t A1[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
      for (int kt = 0; kt < 3; ++kt) {
        const __nv_bfloat16* bp = sW1 + (nt * 8 + gq) * kSW1 + 16 * kt + 2 * tq;
        mma16816(acc[nt], A0[kt], ld32(bp), ld32(bp + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int col = nt * 8 + 2 * tq + (r & 1);
        const float z = acc[nt][r] + sb[col];
        a[r] = gelu(z);
        gg1[nt][r] = gelu_grad(z);
        const bool ok = (r & 2) ? vb : va;
        if (!ok) a[r] = 0.f;
        put(wk.A1t, col, (r & 2) ? sb8 : sa, a[r]);
      }
      const int kt = nt >> 1, hi = nt & 1;
      A1[kt][hi ? 2 : 0] = pack2(a[0], a[1]);
      A1[kt][hi ? 3 : 1] = pack2(a[2], a[3]);
    }
    if (tq == 0) {
      put(wk.A1t, kH, sa, va ? 1.f : 0.f);
      put(wk.A1t, kH, sb8, vb ? 1.f : 0.f);
    }
    // ---- layer 2 ----
    float gg2[8][4];
    uint32_t A2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const __nv_bfloat16* bp = sW2 + (nt * 8 + gq) * kSW2 + 16 * kt + 2 * tq;
        mma16816(acc[nt], A1[kt], ld32(bp), ld32(bp + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int col = nt * 8 + 2 * tq + (r & 1);
        const float z = acc[nt][r] + sb[kH + col];
        a[r] = gelu(z);
        gg2[nt][r] = gelu_grad(z);
        const bool ok = (r & 2) ? vb : va;
        if (!ok) a[r] = 0.f;
        put(wk.A2t, col, (r & 2) ? sb8 : sa, a[r]);
      }
      const int kt = nt >> 1, hi = nt & 1;
      A2[kt][hi ? 2 : 0] = pack2(a[0], a[1]);
      A2[kt][hi ? 3 : 1] = pack2(a[2], a[3]);
    }
    if (tq == 0) {
      put(wk.A2t, kH, sa, va ? 1.f : 0.f);
      put(wk.A2t, kH, sb8, vb ? 1.f : 0.f);
    }
    // ---- output layer and the loss gradient d3 = 2 (y' - t') / n ----
    float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      const __nv_bfloat16* bp = sW3 + gq * kSW3 + 16 * kt + 2 * tq;
      mma16816(y, A2[kt], ld32(bp), ld32(bp + 8));
    }
    float d3[4], lsum = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int o = 2 * tq + (r & 1);
      const int s = (r & 2) ? sb8 : sa;
      const bool ok = o < kOut && ((r & 2) ? vb : va);
      float e = 0.f;
      if (ok) {
        const float tt = (T[(size_t)s * kOut + o] - sn[2 * kIn + o]) / sn[2 * kIn + kOut + o];
        e = y[r] + sb[2 * kH + o] - tt;
      }
      lsum += e * e;
      d3[r] = 2.f * e * inv_n;
      if (o < kRD3) put(wk.D3t, o, s, d3[r]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0) wk.tile_loss[tile] = lsum * inv_n;
    // ---- backward: dA2 = d3 W3, d2 = dA2 gelu'(z2) ----
    uint32_t D3f[4] = {pack2(d3[0], d3[1]), pack2(d3[2], d3[3]), 0u, 0u};
    uint32_t D2f[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
      const __nv_bfloat16* bp = sW3t + (nt * 8 + gq) * kSW3T + 2 * tq;
      mma16816(acc[nt], D3f, ld32(bp), ld32(bp + 8));
      float d[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        d[r] = acc[nt][r] * gg2[nt][r];
        put(wk.D2t, nt * 8 + 2 * tq + (r & 1), (r & 2) ? sb8 : sa, d[r]);
      }
      const int kt = nt >> 1, hi = nt & 1;
      D2f[kt][hi ? 2 : 0] = pack2(d[0], d[1]);
      D2f[kt][hi ? 3 : 1] = pack2(d[2], d[3]);
    }
    // ---- dA1 = d2 W2, d1 = dA1 gelu'(z1) ----
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const __nv_bfloat16* bp = sW2t + (nt * 8 + gq) * kSW2 + 16 * kt + 2 * tq;
        mma16816(acc[nt], D2f[kt], ld32(bp), ld32(bp + 8));
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        put(wk.D1t, nt * 8 + 2 * tq + (r & 1), (r & 2) ? sb8 : sa, acc[nt][r] * gg1[nt][r]);
    }
  }
}

// Weight-gradient partials of one chunk of kChunk samples: P[chunk][layer params] = D^T [A | 1]
// over the chunk, M = the layer's outputs (warp w: rows 16 w .. 16 w + 15), N = its inputs and
// the ones row, K = the samples; A fragments from D (feature-major: a pair of samples is one
// 32-bit load), B fragments from [A | 1] (the same).
__global__ void __launch_bounds__(kTrainThreads) k_mlp_wgrad_mma(TrainWork wk) {
  const int chunk = blockIdx.x, layer = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const __nv_bfloat16 *D, *A;
  int mrows, nin, woff, boff;
  if (layer == 0) { D = wk.D1t; A = wk.A0t; mrows = kH; nin = kIn; woff = kW1; boff = kB1; }
  else if (layer == 1) { D = wk.D2t; A = wk.A1t; mrows = kH; nin = kH; woff = kW2; boff = kB2; }
  else { D = wk.D3t; A = wk.A2t; mrows = kOut; nin = kH; woff = kW3; boff = kB3; }
  if (16 * warp >= mrows) return;
  const int ntn = (nin + 1 + 7) / 8;  // n-tiles: inputs and the ones row
  const size_t np = wk.np;
  const int s0 = chunk * kChunk;
  float acc[9][4];
#pragma unroll
  for (int nt = 0; nt < 9; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
  for (int kt = 0; kt < kChunk / 16; ++kt) {
    const int s = s0 + 16 * kt + 2 * tq;
    const __nv_bfloat16* dr = D + (size_t)(16 * warp + gq) * np + s;
    const uint32_t af[4] = {ld32(dr), ld32(dr + 8 * np), ld32(dr + 8), ld32(dr + 8 * np + 8)};
#pragma unroll
    for (int nt = 0; nt < 9; ++nt) {
      if (nt < ntn) {
        const __nv_bfloat16* ar = A + (size_t)(nt * 8 + gq) * np + s;
        mma16816(acc[nt], af, ld32(ar), ld32(ar + 8));
      }
    }
  }
  float* P = wk.part + (size_t)chunk * kNP;
#pragma unroll
  for (int nt = 0; nt < 9; ++nt) {
    if (nt >= ntn) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int o = 16 * warp + gq + ((r & 2) ? 8 : 0);
      const int i = nt * 8 + 2 * tq + (r & 1);
      if (o >= mrows) continue;
      if (i < nin) P[woff + o * nin + i] = acc[nt][r];
      else if (i == nin) P[boff + o] = acc[nt][r];
    }
  }
}

// grad[q] = sum of the chunks' partials in chunk order; the loss from the tiles' partial losses
// in tile order.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nchunk,
                             const float* __restrict__ tile_loss, int ntiles,
                             float* __restrict__ grad, float* __restrict__ loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < kNP) {
    float acc = 0.f;
    for (int c = 0; c < nchunk; ++c) acc += part[(size_t)c * kNP + q];
    grad[q] = acc;
  }
  if (q == 0) {
    float l = 0.f;
    for (int t = 0; t < ntiles; ++t) l += tile_loss[t];
    *loss = l;
  }
}

__global__ void k_mlp_adam(float* __restrict__ wm, __nv_bfloat16* __restrict__ wb,
                           const float* __restrict__ grad, float* __restrict__ m1,
                           float* __restrict__ m2, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kNP) return;
  const float g = grad[q];
  const float a = b1 * m1[q] + (1.f - b1) * g;
  const float b = b2 * m2[q] + (1.f - b2) * g * g;
  m1[q] = a;
  m2[q] = b;
  const float w = wm[q] - lr * (a / c1) / (sqrtf(b / c2) + eps);
  wm[q] = w;
  wb[q] = __float2bfloat16_rn(w);
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = __float2bfloat16_rn(in[q]);
}

}  // namespace

struct mm_mlp {
  cudaStream_t stream = nullptr;
  float* wm = nullptr;            // FP32 master weights
  __nv_bfloat16* wb = nullptr;    // BF16 weights used by the kernels
  float* norm = nullptr;          // [x mean (kIn), x 1/std (kIn), y mean (kOut), y std (kOut)]
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad = nullptr;
  float* loss = nullptr;
  float* work = nullptr;          // activations / gradients of the current batch
  int work_n = 0;
  long long t = 0;                // Adam step counter
  std::string last_error;
};

namespace {
mm_status mfail(mm_mlp* m, cudaError_t e, const char* what) {
  if (m) m->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return MM_ERR_CUDA;
}
// Bytes of the training work buffer for n samples (padded to whole chunks): the feature-major
// BF16 operands, the chunk partials and the tile losses.
size_t work_bytes(int np) {
  const size_t rows = (size_t)kR0 + 2 * kR1 + 2 * kH + kRD3;
  return rows * np * sizeof(__nv_bfloat16) + (size_t)(np / kChunk) * kNP * sizeof(float) +
         (size_t)(np / 16) * sizeof(float);
}
mm_status ensure_work(mm_mlp* m, int n) {
  const int np = (n + kChunk - 1) / kChunk * kChunk;
  if (np <= m->work_n) return MM_OK;
  cudaFree(m->work);
  m->work = nullptr;
  cudaError_t e = cudaMalloc(&m->work, work_bytes(np));
  if (e != cudaSuccess) return mfail(m, e, "mlp work buffer");
  m->work_n = np;
  return MM_OK;
}
TrainWork carve_work(mm_mlp* m, int np) {
  TrainWork wk;
  __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(m->work);
  wk.A0t = b;
  wk.A1t = wk.A0t + (size_t)kR0 * np;
  wk.A2t = wk.A1t + (size_t)kR1 * np;
  wk.D1t = wk.A2t + (size_t)kR1 * np;
  wk.D2t = wk.D1t + (size_t)kH * np;
  wk.D3t = wk.D2t + (size_t)kH * np;
  wk.part = reinterpret_cast<float*>(wk.D3t + (size_t)kRD3 * np);
  wk.tile_loss = wk.part + (size_t)(np / kChunk) * kNP;
  wk.np = np;
  return wk;
}
}  // namespace

namespace mmk {
void mlp_device_params(const mm_mlp* m, const __nv_bfloat16** w, const float** norm) {
  *w = m->wb;
  *norm = m->norm;
}

void mlp_forward_async(const mm_mlp* m, const float* X, float* Y, int n, cudaStream_t s) {
  if (n <= 0) return;
  const int blocks = std::min((n + kInferThreads - 1) / kInferThreads, 152 * 8);
  cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)infer_smem_bytes());
  k_mlp_infer<<<blocks, kInferThreads, infer_smem_bytes(), s>>>(m->wb, m->norm, X, Y, n);
}
}  // namespace mmk

extern "C" {

mm_status mm_mlp_create(void* cuda_stream, mm_mlp** out) {
  if (!out) return MM_ERR_INVALID_ARG;
  mm_mlp* m = new mm_mlp();
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMalloc(&m->wm, kNP * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->wb, kNP * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->norm, (2 * kIn + 2 * kOut) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->m1, kNP * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->m2, kNP * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, kNP * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, kNP * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, kNP * sizeof(float));
  if (e != cudaSuccess) {
    mm_mlp_destroy(m);
    return MM_ERR_OOM;
  }
  *out = m;
  return MM_OK;
}

mm_status mm_mlp_set_params(mm_mlp* m, const float* params_host, const float* norm_host) {
  if (!m || !params_host || !norm_host) return MM_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(m->wm, params_host, kNP * sizeof(float), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->norm, norm_host, (2 * kIn + 2 * kOut) * sizeof(float),
                        cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) k_to_bf16<<<(kNP + 255) / 256, 256, 0, m->stream>>>(m->wm, m->wb, kNP);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, kNP * sizeof(float), m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, kNP * sizeof(float), m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  m->t = 0;
  return e == cudaSuccess ? MM_OK : mfail(m, e, "set params");
}

mm_status mm_mlp_get_params(mm_mlp* m, float* params_host, float* params_bf16_as_f32_host) {
  if (!m) return MM_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (params_host)
    e = cudaMemcpyAsync(params_host, m->wm, kNP * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
  std::vector<__nv_bfloat16> tmp(kNP);
  if (e == cudaSuccess && params_bf16_as_f32_host)
    e = cudaMemcpyAsync(tmp.data(), m->wb, kNP * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, e, "get params");
  if (params_bf16_as_f32_host)
    for (int q = 0; q < kNP; ++q) params_bf16_as_f32_host[q] = __bfloat162float(tmp[q]);
  return MM_OK;
}

mm_status mm_mlp_forward(mm_mlp* m, const float* X_dev, float* Y_dev, int n) {
  if (!m || !X_dev || !Y_dev || n < 0) return MM_ERR_INVALID_ARG;
  if (n == 0) return MM_OK;
  const int blocks = std::min((n + kInferThreads - 1) / kInferThreads, 152 * 8);
  cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)infer_smem_bytes());
  k_mlp_infer<<<blocks, kInferThreads, infer_smem_bytes(), m->stream>>>(m->wb, m->norm, X_dev,
                                                                        Y_dev, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MM_OK : mfail(m, e, "mlp forward");
}

mm_status mm_mlp_grad(mm_mlp* m, const float* X_dev, const float* T_dev, int n, float* grad_host,
                      float* loss_host) {
  if (!m || !X_dev || !T_dev || n < 1) return MM_ERR_INVALID_ARG;
  mm_status st = ensure_work(m, n);
  if (st != MM_OK) return st;
  const int np = (n + kChunk - 1) / kChunk * kChunk;
  const TrainWork wk = carve_work(m, np);
  // the padding rows and samples of the operands must read as zeros
  cudaError_t e = cudaMemsetAsync(m->work, 0, work_bytes(np), m->stream);
  const int ntiles = np / 16;
  const int blocks = std::min((ntiles + 3) / 4, 152 * 4);
  k_mlp_train<<<blocks, kTrainThreads, 0, m->stream>>>(m->wb, m->norm, X_dev, T_dev, n, wk);
  k_mlp_wgrad_mma<<<dim3(np / kChunk, 3), kTrainThreads, 0, m->stream>>>(wk);
  k_mlp_reduce<<<(kNP + 127) / 128, 128, 0, m->stream>>>(wk.part, np / kChunk, wk.tile_loss,
                                                         ntiles, m->grad, m->loss);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, m->grad, kNP * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && loss_host)
    e = cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && (grad_host || loss_host)) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? MM_OK : mfail(m, e, "mlp grad");
}

mm_status mm_mlp_train_step(mm_mlp* m, const float* X_dev, const float* T_dev, int n, float lr,
                            float* loss_host) {
  mm_status st = mm_mlp_grad(m, X_dev, T_dev, n, nullptr, nullptr);
  if (st != MM_OK) return st;
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)m->t), c2 = 1.f - std::pow(b2, (float)m->t);
  k_mlp_adam<<<(kNP + 255) / 256, 256, 0, m->stream>>>(m->wm, m->wb, m->grad, m->m1, m->m2, lr,
                                                       b1, b2, 1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss_host) {
    e = cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  }
  return e == cudaSuccess ? MM_OK : mfail(m, e, "mlp train step");
}

const char* mm_mlp_last_error(const mm_mlp* m) { return m ? m->last_error.c_str() : "null mlp"; }

void mm_mlp_destroy(mm_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  cudaFree(m->wm);
  cudaFree(m->wb);
  cudaFree(m->norm);
  cudaFree(m->m1);
  cudaFree(m->m2);
  cudaFree(m->grad);
  cudaFree(m->loss);
  cudaFree(m->work);
  delete m;
}

}  // extern "C"
