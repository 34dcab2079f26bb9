// Device code of the closure network shared by the network kernels (mm_mlp.cu) and the fused
// prediction kernel of the hybrid step (mm_closure.cu): sizes, parameter layouts, GELU, the
// shared-memory staging of the BF16 weights and the inference of one sample.
#pragma once

#include <cuda_bf16.h>

#include "mm_internal.cuh"

namespace mmk {
namespace mlp_body {

constexpr int kIn = MM_MLP_IN, kH = MM_MLP_HIDDEN, kOut = MM_MLP_OUT;
// parameter offsets in the flat vector [W1 (kH x kIn), b1, W2 (kH x kH), b2, W3 (kOut x kH), b3]
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH,
              kW3 = kB2 + kH, kB3 = kW3 + kOut * kH, kNP = kB3 + kOut;
static_assert(kNP == MM_MLP_NPARAM, "parameter count");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143267794f * __expf(-0.5f * z * z);
}

// Stage the BF16 weights (as FP32) and the normalisation constants in shared memory.
__device__ __forceinline__ void stage(const __nv_bfloat16* __restrict__ w, const float* __restrict__ norm,
                                      float* sw, float* sn) {
  for (int q = threadIdx.x; q < kNP; q += blockDim.x) sw[q] = __bfloat162float(w[q]);
  for (int q = threadIdx.x; q < 2 * kIn + 2 * kOut; q += blockDim.x) sn[q] = norm[q];
  __syncthreads();
}

// Inference on the tensor cores, 16 samples per warp.  Each layer is a [16 x K] x [K x 64] product
// by mma.sync m16n8k8 TF32 with FP32 accumulation.  The BF16 weights are exact in TF32; each
// activation a is split into two TF32 terms hi = tf32(a), lo = tf32(a - hi), and both are
// multiplied, so the products keep FP32 accuracy (relative 2^-22) while the tensor cores do the
// work.  Shared layout of the staged weights (FP32 values): W1 rows padded to 44 inputs, W2 rows
// padded to 68, W3 transposed [kH][4]; these strides put the 8 rows a fragment reads in
// distinct banks.
constexpr int kS1 = 44, kS2 = 68;
constexpr int kIW1 = 0, kIB1 = kIW1 + kH * kS1, kIW2 = kIB1 + kH, kIB2 = kIW2 + kH * kS2,
              kIW3 = kIB2 + kH, kIB3 = kIW3 + kH * kOut, kINP = kIB3 + kOut;
static_assert(kIn < 40 && kS1 >= 40 && kOut == 4 && kH == 64, "inference layout");
static_assert(kIB1 % 4 == 0 && kIW2 % 4 == 0 && kIW3 % 4 == 0 && kIB3 % 4 == 0, "alignment");
constexpr int kInferThreads = 128;
// per-warp scratch: inputs [16][kS1] and hidden activations [16][kS2] in the same place (a layer
// reads all its input fragments before it writes), outputs [16][4]
constexpr int kTileX = 0, kTileA = 0, kTileY = 16 * kS2, kTile = kTileY + 64;
constexpr int kNormF = 2 * kIn + 2 * kOut;
// dynamic shared memory of an inference CTA: weights, normalisation, one tile per warp
constexpr size_t infer_smem_bytes() {
  return sizeof(float) * ((size_t)kINP + 88 + (size_t)(kInferThreads / 32) * kTile);
}
static_assert(kNormF <= 88, "normalisation slot");

__device__ __forceinline__ void stage_infer(const __nv_bfloat16* __restrict__ w,
                                            const float* __restrict__ norm, float* sw,
                                            float* sn) {
  for (int q = threadIdx.x; q < kH * kS1; q += blockDim.x) {
    const int o = q / kS1, i = q % kS1;
    sw[kIW1 + q] = i < kIn ? __bfloat162float(w[kW1 + o * kIn + i]) : 0.f;
  }
  for (int q = threadIdx.x; q < kH * kS2; q += blockDim.x) {
    const int o = q / kS2, i = q % kS2;
    sw[kIW2 + q] = i < kH ? __bfloat162float(w[kW2 + o * kH + i]) : 0.f;
  }
  for (int q = threadIdx.x; q < kH; q += blockDim.x) {
    sw[kIB1 + q] = __bfloat162float(w[kB1 + q]);
    sw[kIB2 + q] = __bfloat162float(w[kB2 + q]);
    for (int o = 0; o < kOut; ++o) sw[kIW3 + q * kOut + o] = __bfloat162float(w[kW3 + o * kH + q]);
  }
  for (int q = threadIdx.x; q < kOut; q += blockDim.x) sw[kIB3 + q] = __bfloat162float(w[kB3 + q]);
  for (int q = threadIdx.x; q < kNormF; q += blockDim.x) sn[q] = norm[q];
  __syncthreads();
}

__device__ __forceinline__ unsigned tf32_of(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

// D += A B for one m16n8k8 tile: A row-major 16 x 8 (four TF32 registers per lane), B 8 x 8
// (two registers), D 16 x 8 FP32 (four registers).
__device__ __forceinline__ void mma_tf32(float d[4], const unsigned a[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One hidden layer for the 16 rows of a warp tile: out[16][64] = gelu(in[16][K] W^T + b), W rows
// of stride SW.  Fragment layout of m16n8k8 (lane = 4 group + t): A holds (row group, col t),
// (row group + 8, col t), (row group, col t + 4), (row group + 8, col t + 4); B holds (k t, n group)
// and (k t + 4, n group); D holds (row group, cols 2t, 2t + 1) and (row group + 8, same cols).
// The k slices are the outer loop with the eight 16 x 8 output tiles accumulating in registers,
// so in may alias out: every input is read before any output is written.
template <int K, int SIN, int SW>
__device__ __forceinline__ void hidden16(const float* in, const float* W, const float* bias,
                                         float* out) {
  const int lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  float d[kH / 8][4];
#pragma unroll
  for (int nt = 0; nt < kH / 8; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < K / 8; ++ks) {
    const int c = ks * 8 + t;
    unsigned ah[4], al[4];
    split_tf32(in[gq * SIN + c], ah[0], al[0]);
    split_tf32(in[(gq + 8) * SIN + c], ah[1], al[1]);
    split_tf32(in[gq * SIN + c + 4], ah[2], al[2]);
    split_tf32(in[(gq + 8) * SIN + c + 4], ah[3], al[3]);
#pragma unroll
    for (int nt = 0; nt < kH / 8; ++nt) {
      const float* Wr = W + (nt * 8 + gq) * SW + c;
      const unsigned b0 = __float_as_uint(Wr[0]);
      const unsigned b1 = __float_as_uint(Wr[4]);
      mma_tf32(d[nt], ah, b0, b1);
      mma_tf32(d[nt], al, b0, b1);
    }
  }
  __syncwarp();
#pragma unroll
  for (int nt = 0; nt < kH / 8; ++nt) {
    const int col = nt * 8 + 2 * t;
    out[gq * kS2 + col] = gelu(d[nt][0] + bias[col]);
    out[gq * kS2 + col + 1] = gelu(d[nt][1] + bias[col + 1]);
    out[(gq + 8) * kS2 + col] = gelu(d[nt][2] + bias[col]);
    out[(gq + 8) * kS2 + col + 1] = gelu(d[nt][3] + bias[col + 1]);
  }
}

// The network for the 16 rows of a warp tile: tile + kTileX holds standardised inputs (columns
// kIn .. kS1 - 1 zero), tile + kTileY receives the standardised outputs [16][4].
__device__ __forceinline__ void infer16(const float* sw, float* tile) {
  float* X = tile + kTileX;
  float* A = tile + kTileA;
  float* Y = tile + kTileY;
  hidden16<40, kS1, kS1>(X, sw + kIW1, sw + kIB1, A);
  __syncwarp();
  hidden16<kH, kS2, kS2>(A, sw + kIW2, sw + kIB2, A);
  __syncwarp();
  const int lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  float d[4] = {0.f, 0.f, 0.f, 0.f};
  const float* W3 = sw + kIW3;  // [kH][4]: the output index is the column n = group (< 4)
#pragma unroll
  for (int ks = 0; ks < kH / 8; ++ks) {
    const int c = ks * 8 + t;
    unsigned ah[4], al[4];
    split_tf32(A[gq * kS2 + c], ah[0], al[0]);
    split_tf32(A[(gq + 8) * kS2 + c], ah[1], al[1]);
    split_tf32(A[gq * kS2 + c + 4], ah[2], al[2]);
    split_tf32(A[(gq + 8) * kS2 + c + 4], ah[3], al[3]);
    const unsigned b0 = gq < kOut ? __float_as_uint(W3[c * kOut + gq]) : 0u;
    const unsigned b1 = gq < kOut ? __float_as_uint(W3[(c + 4) * kOut + gq]) : 0u;
    mma_tf32(d, ah, b0, b1);
    mma_tf32(d, al, b0, b1);
  }
  if (t < 2) {
    const int col = 2 * t;
    Y[gq * 4 + col] = d[0] + sw[kIB3 + col];
    Y[gq * 4 + col + 1] = d[1] + sw[kIB3 + col + 1];
    Y[(gq + 8) * 4 + col] = d[2] + sw[kIB3 + col];
    Y[(gq + 8) * 4 + col + 1] = d[3] + sw[kIB3 + col + 1];
  }
  __syncwarp();
}

// Standardised inputs of one sample into its tile row (the padding columns zeroed).
__device__ __forceinline__ void put_row(float* tile, int row, const float* x, const float* sn) {
  float* X = tile + kTileX + row * kS1;
#pragma unroll
  for (int i = 0; i < kIn; ++i) X[i] = (x[i] - sn[i]) * sn[kIn + i];
#pragma unroll
  for (int i = kIn; i < kS1; ++i) X[i] = 0.f;
}

// Network output from a standardised output: y std + mean (one rounding).
__device__ __forceinline__ float destandardise(float ys, const float* sn, int o) {
  return fmaf(ys, sn[2 * kIn + kOut + o], sn[2 * kIn + o]);
}

}  // namespace mlp_body
}  // namespace mmk
