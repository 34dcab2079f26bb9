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

// Inference layout in shared memory: W1 rows padded to 40 inputs, W3 transposed to [kH][4], so
// that every weight load is a 16-byte vector load.
constexpr int kInP = 40;
constexpr int kIW1 = 0, kIB1 = kIW1 + kH * kInP, kIW2 = kIB1 + kH, kIB2 = kIW2 + kH * kH,
              kIW3 = kIB2 + kH, kIB3 = kIW3 + kH * kOut, kINP = kIB3 + kOut;
static_assert(kInP % 4 == 0 && kIn < kInP && kOut == 4, "inference layout");
static_assert(kIB1 % 4 == 0 && kIW2 % 4 == 0 && kIW3 % 4 == 0 && kIB3 % 4 == 0, "alignment");
constexpr int kInferThreads = 128;

__device__ __forceinline__ void stage_infer(const __nv_bfloat16* __restrict__ w,
                                            const float* __restrict__ norm, float* sw,
                                            float* sn) {
  for (int q = threadIdx.x; q < kH * kInP; q += blockDim.x) {
    const int o = q / kInP, i = q % kInP;
    sw[kIW1 + q] = i < kIn ? __bfloat162float(w[kW1 + o * kIn + i]) : 0.f;
  }
  for (int q = threadIdx.x; q < kH; q += blockDim.x) {
    sw[kIB1 + q] = __bfloat162float(w[kB1 + q]);
    sw[kIB2 + q] = __bfloat162float(w[kB2 + q]);
    for (int o = 0; o < kOut; ++o) sw[kIW3 + q * kOut + o] = __bfloat162float(w[kW3 + o * kH + q]);
  }
  for (int q = threadIdx.x; q < kH * kH; q += blockDim.x) sw[kIW2 + q] = __bfloat162float(w[kW2 + q]);
  for (int q = threadIdx.x; q < kOut; q += blockDim.x) sw[kIB3 + q] = __bfloat162float(w[kB3 + q]);
  for (int q = threadIdx.x; q < 2 * kIn + 2 * kOut; q += blockDim.x) sn[q] = norm[q];
  __syncthreads();
}

// Inference of one sample from its standardised inputs: standardised output y (layer 2 is folded
// into layer 3 so that only the first hidden layer is held in registers).  The products are
// accumulated in the order of the inputs, as in the training kernels.
__device__ __forceinline__ void infer1(const float* sw, const float xn[kInP], float y[kOut]) {
  const float4* W1 = reinterpret_cast<const float4*>(sw + kIW1);
  const float4* W2 = reinterpret_cast<const float4*>(sw + kIW2);
  const float4* W3 = reinterpret_cast<const float4*>(sw + kIW3);
  float a1[kH];  // fully unrolled loops keep a1 in registers
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float acc = sw[kIB1 + o];
#pragma unroll
    for (int q = 0; q < kInP / 4; ++q) {
      const float4 wv = W1[o * (kInP / 4) + q];
      acc = fmaf(wv.x, xn[4 * q], acc);
      acc = fmaf(wv.y, xn[4 * q + 1], acc);
      acc = fmaf(wv.z, xn[4 * q + 2], acc);
      acc = fmaf(wv.w, xn[4 * q + 3], acc);
    }
    a1[o] = gelu(acc);
  }
  y[0] = sw[kIB3];
  y[1] = sw[kIB3 + 1];
  y[2] = sw[kIB3 + 2];
  y[3] = sw[kIB3 + 3];
  for (int o2 = 0; o2 < kH; ++o2) {
    float acc = sw[kIB2 + o2];
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 wv = W2[o2 * (kH / 4) + q];
      acc = fmaf(wv.x, a1[4 * q], acc);
      acc = fmaf(wv.y, a1[4 * q + 1], acc);
      acc = fmaf(wv.z, a1[4 * q + 2], acc);
      acc = fmaf(wv.w, a1[4 * q + 3], acc);
    }
    const float a2 = gelu(acc);
    const float4 w3 = W3[o2];
    y[0] = fmaf(w3.x, a2, y[0]);
    y[1] = fmaf(w3.y, a2, y[1]);
    y[2] = fmaf(w3.z, a2, y[2]);
    y[3] = fmaf(w3.w, a2, y[3]);
  }
}


// Network output from a standardised output: y std + mean (one rounding).
__device__ __forceinline__ float destandardise(float ys, const float* sn, int o) {
  return fmaf(ys, sn[2 * kIn + kOut + o], sn[2 * kIn + o]);
}

}  // namespace mlp_body
}  // namespace mmk
