// Learned heat-flux closure: a small MLP (39 -> 64 -> 64 -> 4, GELU) with BF16 weights and FP32
// accumulation, trained and evaluated by these kernels.  The network maps local macro features
// of a cell to the dimensionless non-Navier-Stokes part of the heat-flux tensor of Eq. (5-99):
// H = H_CE + eps rho T^{3/2} y, where H_CE is the Chapman-Enskog value, i.e. the moments of the
// transport part of Ghat (Eq. 5-97) for a Gaussian: H111 = -3 eps p Tx / tau, H112 = -eps p Ty /
// tau, H122 = -eps p Tx / tau, H222 = -3 eps p Ty / tau (p = rho T).
//
// Kernels: features (one thread per cell), inference (one thread per sample, weights in shared
// memory), training forward/backward per sample (activations and pre-activation gradients kept
// in global memory), weight gradients as reductions over the batch (one thread per weight, fixed
// order: deterministic), and Adam on FP32 master weights that refreshes the BF16 copies.
#include <cuda_bf16.h>

#include <algorithm>
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

// Per-sample forward and backward of the loss L = (1/n) sum_s sum_o (y_so - t_so)^2, targets
// standardised like the outputs.  The layer inputs A0 (standardised x), A1, A2, the
// pre-activations Z1, Z2 and the pre-activation gradients D1, D2, D3 go to global memory (the
// per-sample activations do not fit in registers) for the weight-gradient reductions.
struct Work {
  float *A0, *A1, *A2, *Z1, *Z2, *D1, *D2, *D3;
};

__global__ void k_mlp_fwd_bwd(const __nv_bfloat16* __restrict__ w, const float* __restrict__ norm,
                              const float* __restrict__ X, const float* __restrict__ T, int n,
                              Work wk, float* __restrict__ loss) {
  __shared__ float sw[kNP];
  __shared__ float sn[2 * kIn + 2 * kOut];
  stage(w, norm, sw, sn);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    float* A0 = wk.A0 + (size_t)s * kIn;
    float* A1 = wk.A1 + (size_t)s * kH;
    float* A2 = wk.A2 + (size_t)s * kH;
    float* Z1 = wk.Z1 + (size_t)s * kH;
    float* Z2 = wk.Z2 + (size_t)s * kH;
    float* D1 = wk.D1 + (size_t)s * kH;
    float* D2 = wk.D2 + (size_t)s * kH;
    float* D3 = wk.D3 + (size_t)s * kOut;
    float xn[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
      xn[i] = (X[(size_t)s * kIn + i] - sn[i]) * sn[kIn + i];
      A0[i] = xn[i];
    }
    for (int o = 0; o < kH; ++o) {
      float acc = sw[kB1 + o];
#pragma unroll
      for (int i = 0; i < kIn; ++i) acc = fmaf(sw[kW1 + o * kIn + i], xn[i], acc);
      Z1[o] = acc;
      A1[o] = gelu(acc);
    }
    float y[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) y[o] = sw[kB3 + o];
    for (int o2 = 0; o2 < kH; ++o2) {
      float acc = sw[kB2 + o2];
      for (int i = 0; i < kH; ++i) acc = fmaf(sw[kW2 + o2 * kH + i], A1[i], acc);
      Z2[o2] = acc;
      const float a2 = gelu(acc);
      A2[o2] = a2;
#pragma unroll
      for (int o = 0; o < kOut; ++o) y[o] = fmaf(sw[kW3 + o * kH + o2], a2, y[o]);
    }
    float d3[kOut], l = 0.f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      const float t = (T[(size_t)s * kOut + o] - sn[2 * kIn + o]) / sn[2 * kIn + kOut + o];
      const float e = y[o] - t;
      l += e * e;
      d3[o] = 2.f * e / n;
      D3[o] = d3[o];
    }
    atomicAdd(loss, l / n);
    for (int i = 0; i < kH; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) acc = fmaf(sw[kW3 + o * kH + i], d3[o], acc);
      D2[i] = acc * gelu_grad(Z2[i]);
    }
    for (int i = 0; i < kH; ++i) {
      float acc = 0.f;
      for (int o = 0; o < kH; ++o) acc = fmaf(sw[kW2 + o * kH + i], D2[o], acc);
      D1[i] = acc * gelu_grad(Z1[i]);
    }
  }
}

// dW[o][i] = sum_s D[s][o] A[s][i], db[o] = sum_s D[s][o]; one thread per parameter, samples in
// order (deterministic).
__global__ void k_mlp_wgrad(const float* __restrict__ A0, const float* __restrict__ A1,
                            const float* __restrict__ A2, const float* __restrict__ D1,
                            const float* __restrict__ D2, const float* __restrict__ D3, int n,
                            float* __restrict__ grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kNP) return;
  const float *D, *A;
  int o, i, nin, nout;
  bool bias = false;
  if (q < kB1) { D = D1; A = A0; nin = kIn; nout = kH; o = q / kIn; i = q % kIn; }
  else if (q < kW2) { D = D1; A = A0; nin = kIn; nout = kH; o = q - kB1; i = 0; bias = true; }
  else if (q < kB2) { D = D2; A = A1; nin = kH; nout = kH; o = (q - kW2) / kH; i = (q - kW2) % kH; }
  else if (q < kW3) { D = D2; A = A1; nin = kH; nout = kH; o = q - kB2; i = 0; bias = true; }
  else if (q < kB3) { D = D3; A = A2; nin = kH; nout = kOut; o = (q - kW3) / kH; i = (q - kW3) % kH; }
  else { D = D3; A = A2; nin = kH; nout = kOut; o = q - kB3; i = 0; bias = true; }
  float acc = 0.f;
  for (int s = 0; s < n; ++s)
    acc = fmaf(D[(size_t)s * nout + o], bias ? 1.f : A[(size_t)s * nin + i], acc);
  grad[q] = acc;
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
mm_status ensure_work(mm_mlp* m, int n) {
  if (n <= m->work_n) return MM_OK;
  cudaFree(m->work);
  m->work = nullptr;
  const size_t per = (size_t)kIn + 6 * (size_t)kH + (size_t)kOut;
  cudaError_t e = cudaMalloc(&m->work, per * n * sizeof(float));
  if (e != cudaSuccess) return mfail(m, e, "mlp work buffer");
  m->work_n = n;
  return MM_OK;
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
  Work wk;
  wk.A0 = m->work;
  wk.A1 = wk.A0 + (size_t)kIn * n;
  wk.A2 = wk.A1 + (size_t)kH * n;
  wk.Z1 = wk.A2 + (size_t)kH * n;
  wk.Z2 = wk.Z1 + (size_t)kH * n;
  wk.D1 = wk.Z2 + (size_t)kH * n;
  wk.D2 = wk.D1 + (size_t)kH * n;
  wk.D3 = wk.D2 + (size_t)kH * n;
  cudaError_t e = cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
  const int blocks = std::min((n + 127) / 128, 152 * 8);
  k_mlp_fwd_bwd<<<blocks, 128, 0, m->stream>>>(m->wb, m->norm, X_dev, T_dev, n, wk, m->loss);
  k_mlp_wgrad<<<(kNP + 127) / 128, 128, 0, m->stream>>>(wk.A0, wk.A1, wk.A2, wk.D1, wk.D2,
                                                        wk.D3, n, m->grad);
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
