// ms_mlp.cu -- the learned format selector's network: a 16 -> 64 -> 64 -> 10 MLP
// (ReLU, fp32) with hand-written forward, forward+backward (mean squared error
// over masked targets) and Adam kernels.
//
// Parameters are one packed fp32 array: W1[16][64], b1[64], W2[64][64], b2[64],
// W3[64][10], b3[10] (row-major, input index first), 5898 values in all.
// Gradients are accumulated per CTA in shared memory in a fixed order and reduced
// over CTAs in a fixed order, so training is deterministic.
#include <algorithm>

#include "ms_host.h"

namespace ms {
namespace {

constexpr int kIn = 16, kH = 64, kOut = 10;
constexpr int oW1 = 0, oB1 = oW1 + kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH * kOut, kParams = oB3 + kOut;
static_assert(kParams == MS_MLP_PARAMS, "parameter count");
constexpr int kMlpThreads = 128;

struct MlpSmem {
  float w[kParams];
  float g[kParams];  // gradient accumulator (forward+backward kernel)
  float x[kIn], h1[kH], h2[kH], out[kOut], dout[kOut], dh2[kH], dh1[kH];
  float loss;
};

// One sample's forward pass by the whole CTA (x already in s->x).
__device__ void mlp_forward_sample(MlpSmem* s, int t) {
  if (t < kH) {
    float a = s->w[oB1 + t];
#pragma unroll
    for (int i = 0; i < kIn; i++) a = fmaf(s->x[i], s->w[oW1 + i * kH + t], a);
    s->h1[t] = fmaxf(a, 0.f);
  }
  __syncthreads();
  if (t < kH) {
    float a = s->w[oB2 + t];
#pragma unroll 16
    for (int i = 0; i < kH; i++) a = fmaf(s->h1[i], s->w[oW2 + i * kH + t], a);
    s->h2[t] = fmaxf(a, 0.f);
  }
  __syncthreads();
  if (t < kOut) {
    float a = s->w[oB3 + t];
#pragma unroll 16
    for (int i = 0; i < kH; i++) a = fmaf(s->h2[i], s->w[oW3 + i * kOut + t], a);
    s->out[t] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const float* params, const float* X, uint64_t n,
                                                             float* Y) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  MlpSmem* s = reinterpret_cast<MlpSmem*>(smem_raw);
  const int t = threadIdx.x;
  for (int p = t; p < kParams; p += blockDim.x) s->w[p] = params[p];
  __syncthreads();
  for (uint64_t r = blockIdx.x; r < n; r += gridDim.x) {
    if (t < kIn) s->x[t] = X[r * kIn + t];
    __syncthreads();
    mlp_forward_sample(s, t);
    if (t < kOut) Y[r * kOut + t] = s->out[t];
    __syncthreads();
  }
}

// Samples [lo, hi) of this CTA: forward, loss 1/count * sum mask*(out-y)^2 and its
// gradient, accumulated in s->g; the partial gradient and loss go to
// partials[blockIdx.x][0 .. kParams].
__global__ void __launch_bounds__(kMlpThreads) k_mlp_grad(const float* params, const float* X, const float* Y,
                                                          const float* M, uint64_t n, float inv_count,
                                                          float* partials) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  MlpSmem* s = reinterpret_cast<MlpSmem*>(smem_raw);
  const int t = threadIdx.x;
  for (int p = t; p < kParams; p += blockDim.x) {
    s->w[p] = params[p];
    s->g[p] = 0.f;
  }
  if (t == 0) s->loss = 0.f;
  __syncthreads();
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t lo = (uint64_t)blockIdx.x * per, hi = min(n, lo + per);
  for (uint64_t r = lo; r < hi; r++) {
    if (t < kIn) s->x[t] = X[r * kIn + t];
    __syncthreads();
    mlp_forward_sample(s, t);
    if (t < kOut) {
      const float m = M[r * kOut + t];
      const float e = (s->out[t] - Y[r * kOut + t]) * m;
      s->dout[t] = 2.f * e * inv_count;
    }
    __syncthreads();
    if (t == 0) {
      float l = 0.f;
      for (int o = 0; o < kOut; o++) {
        const float e = (s->out[o] - Y[r * kOut + o]) * M[r * kOut + o];
        l = fmaf(e, e, l);
      }
      s->loss += l * inv_count;
    }
    // layer 3: dW3[i][o] += h2[i] dout[o]; db3[o] += dout[o]; dh2[i] = relu'(h2) sum_o W3[i][o] dout[o]
    for (int q = t; q < kH * kOut; q += blockDim.x) {
      const int i = q / kOut, o = q % kOut;
      s->g[oW3 + q] = fmaf(s->h2[i], s->dout[o], s->g[oW3 + q]);
    }
    if (t < kOut) s->g[oB3 + t] += s->dout[t];
    if (t < kH) {
      float a = 0.f;
#pragma unroll
      for (int o = 0; o < kOut; o++) a = fmaf(s->w[oW3 + t * kOut + o], s->dout[o], a);
      s->dh2[t] = s->h2[t] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // layer 2
    for (int q = t; q < kH * kH; q += blockDim.x) {
      const int i = q / kH, j = q % kH;
      s->g[oW2 + q] = fmaf(s->h1[i], s->dh2[j], s->g[oW2 + q]);
    }
    if (t < kH) {
      s->g[oB2 + t] += s->dh2[t];
      float a = 0.f;
#pragma unroll 16
      for (int j = 0; j < kH; j++) a = fmaf(s->w[oW2 + t * kH + j], s->dh2[j], a);
      s->dh1[t] = s->h1[t] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // layer 1
    for (int q = t; q < kIn * kH; q += blockDim.x) {
      const int i = q / kH, j = q % kH;
      s->g[oW1 + q] = fmaf(s->x[i], s->dh1[j], s->g[oW1 + q]);
    }
    if (t < kH) s->g[oB1 + t] += s->dh1[t];
    __syncthreads();
  }
  float* out = partials + (uint64_t)blockIdx.x * (kParams + 1);
  for (int p = t; p < kParams; p += blockDim.x) out[p] = s->g[p];
  if (t == 0) out[kParams] = s->loss;
}

// grad[p] = sum over CTAs (in CTA order) of the partials; loss likewise.
__global__ void k_mlp_reduce(const float* partials, int parts, float* grad, float* loss) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= kParams; p += gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int c = 0; c < parts; c++) a += partials[(uint64_t)c * (kParams + 1) + p];
    if (p < kParams) grad[p] = a;
    else *loss = a;
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
__global__ void k_mlp_adam(float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams; p += gridDim.x * blockDim.x) {
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    w[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  }
}

int mlp_grid(uint64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(n, (uint64_t)std::max(sms, 1) * 4));
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_mlp_forward(const float* d_params, const float* d_x, uint64_t n, float* d_y, void* stream) {
  MS_TRACE();
  if (!d_params || (n && (!d_x || !d_y))) return MS_ERR_INVALID_ARG;
  if (n == 0) return MS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t smem = sizeof(MlpSmem);
  if (cuda_status(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      MS_OK)
    return MS_ERR_CUDA;
  k_mlp_forward<<<mlp_grid(n), kMlpThreads, smem, s>>>(d_params, d_x, n, d_y);
  return cuda_status(cudaGetLastError());
}

ms_status ms_mlp_loss_grad(const float* d_params, const float* d_x, const float* d_y, const float* d_mask,
                           uint64_t n, float inv_count, float* d_grad, float* d_loss, float* d_partials,
                           uint64_t partials_floats, void* stream) {
  MS_TRACE();
  if (!d_params || !d_grad || !d_loss || !d_partials || (n && (!d_x || !d_y || !d_mask))) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int grid = mlp_grid(std::max<uint64_t>(n, 1));
  grid = (int)std::min<uint64_t>((uint64_t)grid, partials_floats / (kParams + 1));
  if (grid < 1) return MS_ERR_INVALID_ARG;
  const size_t smem = sizeof(MlpSmem);
  if (cuda_status(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != MS_OK)
    return MS_ERR_CUDA;
  k_mlp_grad<<<grid, kMlpThreads, smem, s>>>(d_params, d_x, d_y, d_mask, n, inv_count, d_partials);
  if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
  k_mlp_reduce<<<(kParams + 256) / 256, 256, 0, s>>>(d_partials, grid, d_grad, d_loss);
  return cuda_status(cudaGetLastError());
}

ms_status ms_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, uint64_t step, float lr,
                      float beta1, float beta2, float eps, void* stream) {
  MS_TRACE();
  if (!d_params || !d_grad || !d_m || !d_v || step == 0) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double p1 = 1.0, p2 = 1.0;
  for (uint64_t i = 0; i < step && i < 100000; i++) {
    p1 *= beta1;
    p2 *= beta2;
  }
  k_mlp_adam<<<(kParams + 255) / 256, 256, 0, s>>>(d_params, d_grad, d_m, d_v, lr, beta1, beta2, eps,
                                                   (float)(1.0 - p1), (float)(1.0 - p2));
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
