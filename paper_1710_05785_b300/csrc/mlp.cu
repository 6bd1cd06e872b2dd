// The learned scorer's network object and its GPU kernels: inference over a
// matrix of features, fused forward + backward with block-reduced FP32
// gradients, and Adam on FP32 master weights that are re-rounded to the BF16
// copy the inference path reads.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "internal.h"
#include "mlp.cuh"

struct maiter_mlp {
  int device = 0;
  float* master = nullptr;          // kMlpParams FP32: w1[64*8], b1[64], w2[64], b2
  maiter::MlpWeights* w = nullptr;  // BF16 copy read by the kernels
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;            // kMlpParams + 1 (loss)
  long long step = 0;
};

namespace maiter {

const MlpWeights* mlp_device_weights(const maiter_mlp* m) { return m ? m->w : nullptr; }
int mlp_device(const maiter_mlp* m) { return m ? m->device : -1; }

__global__ void k_mlp_round(const float* __restrict__ master, MlpWeights* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n1 = kMlpHidden * kMlpIn;
  if (i < n1) w->w1[i] = __float2bfloat16(master[i]);
  else if (i < n1 + kMlpHidden) w->b1[i - n1] = __float2bfloat16(master[i]);
  else if (i < n1 + 2 * kMlpHidden) w->w2[i - n1 - kMlpHidden] = __float2bfloat16(master[i]);
  else if (i == n1 + 2 * kMlpHidden) w->b2 = __float2bfloat16(master[i]);
}

__global__ void k_mlp_forward(const MlpWeights* __restrict__ wg, const float* __restrict__ x,
                              int64_t n, float* __restrict__ out) {
  // the scheduler's inference path: rows scored a warp (32 rows) at a time
  // on the tensor cores
  __shared__ MlpFrag W;
  __shared__ uint4 s_rows[8][32];
  __shared__ float s_out[8][32];
  stage_mlp(wg, &W);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t r0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + wid * 32; r0 < n; r0 += stride) {
    const int64_t r = r0 + lane;
    const int cnt = static_cast<int>(n - r0 < 32 ? n - r0 : 32);
    if (r < n) {
      float f[kMlpIn];
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i) f[i] = bf16r(x[r * kMlpIn + i]);
      s_rows[wid][lane] = pack_features(f);
    }
    __syncwarp();
    warp_score(W, s_rows[wid], cnt, s_out[wid]);
    __syncwarp();
    if (r < n) out[r] = s_out[wid][lane];
    __syncwarp();
  }
}

// Mean-squared-error gradient over rows idx[0..n) (or 0..n when idx is null):
// each thread runs one row forward and backward; gradients are summed per
// block in shared memory (FP32) and added to g once per block.
__global__ void __launch_bounds__(256) k_mlp_grad(const MlpWeights* __restrict__ wg,
                                                  const float* __restrict__ x,
                                                  const float* __restrict__ y,
                                                  const int* __restrict__ idx, int64_t n,
                                                  float scale, float* __restrict__ g) {
  __shared__ MlpWeights W;
  __shared__ float sg[kMlpParams + 1];
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(MlpWeights) / 2); i += blockDim.x)
    reinterpret_cast<unsigned short*>(&W)[i] = reinterpret_cast<const unsigned short*>(wg)[i];
  for (int i = threadIdx.x; i < kMlpParams + 1; i += blockDim.x) sg[i] = 0.0f;
  __syncthreads();
  constexpr int o_b1 = kMlpHidden * kMlpIn, o_w2 = o_b1 + kMlpHidden, o_b2 = o_w2 + kMlpHidden;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = idx ? idx[t] : t;
    float f[kMlpIn];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) f[i] = bf16r(x[r * kMlpIn + i]);
    float h[kMlpHidden];
    const float yh = mlp_forward(W, f, h);
    const float err = yh - y[r];
    const float dy = 2.0f * err * scale;       // d(mean squared error)/d(yh)
    atomicAdd(&sg[kMlpParams], err * err * scale);
    atomicAdd(&sg[o_b2], dy);
#pragma unroll 4
    for (int k = 0; k < kMlpHidden; ++k) {
      if (h[k] <= 0.0f) continue;            // ReLU: no gradient through inactive units
      atomicAdd(&sg[o_w2 + k], dy * h[k]);
      const float dh = dy * __bfloat162float(W.w2[k]);
      atomicAdd(&sg[o_b1 + k], dh);
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i)
        if (f[i] != 0.0f) atomicAdd(&sg[k * kMlpIn + i], dh * f[i]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpParams + 1; i += blockDim.x)
    if (sg[i] != 0.0f) atomicAdd(&g[i], sg[i]);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace maiter

using namespace maiter;

extern "C" {

void maiter_mlp_destroy(maiter_mlp* m) {
  if (!m) return;
  DeviceGuard guard(m->device);
  cudaFree(m->master);
  cudaFree(m->w);
  cudaFree(m->adam_m);
  cudaFree(m->adam_v);
  cudaFree(m->grad);
  delete m;
}

maiter_status maiter_mlp_set_params(maiter_mlp* m, const float* params) {
  set_error("%s", "");
  MAITER_REQUIRE(m && params, "NULL argument");
  DeviceGuard guard(m->device);
  MAITER_CUDA(cudaMemcpy(m->master, params, sizeof(float) * kMlpParams, cudaMemcpyDefault));
  k_mlp_round<<<(kMlpParams + 255) / 256, 256>>>(m->master, m->w);
  MAITER_CUDA(cudaGetLastError());
  MAITER_CUDA(cudaMemset(m->adam_m, 0, sizeof(float) * kMlpParams));
  MAITER_CUDA(cudaMemset(m->adam_v, 0, sizeof(float) * kMlpParams));
  MAITER_CUDA(cudaDeviceSynchronize());
  m->step = 0;
  return MAITER_OK;
}

maiter_status maiter_mlp_get_params(const maiter_mlp* m, float* params) {
  set_error("%s", "");
  MAITER_REQUIRE(m && params, "NULL argument");
  DeviceGuard guard(m->device);
  MAITER_CUDA(cudaMemcpy(params, m->master, sizeof(float) * kMlpParams, cudaMemcpyDefault));
  return MAITER_OK;
}

maiter_status maiter_mlp_create(int device, uint64_t seed, maiter_mlp** out) {
  set_error("%s", "");
  cudaGetLastError();
  MAITER_REQUIRE(out, "NULL argument");
  int ndev = 0;
  MAITER_CUDA(cudaGetDeviceCount(&ndev));
  MAITER_REQUIRE(device >= 0 && device < ndev, "device %d out of range", device);
  DeviceGuard guard(device);
  maiter_mlp* m = new (std::nothrow) maiter_mlp();
  MAITER_REQUIRE(m, "host allocation failed");
  m->device = device;
  cudaError_t e = cudaMalloc(&m->master, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->w, sizeof(MlpWeights));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * (kMlpParams + 1));
  if (e != cudaSuccess) {
    set_error("mlp allocation failed: %s", cudaGetErrorString(e));
    maiter_mlp_destroy(m);
    return MAITER_ERR_OOM;
  }
  // He-style initialisation from a seeded generator, biases zero
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> n1(0.0f, std::sqrt(2.0f / kMlpIn));
  std::normal_distribution<float> n2(0.0f, std::sqrt(1.0f / kMlpHidden));
  std::vector<float> p(kMlpParams, 0.0f);
  for (int i = 0; i < kMlpHidden * kMlpIn; ++i) p[i] = n1(rng);
  for (int k = 0; k < kMlpHidden; ++k) p[kMlpHidden * kMlpIn + kMlpHidden + k] = n2(rng);
  maiter_status s = maiter_mlp_set_params(m, p.data());
  if (s != MAITER_OK) {
    maiter_mlp_destroy(m);
    return s;
  }
  *out = m;
  return MAITER_OK;
}

maiter_status maiter_mlp_forward(const maiter_mlp* m, const float* x, int64_t n, float* out) {
  set_error("%s", "");
  cudaGetLastError();
  MAITER_REQUIRE(m && x && out && n >= 0, "bad argument");
  if (n == 0) return MAITER_OK;
  DeviceGuard guard(m->device);
  float* dx = nullptr;
  float* dout = nullptr;
  MAITER_CUDA(cudaMalloc(&dx, sizeof(float) * kMlpIn * n));
  cudaError_t e = cudaMalloc(&dout, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(float) * kMlpIn * n, cudaMemcpyDefault);
  if (e == cudaSuccess) {
    k_mlp_forward<<<static_cast<int>(std::min<int64_t>((n + 255) / 256, 4096)), 256>>>(m->w, dx, n, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(float) * n, cudaMemcpyDefault);
  cudaFree(dx);
  cudaFree(dout);
  MAITER_CUDA(e);
  return MAITER_OK;
}

maiter_status maiter_mlp_gradients(const maiter_mlp* m, const float* x, const float* y, int64_t n,
                                   float* grad, float* loss) {
  set_error("%s", "");
  cudaGetLastError();
  MAITER_REQUIRE(m && x && y && grad && n > 0, "bad argument");
  DeviceGuard guard(m->device);
  float *dx = nullptr, *dy = nullptr;
  MAITER_CUDA(cudaMalloc(&dx, sizeof(float) * kMlpIn * n));
  cudaError_t e = cudaMalloc(&dy, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(float) * kMlpIn * n, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(dy, y, sizeof(float) * n, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemset(m->grad, 0, sizeof(float) * (kMlpParams + 1));
  if (e == cudaSuccess) {
    k_mlp_grad<<<static_cast<int>(std::min<int64_t>((n + 255) / 256, 1024)), 256>>>(
        m->w, dx, dy, nullptr, n, 1.0f / static_cast<float>(n), m->grad);
    e = cudaGetLastError();
  }
  std::vector<float> h(kMlpParams + 1);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), m->grad, sizeof(float) * (kMlpParams + 1), cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dy);
  MAITER_CUDA(e);
  std::memcpy(grad, h.data(), sizeof(float) * kMlpParams);
  if (loss) *loss = h[kMlpParams];
  return MAITER_OK;
}

maiter_status maiter_mlp_train(maiter_mlp* m, const float* x, const float* y, int64_t n,
                               int32_t epochs, int32_t batch, float lr, uint64_t seed,
                               float* final_loss) {
  set_error("%s", "");
  cudaGetLastError();
  MAITER_REQUIRE(m && x && y && n > 0 && epochs > 0 && batch > 0 && lr > 0.0f, "bad argument");
  DeviceGuard guard(m->device);
  float *dx = nullptr, *dy = nullptr;
  int* didx = nullptr;
  MAITER_CUDA(cudaMalloc(&dx, sizeof(float) * kMlpIn * n));
  cudaError_t e = cudaMalloc(&dy, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&didx, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(float) * kMlpIn * n, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(dy, y, sizeof(float) * n, cudaMemcpyDefault);
  std::mt19937_64 rng(seed);
  std::vector<int> perm(n);
  const float b1 = 0.9f, b2 = 0.999f, aeps = 1e-8f;
  float last = 0.0f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int64_t i = 0; i < n; ++i) perm[i] = static_cast<int>(i);
    std::shuffle(perm.begin(), perm.end(), rng);
    e = cudaMemcpy(didx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    double ep_loss = 0.0;
    for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += batch) {
      const int64_t nb = std::min<int64_t>(batch, n - b0);
      e = cudaMemsetAsync(m->grad, 0, sizeof(float) * (kMlpParams + 1));
      k_mlp_grad<<<static_cast<int>((nb + 255) / 256), 256>>>(m->w, dx, dy, didx + b0, nb,
                                                                1.0f / static_cast<float>(nb), m->grad);
      ++m->step;
      const float c1 = 1.0f - std::pow(b1, static_cast<float>(m->step));
      const float c2 = 1.0f - std::pow(b2, static_cast<float>(m->step));
      k_adam<<<(kMlpParams + 255) / 256, 256>>>(m->master, m->grad, m->adam_m, m->adam_v, lr, b1, b2,
                                                aeps, c1, c2);
      k_mlp_round<<<(kMlpParams + 255) / 256, 256>>>(m->master, m->w);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (b0 + batch >= n && e == cudaSuccess) {
        float l = 0.0f;
        e = cudaMemcpy(&l, m->grad + kMlpParams, sizeof(float), cudaMemcpyDeviceToHost);
        ep_loss = l;
      }
    }
    last = static_cast<float>(ep_loss);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dx);
  cudaFree(dy);
  cudaFree(didx);
  MAITER_CUDA(e);
  if (final_loss) *final_loss = last;
  return MAITER_OK;
}

}  // extern "C"
