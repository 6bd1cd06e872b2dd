// Learned priority scorer: a 2-layer MLP (8 -> 64 -> 1, ReLU) with BF16
// weights and inputs and FP32 accumulation, and the per-vertex features it
// reads.  The same feature function serves trace collection and scheduling,
// so the network is trained on exactly what it sees at run time.
//
// Features of vertex j at round r (log-compressed so one network spans graph
// sizes and iteration stages):
//   sum (PageRank-style) ops                  min (SSSP)
//   f0 log1p(|Delta_j| * n)                   log1p(Delta_j) if finite, else 0
//   f1 log1p(v_j)                             log1p(v_j) if finite, else 0
//   f2 log1p(indeg_j)                         same
//   f3 log1p(outdeg_j)                        same
//   f4 log1p(r - last activation round)       same (never activated: r + 1)
//   f5 1                                      1 if Delta_j finite
//   f6 log1p(|Delta_j| * n / (outdeg_j + 1))  1 if v_j finite
//   f7 0                                      0
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "daic_ops.cuh"

namespace maiter {

constexpr int kMlpIn = 8;
constexpr int kMlpHidden = 64;
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden + 1;  // 641

// BF16 weights as the kernels read them (row-major W1[h][i]).
struct MlpWeights {
  __nv_bfloat16 w1[kMlpHidden * kMlpIn];
  __nv_bfloat16 b1[kMlpHidden];
  __nv_bfloat16 w2[kMlpHidden];
  __nv_bfloat16 b2;
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16(x)); }

template <bool kIsSum>
__device__ __forceinline__ void vertex_features(double delta, double v, bool d_finite, bool v_finite,
                                                int indeg, int outdeg, unsigned age, double n,
                                                float* f) {
  if (kIsSum) {
    const double ad = fabs(delta) * n;
    f[0] = static_cast<float>(log1p(ad));
    f[1] = static_cast<float>(log1p(fabs(v)));
    f[5] = 1.0f;
    f[6] = static_cast<float>(log1p(ad / (static_cast<double>(outdeg) + 1.0)));
  } else {
    f[0] = d_finite ? static_cast<float>(log1p(delta)) : 0.0f;
    f[1] = v_finite ? static_cast<float>(log1p(v)) : 0.0f;
    f[5] = d_finite ? 1.0f : 0.0f;
    f[6] = v_finite ? 1.0f : 0.0f;
  }
  f[2] = log1pf(static_cast<float>(indeg));
  f[3] = log1pf(static_cast<float>(outdeg));
  f[4] = log1pf(static_cast<float>(age));
  f[7] = 0.0f;
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) f[i] = bf16r(f[i]);   // BF16 inputs
}

// Forward pass for one input vector; W is typically staged in shared memory.
__device__ __forceinline__ float mlp_forward(const MlpWeights& W, const float* x, float* h_out) {
  float y = __bfloat162float(W.b2);
#pragma unroll 8
  for (int k = 0; k < kMlpHidden; ++k) {
    float acc = __bfloat162float(W.b1[k]);
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) acc = fmaf(__bfloat162float(W.w1[k * kMlpIn + i]), x[i], acc);
    const float h = acc > 0.0f ? acc : 0.0f;
    if (h_out) h_out[k] = h;
    y = fmaf(__bfloat162float(W.w2[k]), h, y);
  }
  return y;
}

// Order-preserving map of a score to a non-zero 32-bit key (0 = not pending).
__device__ __forceinline__ unsigned score_key(float s) {
  const unsigned u = __float_as_uint(s);
  const unsigned k = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return k ? k : 1u;
}

}  // namespace maiter
