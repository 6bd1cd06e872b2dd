// Learned priority scorer: a 2-layer MLP (8 -> 64 -> 1, ReLU) with BF16
// weights and inputs and FP32 accumulation, and the per-vertex features it
// reads.  The same feature function serves trace collection and scheduling,
// so the network is trained on exactly what it sees at run time.
//
// Features of vertex j at round r.  For + the magnitudes are natural logs
// (scaled by 1/16, floored at 2^-100) so that one network resolves deltas
// from the first round to the last, which lie ten or more decades apart;
// log1p would flatten every |Delta_j| n below 1 to the same input.  Min ops
// keep log1p of the (integer-valued) distances.
//   sum (PageRank-style) ops                        min (SSSP)
//   f0 ln(|Delta_j| n) / 16                         log1p(Delta_j) if finite, else 0
//   f1 ln(|v_j| n) / 16                             log1p(v_j) if finite, else 0
//   f2 log1p(indeg_j)                               same
//   f3 log1p(outdeg_j)                              same
//   f4 log1p(r - last activation round)             same (never activated: r + 1)
//   f5 1                                            1 if Delta_j finite
//   f6 (ln(|Delta_j| n) - log1p(outdeg_j)) / 16     1 if v_j finite
//   f7 0                                            0
#pragma once
#include <cstddef>
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

// Round to the nearest BF16 (ties to even) with integer operations, kept as
// an FP32 (finite inputs; B300 runs float <-> BF16 conversions on its narrow
// FP64 pipe).
__device__ __forceinline__ float bf16r(float x) {
  unsigned u = __float_as_uint(x);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return __uint_as_float(u & 0xFFFF0000u);
}

// Features in FP32 with the hardware logarithm (__logf, about 2^-21 from
// the exact value): the scorer runs inside the frontier scan over every
// pending vertex, the inputs are rounded to BF16 (2^-8) anyway, and FP64 or
// correctly rounded logarithms would make the features the scan's
// bottleneck (B300's FP64 pipe is a small fraction of its FP32 rate).
constexpr float kFeatFloor = 0x1p-100f;
constexpr float kFeatScale = 1.0f / 16.0f;

// Conversions on the integer and FP32 pipes (B300 issues I2F and F2F.F64 on
// its narrow FP64 pipe, which they made the scorer's bottleneck); u32_to_f32
// is in daic_ops.cuh.
// |x| for a double, as an FP32 with the mantissa truncated to 20 bits
// (relative error below 2^-20, far under the BF16 rounding of a feature);
// below FP32's normal range it is 0, above it +inf.
__device__ __forceinline__ float abs_f64_to_f32(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x)) & 0x7FFFFFFFu;
  const int e = static_cast<int>(hi >> 20) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __uint_as_float(0x7F800000u);
  return __uint_as_float((static_cast<unsigned>(e) << 23) | ((hi & 0xFFFFFu) << 3));
}
__device__ __forceinline__ float abs_f32(float x) { return fabsf(x); }
__device__ __forceinline__ float abs_f32(double x) { return abs_f64_to_f32(x); }

__device__ __forceinline__ float log1p_feature(float x) { return __logf(1.0f + x); }

// The BF16 bits (low 16) of x rounded to the nearest BF16.
__device__ __forceinline__ unsigned bf16_bits(float x) { return __float_as_uint(bf16r(x)) >> 16; }

// A vertex's features as one scorer input row: 8 BF16 values, f[2t] in the
// low half of word t.  The graph-static part comes precomputed per vertex
// (static_features): word 1 is (f2, f3), and the FP32 log(1 + outdeg) from
// which f6 = (ln(|Delta| n) - log(1 + outdeg)) / 16 is formed.  agef is
// f4 = log1p(age) (age_feature).  delta and v are magnitudes for +.
__device__ __forceinline__ uint2 static_features(unsigned indeg, unsigned outdeg) {
  const float l_out = log1p_feature(u32_to_f32(outdeg));
  const unsigned w = bf16_bits(log1p_feature(u32_to_f32(indeg))) | (bf16_bits(l_out) << 16);
  return make_uint2(w, __float_as_uint(l_out));
}

__device__ __forceinline__ float age_feature(unsigned age) { return bf16r(log1p_feature(u32_to_f32(age))); }

constexpr unsigned kBf16One = 0x3F80u;

template <bool kIsSum>
__device__ __forceinline__ uint4 feature_row(float delta, float v, bool d_finite, bool v_finite,
                                             uint2 st, float agef, float n) {
  unsigned w0, w2, w3;
  if (kIsSum) {
    const float l0 = __logf(fmaxf(delta * n, kFeatFloor));
    const float l1 = __logf(fmaxf(v * n, kFeatFloor));
    w0 = bf16_bits(l0 * kFeatScale) | (bf16_bits(l1 * kFeatScale) << 16);
    w2 = bf16_bits(agef) | (kBf16One << 16);
    w3 = bf16_bits((l0 - __uint_as_float(st.y)) * kFeatScale);
  } else {
    const unsigned f0 = d_finite ? bf16_bits(log1p_feature(delta)) : 0u;
    const unsigned f1 = v_finite ? bf16_bits(log1p_feature(v)) : 0u;
    w0 = f0 | (f1 << 16);
    w2 = bf16_bits(agef) | ((d_finite ? kBf16One : 0u) << 16);
    w3 = v_finite ? kBf16One : 0u;
  }
  return make_uint4(w0, st.x, w2, w3);
}

// The row's 8 features as FP32 values.
__device__ __forceinline__ void unpack_row(uint4 r, float* f) {
  const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    f[2 * t] = __uint_as_float(w[t] << 16);
    f[2 * t + 1] = __uint_as_float(w[t] & 0xFFFF0000u);
  }
}

static_assert(sizeof(MlpWeights) >= kMlpParams * 2 && offsetof(MlpWeights, b2) == (kMlpParams - 1) * 2,
              "BF16 weights are kMlpParams contiguous values");

// Forward pass for one input vector with the BF16 weights (training: also
// returns the hidden activations).
__device__ __forceinline__ float mlp_forward(const MlpWeights& w, const float* x, float* h_out) {
  float y = __bfloat162float(w.b2);
#pragma unroll 8
  for (int k = 0; k < kMlpHidden; ++k) {
    float acc = __bfloat162float(w.b1[k]);
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) acc = fmaf(__bfloat162float(w.w1[k * kMlpIn + i]), x[i], acc);
    const float h = acc > 0.0f ? acc : 0.0f;
    if (h_out) h_out[k] = h;
    y = fmaf(__bfloat162float(w.w2[k]), h, y);
  }
  return y;
}

// ---------------------------------------------------------------- inference
// The scheduler scores vertices a warp at a time on the tensor cores: the
// first layer is a dense contraction, H (16 vertices x 64) = F (16 x 8,
// padded to K = 16) x W1^T, one mma.sync.m16n8k16 (BF16 in, FP32
// accumulation) per 8 hidden units, with b1 as the accumulator's initial
// value; ReLU, the 64 -> 1 layer and b2 follow in FP32 on the accumulator
// registers, and a quad shuffle sums the four lanes that share a vertex.
// Fragment layouts are those of the PTX ISA for m16n8k16 (g = lane / 4,
// t = lane % 4): A holds F[g][2t, 2t+1] and F[g+8][2t, 2t+1] (the K >= 8
// halves are zero), B holds W1[8 nt + g][2t, 2t+1], and the accumulator
// H[g][8 nt + 2t, +1] and H[g+8][8 nt + 2t, +1].  Inputs and weights are
// BF16, every product is exact in FP32, and only the order of the FP32 sums
// differs from the scalar forward used in training.

// The weights in fragment order, staged once per CTA in shared memory.
struct MlpFrag {
  unsigned w1f[kMlpHidden / 8][32];   // [n-tile][lane]: W1[8 nt + g][2t, 2t+1] (BF16 pair)
  float2 b1f[kMlpHidden / 8][4];      // [n-tile][t]: (b1[8 nt + 2t], b1[8 nt + 2t + 1])
  float2 w2f[kMlpHidden / 8][4];      // [n-tile][t]: (w2[8 nt + 2t], w2[8 nt + 2t + 1])
  float b2;
};

__device__ __forceinline__ void stage_mlp(const MlpWeights* __restrict__ g, MlpFrag* s) {
  const unsigned* w1 = reinterpret_cast<const unsigned*>(g->w1);   // BF16 pairs along i
  for (int x = threadIdx.x; x < (kMlpHidden / 8) * 32; x += blockDim.x) {
    const int nt = x >> 5, lane = x & 31;
    s->w1f[nt][lane] = w1[(8 * nt + (lane >> 2)) * (kMlpIn / 2) + (lane & 3)];
  }
  for (int x = threadIdx.x; x < (kMlpHidden / 8) * 4; x += blockDim.x) {
    const int nt = x >> 2, t = x & 3, k = 8 * nt + 2 * t;
    s->b1f[nt][t] = make_float2(__bfloat162float(g->b1[k]), __bfloat162float(g->b1[k + 1]));
    s->w2f[nt][t] = make_float2(__bfloat162float(g->w2[k]), __bfloat162float(g->w2[k + 1]));
  }
  if (threadIdx.x == 0) s->b2 = __bfloat162float(g->b2);
}

// One scorer input row: the 8 features (already BF16 values, bf16r) as BF16
// bits, f[2t] in the low half of word t.
__device__ __forceinline__ uint4 pack_features(const float* f) {
  unsigned w[4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
    w[t] = (__float_as_uint(f[2 * t]) >> 16) | (__float_as_uint(f[2 * t + 1]) & 0xFFFF0000u);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void mma_bf16_16816(float* c, unsigned a0, unsigned a1, unsigned b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(0u), "r"(0u), "r"(b0), "r"(0u));
}

// Scores rows[0..cnt) (a warp's shared-memory rows) into out[0..cnt).  Called
// by all 32 lanes of a warp with the same cnt.
__device__ __forceinline__ void warp_score(const MlpFrag& w, const uint4* rows, int cnt, float* out) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int base = 0; base < cnt; base += 16) {
    const int r0 = base + g, r1 = base + g + 8;
    const unsigned a0 = r0 < cnt ? reinterpret_cast<const unsigned*>(rows + r0)[t] : 0u;
    const unsigned a1 = r1 < cnt ? reinterpret_cast<const unsigned*>(rows + r1)[t] : 0u;
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int nt = 0; nt < kMlpHidden / 8; ++nt) {
      const float2 bias = w.b1f[nt][t];
      const float2 w2 = w.w2f[nt][t];
      float c[4] = {bias.x, bias.y, bias.x, bias.y};
      mma_bf16_16816(c, a0, a1, w.w1f[nt][lane]);
      y0 = fmaf(w2.x, fmaxf(c[0], 0.0f), y0);
      y0 = fmaf(w2.y, fmaxf(c[1], 0.0f), y0);
      y1 = fmaf(w2.x, fmaxf(c[2], 0.0f), y1);
      y1 = fmaf(w2.y, fmaxf(c[3], 0.0f), y1);
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (t == 0) {
      if (r0 < cnt) out[r0] = y0 + w.b2;
      if (r1 < cnt) out[r1] = y1 + w.b2;
    }
  }
}

// Order-preserving map of a score to a non-zero 32-bit key (0 = not pending).
__device__ __forceinline__ unsigned score_key(float s) {
  const unsigned u = __float_as_uint(s);
  const unsigned k = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return k ? k : 1u;
}

}  // namespace maiter
