// Learned scheduling in the round engine: a sample of pending vertices is
// scored to fix the round's threshold (k_learned_threshold), then the
// frontier scan (k_scan with kLearn) scores every pending vertex in its tile
// pass and selects those whose key reaches the threshold.  A vertex left
// pending for kMaxAge rounds is selected whatever the network says
// (learned_key).  The termination test does not depend on the scheduler.
//
// k_trace records the same features for a sample of vertices, so traces of
// the method's own runs train the network on exactly the inputs it scores.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_kernels.cuh"
#include "mlp.cuh"

namespace maiter {

// The round's selection threshold from a sample, the extraction the paper's
// priority queue uses (Section 5.1, sampling after PrIter) in place of an
// exact order statistic.  kLearnedBlocks CTAs draw one vertex per thread by
// a counter-based hash of (round, draw), score the pending ones with the
// same features and network as the scan, and store the keys; the last CTA
// to finish finds the key ranked ceil(q x pending draws) from the top by a
// four-pass radix select (8 bits a pass) and stores it as the threshold.
// The scan then selects every pending vertex whose key is at least that.
// When few draws hit a pending vertex (kLearnedMinPend) the threshold is 1:
// every pending vertex is selected, so every round makes progress.
// Rounds whose sample holds fewer pending draws than this (a frontier below
// 1/16 of the vertices) select every pending vertex: a small frontier costs
// little to push in full, and holding part of it back would only add rounds,
// whose fixed cost is what the schedule must save.
constexpr unsigned kLearnedMinPend = 256;
constexpr int kLearnedBlock = 256;
constexpr int kLearnedBlocks = kLearnedSample / kLearnedBlock;
static_assert(kLearnedBlocks * kLearnedBlock == kLearnedSample, "one draw per thread");

// The SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): a
// counter-based hash, so the sample of a round is fixed by the round alone.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Launched as a programmatic dependent of the push before it: the weights
// are staged while that grid drains, then griddepcontrol.wait makes its
// writes visible.
template <class Op>
__global__ void __launch_bounds__(kLearnedBlock) k_learned_threshold(KArgs<Op> a, TopqCtl* tq) {
  __shared__ MlpFrag s_w;
  __shared__ uint4 s_lf[kLearnedBlock / 32][32];
  __shared__ float s_ly[kLearnedBlock / 32][32];
  __shared__ unsigned s_hist[256];
  __shared__ unsigned s_prefix, s_rank;
  __shared__ int s_last;
  stage_mlp(a.mlp, &s_w);
  __syncthreads();
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  if (a.ctl->status != 0) return;   // a round after the stopping one (uniform)
  const unsigned round = static_cast<unsigned>(a.ctl->rounds);
  const int draw = blockIdx.x * kLearnedBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  bool p = false;
  LearnIn<Op> in{};
  if (a.n > 0) {
    const unsigned long long h =
        splitmix64((static_cast<unsigned long long>(round) << 20) ^ static_cast<unsigned long long>(draw));
    const int j = static_cast<int>(h % static_cast<unsigned long long>(a.n));
    in = learn_in(a, j);
    p = Op::pending(in.d, Op::kIsSum ? typename Op::V(0) : in.v);
  }
  const bool aged = p && aged_out(in.la, round);
  const bool sc = p && !aged;
  const unsigned b = __ballot_sync(0xffffffffu, sc);
  const int slot = __popc(b & ((1u << lane) - 1u));
  if (sc) s_lf[wid][slot] = learn_row(a, in, age_feature(age_of(in.la, round)));
  __syncwarp();
  warp_score(s_w, s_lf[wid], __popc(b), s_ly[wid]);
  __syncwarp();
  const unsigned key = aged ? kAgedKey : (sc ? score_key(s_ly[wid][slot]) : 0u);
  tq->sample[draw] = key;
  const int pend = __syncthreads_count(key != 0u);
  if (threadIdx.x == 0) {
    if (pend) atomicAdd(&tq->sample_pend, static_cast<unsigned>(pend));
    __threadfence();
    s_last = atomicAdd(&tq->sample_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last CTA: every draw's key is in tq->sample (read past L1)
  unsigned kk[kLearnedSample / kLearnedBlock];
#pragma unroll
  for (int t = 0; t < kLearnedSample / kLearnedBlock; ++t)
    kk[t] = __ldcg(tq->sample + t * kLearnedBlock + threadIdx.x);
  const unsigned P = atomicAdd(&tq->sample_pend, 0u);
  if (P < kLearnedMinPend) {
    if (threadIdx.x == 0) {
      tq->key_thr = 1u;
      tq->sample_done = 0u;
    }
    return;
  }
  if (threadIdx.x == 0) {
    const double want = ceil(tq->frac * static_cast<double>(P));
    s_rank = static_cast<unsigned>(want < 1.0 ? 1.0 : (want > P ? P : want));
    s_prefix = 0u;
  }
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    s_hist[threadIdx.x] = 0u;   // kLearnedBlock == 256 bins
    __syncthreads();
    const unsigned prefix = s_prefix;
#pragma unroll
    for (int t = 0; t < kLearnedSample / kLearnedBlock; ++t) {
      const unsigned k = kk[t];
      const bool in = k != 0u && (pass == 0 || (k >> (shift + 8)) == prefix);
      if (in) atomicAdd(&s_hist[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // lane l holds bins 255 - 8l down to 248 - 8l (the largest first)
      unsigned c[8], sum = 0u;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        c[b] = s_hist[255 - 8 * lane - b];
        sum += c[b];
      }
      unsigned inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const unsigned rank = s_rank;
      const unsigned hit = __ballot_sync(0xffffffffu, inc >= rank);
      if (hit && lane == __ffs(hit) - 1) {
        unsigned before = inc - sum;
        int bin = 255 - 8 * lane;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          if (before + c[b] >= rank) {
            bin = 255 - 8 * lane - b;
            break;
          }
          before += c[b];
        }
        s_prefix = (prefix << 8) | static_cast<unsigned>(bin);
        s_rank = rank - before;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tq->key_thr = s_prefix > 1u ? s_prefix : 1u;
    tq->sample_pend = 0u;
    tq->sample_done = 0u;
  }
}

// Records features, delta, state and last-update round of sampled vertices.
template <class Op>
__global__ void k_trace(KArgs<Op> a, const int* __restrict__ sample, int ns, float* __restrict__ feat,
                        double* __restrict__ dl, double* __restrict__ vs, unsigned* __restrict__ la) {
  const unsigned round = static_cast<unsigned>(a.ctl->rounds);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    const int j = sample[s];
    const LearnIn<Op> in = learn_in(a, j);
    unpack_row(learn_row(a, in, age_feature(age_of(in.la, round))),
               feat + static_cast<int64_t>(s) * kMlpIn);
    dl[s] = static_cast<double>(a.delta[j]);
    vs[s] = static_cast<double>(a.v[j]);
    la[s] = a.last_act ? a.last_act[j] : 0u;
  }
}

// In-degree of every vertex (a feature), from the out-edge CSR.
static __global__ void k_indegree(const int* __restrict__ col, int64_t m, int* __restrict__ indeg) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicAdd(indeg + col[e], 1);
}

// The graph-static scorer features of every vertex (static_features).
static __global__ void k_learn_static(const int* __restrict__ rp, const int* __restrict__ indeg, int n,
                                      uint2* __restrict__ st) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    st[j] = static_features(static_cast<unsigned>(indeg[j]), static_cast<unsigned>(rp[j + 1] - rp[j]));
}

}  // namespace maiter
