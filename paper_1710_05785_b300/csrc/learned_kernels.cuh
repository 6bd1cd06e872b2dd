// Learned scheduling in the round engine: the scorer kernel writes one
// priority key per pending vertex from the MLP, the top-q radix select then
// picks the round's frontier from those keys (topq_kernels.cuh).  Every
// kFairPeriod-th round every pending vertex is keyed alike, so it is selected
// whatever the network says: no vertex can be starved, which the convergence
// of priority scheduling (Lemma 5, Theorem 3) needs.  The termination test
// does not depend on the scheduler.
//
// k_trace records the same features for a sample of vertices, so traces of
// the method's own runs train the network on exactly the inputs it scores.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_kernels.cuh"
#include "mlp.cuh"

namespace maiter {

constexpr int kFairPeriod = 8;

template <class Op>
__device__ __forceinline__ void features_of(const KArgs<Op>& a, const int* __restrict__ indeg, int j,
                                            unsigned round, float* f) {
  const typename Op::D d = a.delta[j];
  const typename Op::V vv = a.v[j];
  const int deg = __ldg(a.rp + j + 1) - __ldg(a.rp + j);
  const unsigned la = a.last_act ? a.last_act[j] : 0u;
  const unsigned age = la ? round + 1u - la : round + 1u;
  if constexpr (Op::kIsSum) {
    vertex_features<true>(static_cast<double>(d), static_cast<double>(vv), true, true, indeg[j], deg,
                          age, static_cast<double>(a.n), f);
  } else {
    vertex_features<false>(Op::value(d), Op::value(vv), d != Op::kNone, vv != Op::kNone,
                           indeg[j], deg, age, static_cast<double>(a.n), f);
  }
}

template <class Op, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_score(KArgs<Op> a, const MlpWeights* __restrict__ wg,
                                                 const int* __restrict__ indeg,
                                                 unsigned* __restrict__ keys) {
  __shared__ MlpWeights W;
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(MlpWeights) / 2); i += BLOCK)
    reinterpret_cast<unsigned short*>(&W)[i] = reinterpret_cast<const unsigned short*>(wg)[i];
  __syncthreads();
  const unsigned round = static_cast<unsigned>(a.ctl->rounds);
  const bool fair = (round % kFairPeriod) == kFairPeriod - 1;
  for (int j = blockIdx.x * BLOCK + threadIdx.x; j < a.n; j += gridDim.x * BLOCK) {
    const typename Op::V vv = Op::kIsSum ? typename Op::V(0) : a.v[j];
    if (!Op::pending(a.delta[j], vv)) {
      keys[j] = 0u;
      continue;
    }
    if (fair) {
      keys[j] = 1u;
      continue;
    }
    float f[kMlpIn];
    features_of(a, indeg, j, round, f);
    keys[j] = score_key(mlp_forward(W, f, nullptr));
  }
}

// Records features, delta, state and last-update round of sampled vertices.
template <class Op>
__global__ void k_trace(KArgs<Op> a, const int* __restrict__ indeg, const int* __restrict__ sample,
                        int ns, float* __restrict__ feat, double* __restrict__ dl,
                        double* __restrict__ vs, unsigned* __restrict__ la) {
  const unsigned round = static_cast<unsigned>(a.ctl->rounds);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    const int j = sample[s];
    features_of(a, indeg, j, round, feat + static_cast<int64_t>(s) * kMlpIn);
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

}  // namespace maiter
