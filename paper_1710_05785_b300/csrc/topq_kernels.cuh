// Top-fraction priority selection (priority queue extraction, Section 5.1):
// the activation threshold of a round is the exact k-th largest priority key,
// k = ceil(q * #pending), found by a three-pass radix select on the 32-bit
// key (11 + 11 + 10 bits); every pending vertex whose key is >= it is
// activated, ties included.
//
// Priority key (Section 3.5, |v (+) Delta - v|, rounded to FP32 so the
// comparison is on 32 bits): |Delta_j| for +; v_j - Delta_j for min, with
// v_j = infinity mapped to +inf.  Positive floats order like their bit
// patterns, so the key is the float's bits; 0 means "not pending".
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_kernels.cuh"

namespace maiter {

// Pass p histograms bits [hi_bit - width, hi_bit) of the keys whose higher
// bits equal the prefix found so far.  The last block picks the bucket that
// holds the k-th largest key and narrows the prefix; after pass 2 the prefix
// is the threshold key itself.
template <class Op, int BLOCK, int PASS>
__global__ void __launch_bounds__(BLOCK) k_topq_hist(KArgs<Op> a, TopqCtl* tq) {
  constexpr int kShift = PASS == 0 ? 21 : (PASS == 1 ? 10 : 0);
  constexpr int kWidth = PASS == 2 ? 10 : 11;
  constexpr unsigned kMask = (1u << kWidth) - 1u;
  constexpr int kHigh = kShift + kWidth;            // bits above this are fixed
  __shared__ unsigned s_hist[1 << kWidth];
  __shared__ int s_last;
  for (int i = threadIdx.x; i < (1 << kWidth); i += BLOCK) s_hist[i] = 0;
  __syncthreads();
  const unsigned prefix = tq->prefix;
  unsigned long long npend = 0;
  for (int j = blockIdx.x * BLOCK + threadIdx.x; j < a.n; j += gridDim.x * BLOCK) {
    const typename Op::V vv = Op::kIsSum ? typename Op::V(0) : a.v[j];
    const unsigned key = priority_key<Op>(a.delta[j], vv);
    if (key == 0u) continue;
    if (PASS == 0) ++npend;
    if (PASS == 0 || (key >> kHigh) == prefix)
      atomicAdd(&s_hist[(key >> kShift) & kMask], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << kWidth); i += BLOCK)
    if (s_hist[i]) atomicAdd(&tq->hist[PASS][i], s_hist[i]);
  if (PASS == 0) {
    for (int o = 16; o > 0; o >>= 1) npend += __shfl_xor_sync(0xffffffffu, npend, o);
    if ((threadIdx.x & 31) == 0 && npend) atomicAdd(&tq->pend, npend);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&tq->ticket[PASS], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  volatile TopqCtl* vt = tq;
  for (int i = threadIdx.x; i < (1 << kWidth); i += BLOCK) {
    s_hist[i] = vt->hist[PASS][i];
    tq->hist[PASS][i] = 0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned k;
  if (PASS == 0) {
    const unsigned long long pend = vt->pend;
    tq->pend = 0;
    if (pend == 0) {
      tq->key_thr = 0xFFFFFFFFu;   // nothing pending: select none
      tq->kth = 0;
      tq->prefix = 0;
      tq->ticket[PASS] = 0;
      return;
    }
    const double want = ceil(vt->frac * static_cast<double>(pend));
    k = static_cast<unsigned>(want < 1.0 ? 1.0 : (want > static_cast<double>(pend) ? pend : want));
  } else {
    k = vt->kth;
  }
  if (k == 0) {                    // pass 0 found nothing pending
    tq->ticket[PASS] = 0;
    return;
  }
  // walk buckets from the largest key down to the one holding the k-th
  unsigned bucket = 0, above = 0;
  for (int b = (1 << kWidth) - 1; b >= 0; --b) {
    const unsigned c = s_hist[b];
    if (above + c >= k) { bucket = static_cast<unsigned>(b); break; }
    above += c;
  }
  const unsigned np = ((PASS == 0 ? 0u : vt->prefix) << kWidth) | bucket;
  tq->prefix = np;
  tq->kth = k - above;
  if (PASS == 2) tq->key_thr = np;
  tq->ticket[PASS] = 0;
}

}  // namespace maiter
