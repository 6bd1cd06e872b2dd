// Receive-side rounds for a group of up to kVQ personalised-PageRank queries
// on one graph (batch mode 3): the receive-side engine's round (reading of
// Eq. 5 at the receivers, see pull_kernels.cuh) with every vertex's delta,
// state and message a vector of the group's queries, stored query-minor
// (vertex k's kVQ values contiguous).  Per in-edge a warp reads the sender's
// whole message vector, kVQ x 4 bytes in one coalesced transaction, where
// one query alone would read 4 bytes at a random address: the random access
// is paid once for the group.  Lane l holds queries 2l and 2l + 1.
//
// Each query keeps its own damping d_q (message c_kq Delta = d_q / outdeg(k)
// Delta, with d_q as an FP32 pair dq + dq_lo: a damping rounded once to FP32
// would scale every hop by the same 1 + 2^-24-ish factor, a bias that the
// PageRank sum amplifies by d / (1 - d)^2, 1.1e-6 for d = 0.85), tolerance
// and FP64 residual sum_k |Delta_kq|; the group's loop
// ends when every query's residual is below half its eps_q (each query's
// round of convergence is recorded; later rounds only shrink its residual
// further).  FP32 deltas and messages, FP64 state and residuals, as the
// receive-side engine's headline precision.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pull_kernels.cuh"

namespace maiter {

constexpr int kVQ = 64;            // queries of a group
// A query stops at sum |Delta| < kVecEpsFrac x eps_q: its error bound
// eps_q / (1 - d) (in L1) is shared between the termination test and the
// FP32 rounding of the deltas and messages (about 1e-7 relative).
constexpr double kVecEpsFrac = 0.5;
constexpr int kVBlock = 256;

struct VCtl {
  double resid_acc[2][kVQ];        // [set][slot] sum |Delta| of the round's new deltas
  double eps[kVQ];                 // per slot: tolerance (0 for an empty slot)
  float dq[kVQ];                   // per slot: damping rounded to FP32 (0 for an empty slot)
  float dq_lo[kVQ];                // per slot: damping - dq (FP32): the rounding put back
  int conv_round[kVQ];             // per slot: round at which its residual fell below eps (-1)
  int nq;                          // slots in use
  unsigned scan_set, push_set;
  int status;                      // 0 running, 1 every query converged, 2 round cap
  unsigned long long rounds;
  long long max_rounds;
};

struct PullVArgs {
  int n;
  const int* __restrict__ crp;
  const int* __restrict__ csrc;          // sender rank of every in-edge
  const int* __restrict__ sbase;         // senders before every word of 32 rows
  const unsigned* __restrict__ smask;    // the word's senders, one bit per row
  const int4* __restrict__ large;
  const int* __restrict__ large_nch;
  const unsigned* __restrict__ lbits;
  int nlarge;
  double* lacc;                    // [large row][kVQ]: FP64 sums, zero between rounds
  unsigned* lcnt;                  // [large row]: chunks added this round
  const float2* __restrict__ inv_deg;  // 1 / outdeg as an FP32 pair hi + lo (0 without out-edges)
  double* v;                       // [n][kVQ]
  float* delta;                    // [n][kVQ]
  float* msg[2];                   // [sender rank][kVQ] each, alternating by set
  VCtl* ctl;
};

// Zero state and deltas, then (k_vec_seed) the seeds; the control block
// starts from `init`.
static __global__ void k_vec_init(PullVArgs a, VCtl init) {
  const int64_t total = static_cast<int64_t>(a.n) * kVQ;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    a.v[i] = 0.0;
    a.delta[i] = 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.ctl = init;
}

// seeds[i] = (slot, vertex), value[i] = (1 - d) / |S| of its query.
static __global__ void k_vec_seed(PullVArgs a, const int2* __restrict__ seeds,
                                  const float* __restrict__ value, int ns) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ns) {
    const int2 s = seeds[i];
    a.delta[static_cast<int64_t>(s.y) * kVQ + s.x] = value[i];
  }
}

// The two messages d_q / outdeg(k) x Delta of a lane: t = Delta / outdeg
// (Delta x (hi + lo) in one fused rounding), then t x (dq + dq_lo) with one
// more.  Both constants enter as FP32 pairs: a coefficient rounded once to
// FP32 would scale every message of the vertex by the same error, a bias the
// PageRank sum amplifies by up to d / (1 - d).
__device__ __forceinline__ float2 vec_message(float s0, float s1, float2 inv_deg, float2 dq,
                                              float2 dl) {
  const float t0 = fmaf(s0, inv_deg.x, s0 * inv_deg.y), t1 = fmaf(s1, inv_deg.x, s1 * inv_deg.y);
  return make_float2(fmaf(t0, dq.x, t0 * dl.x), fmaf(t1, dq.y, t1 * dl.y));
}

// Per-slot FP64 sums of the block's lanes into set ws (one atomic per slot
// per block).
__device__ __forceinline__ void vec_block_resid(VCtl* ctl, unsigned ws, double r0, double r1) {
  __shared__ double s_r[kVBlock / 32][kVQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  s_r[wid][2 * lane] = r0;
  s_r[wid][2 * lane + 1] = r1;
  __syncthreads();
  if (threadIdx.x < kVQ) {
    double t = 0.0;
    for (int w = 0; w < kVBlock / 32; ++w) t += s_r[w][threadIdx.x];
    if (t != 0.0) atomicAdd(&ctl->resid_acc[ws][threadIdx.x], t);
  }
}

// The first messages: msg[ws][k] = c_k d_q Delta_kq, and the residuals of
// the first deltas into set ws.  A warp per vertex.
static __global__ void __launch_bounds__(kVBlock) k_vec_prime(PullVArgs a) {
  VCtl* ctl = a.ctl;
  const unsigned ws = ctl->scan_set;
  const int lane = threadIdx.x & 31;
  const float2 dq = make_float2(ctl->dq[2 * lane], ctl->dq[2 * lane + 1]);
  const float2 dl = make_float2(ctl->dq_lo[2 * lane], ctl->dq_lo[2 * lane + 1]);
  float* msg = a.msg[ws];
  double r0 = 0.0, r1 = 0.0;
  const int w0 = (blockIdx.x * kVBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kVBlock) >> 5;
  for (int k = w0; k < a.n; k += nw) {
    const int64_t o = static_cast<int64_t>(k) * kVQ + 2 * lane;
    const float2 d = *reinterpret_cast<const float2*>(a.delta + o);
    const float2 c = __ldg(a.inv_deg + k);
    if (c.x != 0.0f) {   // a sender: its message slot is its rank
      const int64_t om = static_cast<int64_t>(sender_index(a.sbase, a.smask, k)) * kVQ + 2 * lane;
      *reinterpret_cast<float2*>(msg + om) = vec_message(d.x, d.y, c, dq, dl);
    }
    r0 += fabs(static_cast<double>(d.x));
    r1 += fabs(static_cast<double>(d.y));
  }
  vec_block_resid(ctl, ws, r0, r1);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->push_set = ws;
}

// The round's decision (one warp pair, kVQ threads): every query whose
// residual fell below its eps records the round; the loop goes on while a
// query has not, up to the round cap.
static __global__ void k_vec_decide(VCtl* ctl, cudaGraphConditionalHandle cond, int use_cond) {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  const int q = threadIdx.x;
  const int st0 = ctl->status;
  if (st0 != 0) {
    if (q == 0 && use_cond) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const unsigned ps = ctl->push_set, ns = ps ^ 1u;
  const unsigned long long rounds = ctl->rounds;
  bool done = true;
  if (q < ctl->nq) {
    if (ctl->conv_round[q] < 0 && ctl->resid_acc[ps][q] < ctl->eps[q])
      ctl->conv_round[q] = static_cast<int>(rounds);
    done = ctl->conv_round[q] >= 0;
  }
  const bool all = __syncthreads_and(done);
  ctl->resid_acc[ns][q] = 0.0;
  if (q == 0) {
    unsigned cont = 0;
    if (all) ctl->status = 1;
    else if (static_cast<long long>(rounds) >= ctl->max_rounds) ctl->status = 2;
    else cont = 1;
    if (cont) ctl->rounds = rounds + 1;
    ctl->scan_set = ns;
    if (use_cond) cudaGraphSetConditional(cond, cont);
  }
}

// One round for the group: the large rows' chunks, a warp each (FP64
// accumulation per row, the last chunk folds), then the other rows, a warp
// per row.
static __global__ void __launch_bounds__(kVBlock, 4) k_vec_pull(PullVArgs a) {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  VCtl* ctl = a.ctl;
  if (ctl->status != 0) return;
  const unsigned ws = ctl->scan_set;
  const float* __restrict__ msg_in = a.msg[ws ^ 1u];
  float* msg_out = a.msg[ws];
  const int lane = threadIdx.x & 31;
  const float2 dq = make_float2(ctl->dq[2 * lane], ctl->dq[2 * lane + 1]);
  const float2 dl = make_float2(ctl->dq_lo[2 * lane], ctl->dq_lo[2 * lane + 1]);
  double r0 = 0.0, r1 = 0.0;
  const int gw = (blockIdx.x * kVBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kVBlock) >> 5;

  auto fold = [&](int k, float s0, float s1) {
    const int64_t o = static_cast<int64_t>(k) * kVQ + 2 * lane;
    const float2 dold = *reinterpret_cast<const float2*>(a.delta + o);
    double2 vv = *reinterpret_cast<const double2*>(a.v + o);
    vv.x += static_cast<double>(dold.x);
    vv.y += static_cast<double>(dold.y);
    *reinterpret_cast<double2*>(a.v + o) = vv;
    *reinterpret_cast<float2*>(a.delta + o) = make_float2(s0, s1);
    const float2 c = __ldg(a.inv_deg + k);
    if (c.x != 0.0f) {
      const int64_t om = static_cast<int64_t>(sender_index(a.sbase, a.smask, k)) * kVQ + 2 * lane;
      *reinterpret_cast<float2*>(msg_out + om) = vec_message(s0, s1, c, dq, dl);
    }
    r0 += fabs(static_cast<double>(s0));
    r1 += fabs(static_cast<double>(s1));
  };

  // large rows: a warp per chunk
  for (int c = gw; c < a.nlarge; c += nw) {
    const int4 ent = __ldg(a.large + c);
    float2 acc = make_float2(0.0f, 0.0f);
    for (int e0 = ent.y; e0 < ent.z; e0 += 32) {
      const int my = e0 + lane < ent.z ? __ldcs(a.csrc + e0 + lane) : -1;
      const int cnt = min(32, ent.z - e0);
      for (int i = 0; i < cnt; ++i) {
        const int j = __shfl_sync(0xffffffffu, my, i);
        const float2 m = *reinterpret_cast<const float2*>(msg_in + static_cast<int64_t>(j) * kVQ + 2 * lane);
        acc.x += m.x;
        acc.y += m.y;
      }
    }
    double* la = a.lacc + static_cast<int64_t>(ent.w) * kVQ + 2 * lane;
    atomicAdd(la, static_cast<double>(acc.x));
    atomicAdd(la + 1, static_cast<double>(acc.y));
    __threadfence();
    int last = 0;
    if (lane == 0)
      last = atomicAdd(a.lcnt + ent.w, 1u) == static_cast<unsigned>(__ldg(a.large_nch + ent.w)) - 1u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      const double s0 = __longlong_as_double(static_cast<long long>(
          atomicExch(reinterpret_cast<unsigned long long*>(la), 0ull)));
      const double s1 = __longlong_as_double(static_cast<long long>(
          atomicExch(reinterpret_cast<unsigned long long*>(la + 1), 0ull)));
      if (lane == 0) a.lcnt[ent.w] = 0u;
      fold(ent.x, static_cast<float>(s0), static_cast<float>(s1));
    }
  }

  // the other rows: a warp per row; its senders read 32 at a time, their
  // message vectors four at a time
  for (int k = gw; k < a.n; k += nw) {
    if ((__ldg(a.lbits + (k >> 5)) >> (k & 31)) & 1u) continue;   // summed by its chunks
    const int b = __ldg(a.crp + k), e = __ldg(a.crp + k + 1);
    float2 acc = make_float2(0.0f, 0.0f);
    for (int e0 = b; e0 < e; e0 += 32) {
      const int my = e0 + lane < e ? __ldcs(a.csrc + e0 + lane) : -1;
      const int cnt = min(32, e - e0);
      int i = 0;
      for (; i + 4 <= cnt; i += 4) {
        float2 m[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = __shfl_sync(0xffffffffu, my, i + u);
          m[u] = *reinterpret_cast<const float2*>(msg_in + static_cast<int64_t>(j) * kVQ + 2 * lane);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc.x += m[u].x;
          acc.y += m[u].y;
        }
      }
      for (; i < cnt; ++i) {
        const int j = __shfl_sync(0xffffffffu, my, i);
        const float2 m = *reinterpret_cast<const float2*>(msg_in + static_cast<int64_t>(j) * kVQ + 2 * lane);
        acc.x += m.x;
        acc.y += m.y;
      }
    }
    fold(k, acc.x, acc.y);
  }
  vec_block_resid(ctl, ws, r0, r1);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->push_set = ws;
}

// 1 / outdeg of every vertex as an FP32 pair: hi = 1 / outdeg rounded, lo =
// the remainder rounded (0, 0 without out-edges).
static __global__ void k_vec_inv_deg(const int* __restrict__ rp, int n, float2* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int d = __ldg(rp + k + 1) - __ldg(rp + k);
    const double x = d > 0 ? 1.0 / static_cast<double>(d) : 0.0;
    const float hi = static_cast<float>(x);
    out[k] = make_float2(hi, static_cast<float>(x - static_cast<double>(hi)));
  }
}

}  // namespace maiter
