// Hot-path kernels of the round-synchronous DAIC engine.
//
//   k_scan  - frontier builder (scheduler, Section 3.5 / Section 5.1) fused
//             with the termination reduction (progress estimator, Section 5.1):
//             one coalesced pass over Delta (and v for min) that
//               * reduces sum_j |Delta_j| in FP64 (or counts pending vertices),
//               * selects the vertices to activate (all pending, or priority
//                 above a threshold),
//               * compacts them with warp ballots into three lists by
//                 out-degree (small / medium / large),
//             and whose last block decides, on the device, whether another
//             round follows (it sets the WHILE condition of the CUDA graph).
//   k_push  - the update of Eq. 5 for every listed vertex: read-and-reset of
//             Delta_j, fold into v_j, and the scatter of g_{j,k}(Delta_j) into
//             every out-neighbour's Delta_k with atomics.  Work granularity by
//             degree: a whole CTA per large vertex, a warp per medium vertex,
//             and for small vertices a warp that gathers the edges of 32
//             vertices and processes them 32 at a time (prefix sum + search),
//             so every lane has an edge on every step.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_ops.cuh"

namespace maiter {

constexpr int kBuckets = 3;

// Device-resident control block of one run.  Everything the round loop needs
// to decide on its own lives here, so the loop never returns to the host.
struct DevCtl {
  unsigned int cnt[2][4];        // [set][bucket] frontier sizes (double-buffered)
  unsigned int rset;             // set the next push reads
  unsigned int wset;             // set the next scan writes
  unsigned int ticket;           // last-block election in k_scan
  int status;                    // 0 running, 1 converged, 2 round cap hit
  double resid_acc;              // this scan: sum |Delta| (sum) or pending count (min)
  unsigned long long act_acc;    // this scan: selected vertices
  unsigned long long push_acc;   // this scan: sum of out-degrees of selected vertices
  unsigned long long pend_acc;   // this scan: pending vertices (Delta != 0 / Delta < v)
  unsigned long long rounds;
  unsigned long long activations;
  unsigned long long pushes;
  double residual;               // last decided residual
  double tau;                    // current activation threshold (sum ops)
  double eps;                    // termination bound (sum ops)
  long long max_rounds;
  int sched;                     // maiter_sched
  int pad;
};

template <class Op>
struct KArgs {
  int n;
  const int* __restrict__ rp;    // n + 1 offsets (int32)
  EdgeCtx edges;
  const typename Op::C* coef;    // nullable
  double damping;
  typename Op::V* v;
  typename Op::D* delta;
  int* list[kBuckets];
  DevCtl* ctl;
  int cut_warp;                  // deg <  cut_warp : small bucket
  int cut_cta;                   // deg >= cut_cta  : large bucket
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// ------------------------------------------------------------------ scan

template <class Op, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_scan(KArgs<Op> a, cudaGraphConditionalHandle cond,
                                                 int use_cond) {
  static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block");
  DevCtl* ctl = a.ctl;
  const unsigned ws = ctl->wset;
  const double tau = ctl->tau;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;

  double rsum = 0.0;
  unsigned long long nact = 0, npush = 0, npend = 0;

  // Warps walk 32 consecutive vertices at a time: coalesced loads, and each
  // ballot covers one aligned group so compaction needs one atomic per bucket.
  const int stride = gridDim.x * BLOCK;
  for (int base = blockIdx.x * BLOCK + (threadIdx.x & ~31); base < a.n; base += stride) {
    const int j = base + lane;
    bool sel = false;
    int deg = 0;
    if (j < a.n) {
      typename Op::D d = a.delta[j];
      typename Op::V vv = Op::kIsSum ? typename Op::V(0) : a.v[j];
      bool pend = Op::pending(d, vv);
      npend += pend;
      if (Op::kIsSum) {
        double p = Op::priority(d, vv);
        rsum += p;
        sel = pend && p > tau;
      } else {
        sel = pend;
      }
      if (sel) deg = __ldg(a.rp + j + 1) - __ldg(a.rp + j);
    }
    const int bucket = deg < a.cut_warp ? 0 : (deg < a.cut_cta ? 1 : 2);
#pragma unroll
    for (int b = 0; b < kBuckets; ++b) {
      const bool mine = sel && bucket == b;
      const unsigned mask = __ballot_sync(0xffffffffu, mine);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        unsigned pos = 0;
        if (lane == leader) pos = atomicAdd(&ctl->cnt[ws][b], static_cast<unsigned>(__popc(mask)));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (mine) a.list[b][pos + __popc(mask & lt_mask)] = j;
      }
    }
    nact += sel;
    npush += static_cast<unsigned long long>(deg);
  }

  // Block reduction, one atomic per block per counter.
  __shared__ double s_r[BLOCK / 32];
  __shared__ unsigned long long s_a[BLOCK / 32], s_p[BLOCK / 32], s_q[BLOCK / 32];
  __shared__ bool s_last;
  rsum = warp_sum(rsum);
  nact = warp_sum(nact);
  npush = warp_sum(npush);
  npend = warp_sum(npend);
  const int wid = threadIdx.x >> 5;
  if (lane == 0) { s_r[wid] = rsum; s_a[wid] = nact; s_p[wid] = npush; s_q[wid] = npend; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    unsigned long long x = 0, y = 0, z = 0;
    for (int i = 0; i < BLOCK / 32; ++i) { r += s_r[i]; x += s_a[i]; y += s_p[i]; z += s_q[i]; }
    if (Op::kIsSum && r != 0.0) atomicAdd(&ctl->resid_acc, r);
    if (x) atomicAdd(&ctl->act_acc, x);
    if (y) atomicAdd(&ctl->push_acc, y);
    if (z) atomicAdd(&ctl->pend_acc, z);
    __threadfence();
    const unsigned t = atomicAdd(&ctl->ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;

  // Last block: every other block's counters are visible (fence + ticket).
  __threadfence();
  volatile DevCtl* vc = ctl;
  const double resid = Op::kIsSum ? vc->resid_acc : static_cast<double>(vc->pend_acc);
  const unsigned long long act = vc->act_acc;
  const unsigned long long psh = vc->push_acc;
  const unsigned long long pend = vc->pend_acc;
  const bool converged = Op::kIsSum ? (resid < vc->eps || pend == 0) : (pend == 0);
  unsigned cont = 0;
  ctl->residual = resid;
  if (converged) {
    ctl->status = 1;
  } else if (static_cast<long long>(vc->rounds) >= vc->max_rounds) {
    ctl->status = 2;
  } else {
    cont = 1;
    ctl->rounds = vc->rounds + 1;
    ctl->activations = vc->activations + act;
    ctl->pushes = vc->pushes + psh;
    // Threshold selected nothing although work remains: lower it (x0.1, to 0)
    // so the run always terminates.
    if (Op::kIsSum && act == 0) ctl->tau = (vc->tau < 1e-300) ? 0.0 : vc->tau * 0.1;
  }
  ctl->resid_acc = 0.0;
  ctl->act_acc = 0;
  ctl->push_acc = 0;
  ctl->pend_acc = 0;
  ctl->ticket = 0;
  // The lists just written are pushed next; the other count set is recycled.
  if (cont) {
    ctl->rset = ws;
    ctl->wset = ws ^ 1u;
    for (int b = 0; b < 4; ++b) ctl->cnt[ws ^ 1u][b] = 0;
  } else {
    for (int b = 0; b < 4; ++b) ctl->cnt[ws][b] = 0;
  }
  __threadfence();
  if (use_cond) cudaGraphSetConditional(cond, cont);
}

// ------------------------------------------------------------------ push

template <class Op, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_push(KArgs<Op> a) {
  using Msg = typename Op::Msg;
  const DevCtl* ctl = a.ctl;
  const unsigned rs = ctl->rset;
  const int cS = static_cast<int>(ctl->cnt[rs][0]);
  const int cM = static_cast<int>(ctl->cnt[rs][1]);
  const int cL = static_cast<int>(ctl->cnt[rs][2]);
  const int lane = threadIdx.x & 31;

  // Large vertices: one CTA each.
  __shared__ Msg s_msg;
  __shared__ int s_beg, s_end;
  for (int i = blockIdx.x; i < cL; i += gridDim.x) {
    if (threadIdx.x == 0) {
      const int j = a.list[2][i];
      const int beg = __ldg(a.rp + j), end = __ldg(a.rp + j + 1);
      s_msg = Op::fold(j, end - beg, a.delta, a.v, a.coef, a.damping);
      s_beg = beg;
      s_end = end;
    }
    __syncthreads();
    const Msg m = s_msg;
    if (Op::live(m)) {
      for (int e = s_beg + threadIdx.x; e < s_end; e += BLOCK) Op::scatter(a.edges, e, m, a.delta);
    }
    __syncthreads();
  }

  const int warp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * BLOCK) >> 5;

  // Medium vertices: one warp each.
  for (int i = warp; i < cM; i += nwarps) {
    Msg m{};
    int beg = 0, end = 0;
    if (lane == 0) {
      const int j = a.list[1][i];
      beg = __ldg(a.rp + j);
      end = __ldg(a.rp + j + 1);
      m = Op::fold(j, end - beg, a.delta, a.v, a.coef, a.damping);
    }
    m = __shfl_sync(0xffffffffu, m, 0);
    beg = __shfl_sync(0xffffffffu, beg, 0);
    end = __shfl_sync(0xffffffffu, end, 0);
    if (Op::live(m)) {
      for (int e = beg + lane; e < end; e += 32) Op::scatter(a.edges, e, m, a.delta);
    }
  }

  // Small vertices: 32 per warp step; their edges are gathered into one
  // index space [0, total) and walked 32 at a time.
  for (int base = warp * 32; base < cS; base += nwarps * 32) {
    const int i = base + lane;
    Msg m{};
    int beg = 0, deg = 0;
    if (i < cS) {
      const int j = a.list[0][i];
      beg = __ldg(a.rp + j);
      deg = __ldg(a.rp + j + 1) - beg;
      m = Op::fold(j, deg, a.delta, a.v, a.coef, a.damping);
      if (!Op::live(m)) deg = 0;
    }
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - deg;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      // owner = number of lanes whose inclusive prefix is <= t
      int owner = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int probe = __shfl_sync(0xffffffffu, incl, owner + step - 1);
        if (probe <= t) owner += step;
      }
      const int ob = __shfl_sync(0xffffffffu, beg, owner);
      const int oe = __shfl_sync(0xffffffffu, excl, owner);
      const Msg om = __shfl_sync(0xffffffffu, m, owner);
      if (t < total) Op::scatter(a.edges, static_cast<int64_t>(ob) + (t - oe), om, a.delta);
    }
  }
}

// ------------------------------------------------------------- utilities

template <class T>
__global__ void k_fill(T* __restrict__ x, int64_t n, T value) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] = value;
}

}  // namespace maiter
