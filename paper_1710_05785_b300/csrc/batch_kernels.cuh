// Batched DAIC: many queries (personalised PageRank with + and SSSP with min)
// over several graphs, advanced together round by round inside one CUDA graph.
//
// The unit of work is an item (query, vertex).  Each query owns its own v and
// Delta arrays (query-major layout, one slice per query).  A round:
//   k_b_take - for every item of a high-degree vertex: the update of Eq. 5
//              (take Delta, fold into v, form the message) and its expansion
//              into chunks of kBChunk edges;
//   k_b_push - the scatter of every item: chunks one CTA each, other items
//              warp-gathered 32 at a time.  A receiver whose delta crosses its
//              query's threshold (sum) or whose distance improves (min) is
//              appended to the next round's frontier, so frontiers stay sparse:
//              a query touches only the vertices its messages reach.
// The push kernel's last block swaps the frontiers and sets the graph's WHILE
// condition; the loop ends when no query has an item left.
//
// Termination per query: the frontier of a sum query is empty only when no
// vertex has |Delta| > tau_q, hence sum |Delta| <= n * tau_q = eps_q; a min
// query ends when no distance can improve (exact).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_ops.cuh"

namespace maiter {

constexpr int kBOps = 2;          // 0: sum (FP64), 1: min (uint32)

struct BGraph {
  const int* rp;
  const int* col;
  const uint32_t* w;
  int n;
  int pad;
};

struct BQuery {
  int graph;
  int op;                         // 0 sum, 1 min
  long long off;                  // offset of this query's slice in v / Delta
  double tau;                     // sum: activation threshold eps_q / n
  double damping;                 // sum: d (coefficient d / outdeg)
  double init;                    // sum: Delta1 at each seed, (1 - d) / |S|
};

struct BItem {
  unsigned int q;
  int u;
};

struct BChunk {
  unsigned int q;
  int u;
  int chunk;
  int pad;
  double msg;                     // sum: message; min: the taken distance (as double)
};

struct BCtl {
  unsigned int cnt[2][kBOps][2];  // [set][op][0 general, 1 large]
  unsigned int nchunks;           // chunk entries of the current round
  unsigned int rset, wset;        // set the push reads / appends to
  unsigned int ticket;
  int status;                     // 0 running, 1 done, 2 round cap, 3 overflow
  unsigned int overflow;
  unsigned long long rounds, updates, pushes;
  long long max_rounds;
};

struct BArgs {
  const BGraph* graphs;
  const BQuery* queries;
  double* v_sum;
  double* d_sum;
  uint32_t* v_min;
  uint32_t* d_min;
  unsigned int* stamp;            // min states: round stamp of the last append
  BItem* items[2][kBOps][2];      // [set][op][general / large]
  unsigned int cap[kBOps][2];
  BChunk* chunks;
  unsigned int chunk_cap;
  unsigned int* qlast;            // per query: last round it had items
  BCtl* ctl;
  int cut_large;                  // degree at or above which items are chunked
  int chunk;                      // edges per chunk
};

// Appends the lanes with `want` to the next frontier of op `op`, sorted into
// general / large by the receiver's out-degree (one atomic per list per warp).
__device__ __forceinline__ void b_append(const BArgs& a, unsigned ws, int op, bool want,
                                         unsigned q, int k, int deg_k, int lane) {
  const bool big = deg_k >= a.cut_large;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const bool mine = want && (big == (l == 1));
    const unsigned mask = __ballot_sync(0xffffffffu, mine);
    if (!mask) continue;
    const int leader = __ffs(mask) - 1;
    unsigned pos = 0;
    if (lane == leader) pos = atomicAdd(&a.ctl->cnt[ws][op][l], static_cast<unsigned>(__popc(mask)));
    pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(mask & ((1u << lane) - 1u));
    if (mine) {
      if (pos < a.cap[op][l]) a.items[ws][op][l][pos] = BItem{q, k};
      else atomicOr(&a.ctl->overflow, 1u);
    }
  }
}

// One message over one edge; decides whether the receiver joins the next
// frontier.
__device__ __forceinline__ bool b_apply_sum(const BArgs& a, const BQuery& Q, int k, double m) {
  double* dk = a.d_sum + Q.off + k;
  const double old = atomicAdd(dk, m);
  return fabs(old) <= Q.tau && fabs(old + m) > Q.tau;
}
__device__ __forceinline__ bool b_apply_min(const BArgs& a, const BQuery& Q, int k, uint32_t nd,
                                            unsigned round_stamp) {
  uint32_t* dk = a.d_min + Q.off + k;
  if (!(nd < __ldcg(dk))) return false;
  const uint32_t old = atomicMin(dk, nd);
  if (!(nd < old) || !(nd < __ldcg(a.v_min + Q.off + k))) return false;
  return atomicExch(a.stamp + Q.off + k, round_stamp) != round_stamp;
}

// Update of one item (fold + message).  Returns false if there is nothing to send.
__device__ __forceinline__ bool b_fold(const BArgs& a, int op, const BQuery& Q, int u, int deg,
                                       double* msg_sum, uint32_t* msg_min) {
  if (op == 0) {
    const double d = atomic_take(a.d_sum + Q.off + u);
    if (d == 0.0) return false;
    // an item can be queued twice in one round (it may cross the threshold
    // again after its own update), so the fold into v is atomic
    atomicAdd(a.v_sum + Q.off + u, d);
    if (deg == 0) return false;
    *msg_sum = Q.damping / static_cast<double>(deg) * d;
    return *msg_sum != 0.0;
  }
  const uint32_t d = __ldcg(a.d_min + Q.off + u);
  const uint32_t old = atomicMin(a.v_min + Q.off + u, d);
  if (!(d < old)) return false;
  *msg_min = d;
  return deg > 0;
}

// High-degree items: update once, expand into chunks (count in ctl->nchunks).
template <int BLOCK>
static __global__ void __launch_bounds__(BLOCK) k_b_take(BArgs a) {
  BCtl* ctl = a.ctl;
  const unsigned rs = ctl->rset;
  for (int op = 0; op < kBOps; ++op) {
    const unsigned n = min(ctl->cnt[rs][op][1], a.cap[op][1]);
    for (unsigned i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
      const BItem it = a.items[rs][op][1][i];
      const BQuery Q = a.queries[it.q];
      const BGraph G = a.graphs[Q.graph];
      const int rb = __ldg(G.rp + it.u), deg = __ldg(G.rp + it.u + 1) - rb;
      double ms = 0.0;
      uint32_t mm = 0;
      if (!b_fold(a, op, Q, it.u, deg, &ms, &mm)) continue;
      atomicAdd(&ctl->updates, 1ull);
      const int nc = (deg + a.chunk - 1) / a.chunk;
      const unsigned p0 = atomicAdd(&ctl->nchunks, static_cast<unsigned>(nc));
      if (p0 + static_cast<unsigned>(nc) > a.chunk_cap) {
        atomicOr(&ctl->overflow, 1u);
        continue;
      }
      for (int c = 0; c < nc; ++c)
        a.chunks[p0 + c] = BChunk{it.q, it.u, c, op, op == 0 ? ms : static_cast<double>(mm)};
    }
  }
}

template <int BLOCK>
static __global__ void __launch_bounds__(BLOCK) k_b_push(BArgs a, cudaGraphConditionalHandle cond,
                                                  int use_cond) {
  BCtl* ctl = a.ctl;
  const unsigned rs = ctl->rset, ws = ctl->wset;
  const unsigned stamp = static_cast<unsigned>(ctl->rounds) + 1u;
  const int lane = threadIdx.x & 31;
  unsigned long long my_up = 0, my_push = 0;

  // Chunks of high-degree items: one CTA each.
  const unsigned nch = min(ctl->nchunks, a.chunk_cap);
  for (unsigned i = blockIdx.x; i < nch; i += gridDim.x) {
    const BChunk c = a.chunks[i];
    const BQuery Q = a.queries[c.q];
    const BGraph G = a.graphs[Q.graph];
    const int rb = __ldg(G.rp + c.u), re = __ldg(G.rp + c.u + 1);
    const int beg = rb + c.chunk * a.chunk, end = min(re, beg + a.chunk);
    // the loop runs the same trip count on every warp of the CTA, so the
    // warp-level append inside stays converged
    for (int e0 = beg; e0 < end; e0 += BLOCK) {
      const int e = e0 + static_cast<int>(threadIdx.x);
      bool want = false;
      int k = 0, dk = 0;
      if (e < end) {
        k = __ldcs(G.col + e);
        if (c.pad == 0) {
          want = b_apply_sum(a, Q, k, c.msg);
        } else {
          const uint32_t base = static_cast<uint32_t>(c.msg), wk = __ldcs(G.w + e);
          const uint32_t s = base + wk;
          want = b_apply_min(a, Q, k, s < base ? kInfU32 : s, stamp);
        }
        if (want) dk = __ldg(G.rp + k + 1) - __ldg(G.rp + k);
        if (want) atomicMax(a.qlast + c.q, stamp);
      }
      b_append(a, ws, c.pad, want, c.q, k, dk, lane);
    }
    my_push += (threadIdx.x == 0) ? static_cast<unsigned long long>(end - beg) : 0ull;
  }

  // General items, both ops: 32 per warp step, edges gathered across lanes.
  const int warp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * BLOCK) >> 5;
  for (int op = 0; op < kBOps; ++op) {
    const int n = static_cast<int>(min(ctl->cnt[rs][op][0], a.cap[op][0]));
    for (int base = warp * 32; base < n; base += nwarps * 32) {
      const int i = base + lane;
      unsigned q = 0;
      int u = 0, beg = 0, deg = 0, g = 0;
      double ms = 0.0;
      uint32_t mm = 0;
      if (i < n) {
        const BItem it = a.items[rs][op][0][i];
        q = it.q;
        u = it.u;
        const BQuery Q = a.queries[q];
        g = Q.graph;
        const BGraph G = a.graphs[g];
        beg = __ldg(G.rp + u);
        deg = __ldg(G.rp + u + 1) - beg;
        if (b_fold(a, op, Q, u, deg, &ms, &mm)) ++my_up;
        else deg = 0;
      }
      int incl = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const int excl = incl - deg;
      my_push += static_cast<unsigned long long>(deg);
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int probe = __shfl_sync(0xffffffffu, incl, owner + step - 1);
          if (probe <= t) owner += step;
        }
        const int ob = __shfl_sync(0xffffffffu, beg, owner);
        const int oe = __shfl_sync(0xffffffffu, excl, owner);
        const unsigned oq = __shfl_sync(0xffffffffu, q, owner);
        const double oms = __shfl_sync(0xffffffffu, ms, owner);
        const uint32_t omm = __shfl_sync(0xffffffffu, mm, owner);
        bool want = false;
        int k = 0, dk = 0;
        if (t < total) {
          const BQuery Q = a.queries[oq];
          const BGraph G = a.graphs[Q.graph];
          const int e = ob + (t - oe);
          k = __ldcs(G.col + e);
          if (op == 0) {
            want = b_apply_sum(a, Q, k, oms);
          } else {
            const uint32_t wk = __ldcs(G.w + e), s = omm + wk;
            want = b_apply_min(a, Q, k, s < omm ? kInfU32 : s, stamp);
          }
          if (want) {
            dk = __ldg(G.rp + k + 1) - __ldg(G.rp + k);
            atomicMax(a.qlast + oq, stamp);
          }
        }
        b_append(a, ws, op, want, oq, k, dk, lane);
      }
    }
  }

  // Counters, then the last block closes the round.
  for (int o = 16; o > 0; o >>= 1) {
    my_up += __shfl_xor_sync(0xffffffffu, my_up, o);
    my_push += __shfl_xor_sync(0xffffffffu, my_push, o);
  }
  if (lane == 0) {
    if (my_up) atomicAdd(&ctl->updates, my_up);
    if (my_push) atomicAdd(&ctl->pushes, my_push);
  }
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  volatile BCtl* vc = ctl;
  // large-item updates happen in k_b_take and count there
  unsigned long long next = 0;
  for (int op = 0; op < kBOps; ++op) next += vc->cnt[ws][op][0] + vc->cnt[ws][op][1];
  unsigned cont = 0;
  if (vc->overflow) {
    ctl->status = 3;
  } else if (next == 0) {
    ctl->status = 1;
  } else if (static_cast<long long>(vc->rounds) + 1 >= vc->max_rounds) {
    ctl->status = 2;
  } else {
    cont = 1;
  }
  ctl->rounds = vc->rounds + 1;
  // the lists just read are recycled for the round after next
  for (int op = 0; op < kBOps; ++op) {
    ctl->cnt[rs][op][0] = 0;
    ctl->cnt[rs][op][1] = 0;
  }
  ctl->rset = ws;
  ctl->wset = rs;
  ctl->nchunks = 0;
  ctl->ticket = 0;
  __threadfence();
  if (use_cond) cudaGraphSetConditional(cond, cont);
}

// Initial frontier: the seeds of every query, with Delta1 at each seed
// ((1 - d) / |S| for personalised PageRank, 0 for SSSP; every other delta was
// cleared to the identity on the host).
static __global__ void k_b_seed(BArgs a, const BItem* seeds, int nseeds) {
  const unsigned ws = a.ctl->rset;   // the first push reads the set seeded here
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nseeds;
       base += gridDim.x * blockDim.x) {
    const int i = base + lane;
    bool want = false;
    int op = 0, dk = 0;
    BItem it{0, 0};
    if (i < nseeds) {
      it = seeds[i];
      const BQuery Q = a.queries[it.q];
      const BGraph G = a.graphs[Q.graph];
      op = Q.op;
      if (op == 0) a.d_sum[Q.off + it.u] = Q.init;
      else a.d_min[Q.off + it.u] = 0u;
      dk = __ldg(G.rp + it.u + 1) - __ldg(G.rp + it.u);
      want = true;
    }
    // both ops may appear in one warp: append per op
    for (int o = 0; o < kBOps; ++o) b_append(a, ws, o, want && op == o, it.q, it.u, dk, lane);
  }
}

}  // namespace maiter
