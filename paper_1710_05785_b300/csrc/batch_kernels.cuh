// Batched DAIC: many queries (personalised PageRank with + and SSSP with min)
// over several graphs, advanced together round by round inside one CUDA graph.
//
// The unit of work is an item (query, vertex).  Each query owns its own v and
// Delta arrays (query-major layout, one slice per query).  A round:
//   k_b_take - walks the current frontier once: every item of a vertex with at
//              least cut_large out-edges gets the update of Eq. 5 (take Delta,
//              fold into v, form the message), is split into chunks of `chunk`
//              edges for separate CTAs, and is marked done in the list;
//   k_b_push - the scatter of every item: chunks one CTA each, other items
//              warp-gathered 32 at a time (the query's and graph's fields are
//              loaded once per item and shuffled to the lanes of its edges).
//              A receiver whose delta crosses its query's threshold (sum) or
//              whose distance improves (min) is appended to the next round's
//              frontier, so frontiers stay sparse: a query touches only the
//              vertices its messages reach.
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
  int u;                          // -1: handled by the chunk path this round
};

struct BChunk {
  unsigned int q;
  int u;
  int chunk;
  int op;
  double msg;                     // sum: message; min: the taken distance (as double)
};

struct BCtl {
  unsigned int cnt[2][kBOps];     // [set][op] frontier sizes
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
  BItem* items[2][kBOps];         // [set][op]
  unsigned int cap[kBOps];
  BChunk* chunks;
  unsigned int chunk_cap;
  unsigned int* qlast;            // per query: last round it had items
  BCtl* ctl;
  int cut_large;                  // degree at or above which items are chunked
  int chunk;                      // edges per chunk
};

// Appends the lanes with `want` to the next frontier of op `op` (one atomic
// per warp).
__device__ __forceinline__ void b_append(const BArgs& a, unsigned ws, int op, bool want,
                                         unsigned q, int k, int lane) {
  const unsigned mask = __ballot_sync(0xffffffffu, want);
  if (!mask) return;
  const int leader = __ffs(mask) - 1;
  unsigned pos = 0;
  if (lane == leader) pos = atomicAdd(&a.ctl->cnt[ws][op], static_cast<unsigned>(__popc(mask)));
  pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(mask & ((1u << lane) - 1u));
  if (want) {
    if (pos < a.cap[op]) a.items[ws][op][pos] = BItem{q, k};
    else atomicOr(&a.ctl->overflow, 1u);
  }
}

// One message over one edge; true if the receiver joins the next frontier.
__device__ __forceinline__ bool b_apply_sum(double* d_slice, double tau, int k, double m) {
  const double old = atomicAdd(d_slice + k, m);
  return fabs(old) <= tau && fabs(old + m) > tau;
}
__device__ __forceinline__ bool b_apply_min(uint32_t* d_slice, const uint32_t* v_slice,
                                            unsigned* st_slice, int k, uint32_t nd,
                                            unsigned round_stamp) {
  if (!(nd < __ldcg(d_slice + k))) return false;
  const uint32_t old = atomicMin(d_slice + k, nd);
  if (!(nd < old) || !(nd < __ldcg(v_slice + k))) return false;
  return atomicExch(st_slice + k, round_stamp) != round_stamp;
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

// Items of high-degree vertices: update once, expand into chunks, mark done.
template <int BLOCK>
static __global__ void __launch_bounds__(BLOCK) k_b_take(BArgs a) {
  BCtl* ctl = a.ctl;
  const unsigned rs = ctl->rset;
  unsigned long long ups = 0;
  for (int op = 0; op < kBOps; ++op) {
    const unsigned n = min(ctl->cnt[rs][op], a.cap[op]);
    BItem* list = a.items[rs][op];
    for (unsigned i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
      const BItem it = list[i];
      const BQuery Q = a.queries[it.q];
      const int* rp = a.graphs[Q.graph].rp;
      const int rb = __ldg(rp + it.u), deg = __ldg(rp + it.u + 1) - rb;
      if (deg < a.cut_large) continue;
      list[i].u = -1;
      double ms = 0.0;
      uint32_t mm = 0;
      if (!b_fold(a, op, Q, it.u, deg, &ms, &mm)) continue;
      ++ups;
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
  for (int o = 16; o > 0; o >>= 1) ups += __shfl_xor_sync(0xffffffffu, ups, o);
  if ((threadIdx.x & 31) == 0 && ups) atomicAdd(&ctl->updates, ups);
}

__device__ __forceinline__ unsigned long long shfl64(unsigned long long x, int src) {
  return __shfl_sync(0xffffffffu, x, src);
}

// Warp-gathered scatter of the general items of one op (OP 0 sum, 1 min).
template <int OP>
__device__ __forceinline__ void b_push_items(const BArgs& a, unsigned rs, unsigned ws,
                                             unsigned stamp, int warp, int nwarps, int lane,
                                             unsigned long long* my_up,
                                             unsigned long long* my_push) {
  const int n = static_cast<int>(min(a.ctl->cnt[rs][OP], a.cap[OP]));
  const BItem* list = a.items[rs][OP];
  for (int base = warp * 32; base < n; base += nwarps * 32) {
    const int i = base + lane;
    unsigned q = 0;
    int beg = 0, deg = 0;
    double ms = 0.0, tau = 0.0;
    uint32_t mm = 0;
    unsigned long long off = 0, colp = 0, wp = 0;
    if (i < n) {
      const BItem it = list[i];
      if (it.u >= 0) {
        q = it.q;
        const BQuery Q = a.queries[q];
        const BGraph G = a.graphs[Q.graph];
        beg = __ldg(G.rp + it.u);
        deg = __ldg(G.rp + it.u + 1) - beg;
        off = static_cast<unsigned long long>(Q.off);
        tau = Q.tau;
        colp = reinterpret_cast<unsigned long long>(G.col);
        wp = reinterpret_cast<unsigned long long>(G.w);
        if (b_fold(a, OP, Q, it.u, deg, &ms, &mm)) ++*my_up;
        else deg = 0;
      }
    }
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - deg;
    *my_push += static_cast<unsigned long long>(deg);
    for (int t0 = 0; t0 < total; t0 += 64) {
      // two edge steps in flight: owners, fields and edge loads first
      int k[2];
      uint32_t wk[2];
      int own[2];
      bool ok[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int t = t0 + u * 32 + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int probe = __shfl_sync(0xffffffffu, incl, owner + step - 1);
          if (probe <= t) owner += step;
        }
        own[u] = owner;
        ok[u] = t < total;
        const int ob = __shfl_sync(0xffffffffu, beg, owner);
        const int oe = __shfl_sync(0xffffffffu, excl, owner);
        const int* col = reinterpret_cast<const int*>(shfl64(colp, owner));
        const int e = ob + (t - oe);
        k[u] = ok[u] ? __ldcs(col + e) : 0;
        if (OP == 1) {
          const uint32_t* w = reinterpret_cast<const uint32_t*>(shfl64(wp, owner));
          wk[u] = ok[u] ? __ldcs(w + e) : 0u;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int owner = own[u];
        const unsigned oq = __shfl_sync(0xffffffffu, q, owner);
        const unsigned long long ooff = shfl64(off, owner);
        bool want = false;
        if (OP == 0) {
          const double oms = __shfl_sync(0xffffffffu, ms, owner);
          const double otau = __shfl_sync(0xffffffffu, tau, owner);
          if (ok[u]) want = b_apply_sum(a.d_sum + ooff, otau, k[u], oms);
        } else {
          const uint32_t omm = __shfl_sync(0xffffffffu, mm, owner);
          if (ok[u]) {
            const uint32_t s = omm + wk[u];
            want = b_apply_min(a.d_min + ooff, a.v_min + ooff, a.stamp + ooff, k[u],
                               s < omm ? kInfU32 : s, stamp);
          }
        }
        if (want) atomicMax(a.qlast + oq, stamp);
        b_append(a, ws, OP, want, oq, k[u], lane);
      }
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
    // every warp of the CTA runs the same trip count, so the warp-level
    // append inside stays converged
    for (int e0 = beg; e0 < end; e0 += BLOCK) {
      const int e = e0 + static_cast<int>(threadIdx.x);
      bool want = false;
      int k = 0;
      if (e < end) {
        k = __ldcs(G.col + e);
        if (c.op == 0) {
          want = b_apply_sum(a.d_sum + Q.off, Q.tau, k, c.msg);
        } else {
          const uint32_t base = static_cast<uint32_t>(c.msg), wk = __ldcs(G.w + e);
          const uint32_t s = base + wk;
          want = b_apply_min(a.d_min + Q.off, a.v_min + Q.off, a.stamp + Q.off, k,
                             s < base ? kInfU32 : s, stamp);
        }
        if (want) atomicMax(a.qlast + c.q, stamp);
      }
      b_append(a, ws, c.op, want, c.q, k, lane);
    }
    my_push += (threadIdx.x == 0) ? static_cast<unsigned long long>(end - beg) : 0ull;
  }

  // General items: 32 per warp step, edges gathered across lanes.
  const int warp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * BLOCK) >> 5;
  b_push_items<0>(a, rs, ws, stamp, warp, nwarps, lane, &my_up, &my_push);
  b_push_items<1>(a, rs, ws, stamp, warp, nwarps, lane, &my_up, &my_push);

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
  unsigned long long next = 0;
  for (int op = 0; op < kBOps; ++op) next += vc->cnt[ws][op];
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
  for (int op = 0; op < kBOps; ++op) ctl->cnt[rs][op] = 0;
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
    int op = 0;
    BItem it{0, 0};
    if (i < nseeds) {
      it = seeds[i];
      const BQuery Q = a.queries[it.q];
      op = Q.op;
      if (op == 0) a.d_sum[Q.off + it.u] = Q.init;
      else a.d_min[Q.off + it.u] = 0u;
      want = true;
    }
    // both ops may appear in one warp: append per op
    for (int o = 0; o < kBOps; ++o) b_append(a, ws, o, want && op == o, it.q, it.u, lane);
  }
}

}  // namespace maiter
