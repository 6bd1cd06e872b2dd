// Persistent asynchronous DAIC (Section 3.2, Eq. 5; Section 5.1).
//
// One launch processes vertices from a device work queue until the queue is
// quiescent.  No CTA ever waits for another at a barrier: warps claim batches
// of queued vertices, update them, and re-enqueue receivers whose delta just
// became worth an update, exactly as Maiter's update thread takes vertices
// from its priority queue while the receive thread accumulates messages.
//
// Queue: a ring of int32 vertex ids (empty slot = -1), monotonic 64-bit head
// (next to claim) and tail (next to reserve), a per-vertex in-queue flag so a
// vertex is queued at most once, and `pending` = vertices reserved in the
// queue or being processed.  pending == 0 means quiescence: nothing queued and
// nothing in flight, so no message can still create work.
//
// Termination of the run (the paper's periodic check, Section 5.1) is an
// exact reduction between launches (k_async_seed): it measures sum |Delta|
// (or the pending count for min) with no update in flight, decides, and seeds
// the next launch with every vertex above the activation threshold.
//
// Every spin is bounded: a wait that sees no progress for timeout_ns on the
// global timer records status 4 (timeout) or 5 (queue slot never freed) and
// returns.  The (v, Delta) state stays a valid DAIC state in that case: no
// taken delta is ever dropped.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_ops.cuh"

namespace maiter {

// The three hot counters sit on cache lines of their own: idle warps poll
// them and every claim and enqueue hits them.
struct AsyncCtl {
  alignas(128) unsigned long long head;   // next queue index to claim
  alignas(128) unsigned long long tail;   // next queue index to reserve
  alignas(128) long long pending;         // reserved + in-flight vertices
  alignas(128) unsigned int ticket;       // last-block election in k_async_seed
  int status;                    // 0 running, 1 converged, 2 epoch cap, 4 timeout, 5 queue full
  double resid_acc;
  unsigned long long pend_acc;
  unsigned long long sel_acc;
  unsigned long long epochs;
  unsigned long long updates;    // vertex updates performed
  unsigned long long pushes;     // messages sent
  double residual;
  double tau;                    // activation threshold (sums)
  double eps;
  long long max_epochs;
  unsigned long long timeout_ns; // longest wait without progress
  int inject_stall;              // testing: one phantom pending item per launch
  int pad;
};

template <class Op>
struct AArgs {
  int n;
  const int* __restrict__ rp;
  EdgeCtx edges;
  const typename Op::C* coef;
  double damping;
  typename Op::V* v;
  typename Op::D* delta;
  int* queue;                    // cap slots
  unsigned long long cap;
  unsigned int* inq;             // n in-queue flags
  AsyncCtl* ctl;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Warp-aggregated enqueue of the lanes with `want` (their flags already
// acquired).  Reserves slots and pending counts first, then writes each id
// into its slot once the slot is empty (bounded wait).
template <class Op>
__device__ __forceinline__ void enqueue_warp(const AArgs<Op>& a, bool want, int k, int lane) {
  const unsigned mask = __ballot_sync(0xffffffffu, want);
  if (!mask) return;
  const int cnt = __popc(mask);
  unsigned long long base = 0;
  if (lane == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.ctl->pending),
              static_cast<unsigned long long>(cnt));
    base = atomicAdd(&a.ctl->tail, static_cast<unsigned long long>(cnt));
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if (want) {
    const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
    volatile int* slot = a.queue + (idx % a.cap);
    if (*slot != -1) {
      const unsigned long long t0 = global_ns();
      while (*slot != -1) {
        if (global_ns() - t0 > a.ctl->timeout_ns) {
          atomicMax(&a.ctl->status, 5);
          return;
        }
        __nanosleep(64);
      }
    }
    *slot = k;
  }
}

// Claims up to kClaim queued indices for the calling warp (processed 32 at a
// time): returns the first index and the count (0 when nothing is claimable
// right now).  Large claims keep the rate of compare-and-swap on head low.
constexpr int kClaim = 128;
__device__ __forceinline__ int claim_warp(AsyncCtl* ctl, unsigned long long* first, int lane) {
  int got = 0;
  unsigned long long h = 0;
  if (lane == 0) {
    volatile AsyncCtl* vc = ctl;
    for (int tries = 0; tries < 64; ++tries) {
      h = vc->head;
      const unsigned long long t = vc->tail;
      if (h >= t) break;
      const unsigned long long take =
          (t - h) < static_cast<unsigned long long>(kClaim) ? (t - h) : kClaim;
      if (atomicCAS(&ctl->head, h, h + take) == h) {
        got = static_cast<int>(take);
        break;
      }
      __nanosleep(32 + (tries & 7) * 16);
    }
  }
  got = __shfl_sync(0xffffffffu, got, 0);
  *first = __shfl_sync(0xffffffffu, h, 0);
  return got;
}

template <class Op, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_async(AArgs<Op> a) {
  using Msg = typename Op::Msg;
  using D = typename Op::D;
  AsyncCtl* ctl = a.ctl;
  volatile AsyncCtl* vc = ctl;
  const int lane = threadIdx.x & 31;
  const double tau = ctl->tau;
  const unsigned long long timeout = ctl->timeout_ns;
  unsigned long long my_updates = 0, my_pushes = 0;
  // idle-wait bookkeeping (lane 0): the wait restarts whenever work moves
  unsigned long long idle_since = 0, seen_head = ~0ull;
  long long seen_pending = -1;
  unsigned backoff = 128;          // idle poll interval (ns), doubled up to 8 us

  for (;;) {
    if (vc->status >= 4) break;
    unsigned long long first;
    const int got = claim_warp(ctl, &first, lane);
    if (got == 0) {
      // Nothing claimable: done if quiescent, else wait (bounded: timeout
      // without any claim or completion anywhere in the grid).
      int quit = 0;
      if (lane == 0) {
        const long long pend = vc->pending;
        const unsigned long long h = vc->head;
        if (pend == 0) {
          quit = 1;
        } else {
          const unsigned long long now = global_ns();
          if (pend != seen_pending || h != seen_head) {
            seen_pending = pend;
            seen_head = h;
            idle_since = now;
          } else if (now - idle_since > timeout) {
            atomicMax(&ctl->status, 4);
            quit = 1;
          }
          if (!quit) {
            __nanosleep(backoff);
            backoff = backoff < 8192u ? backoff * 2u : 8192u;
          }
        }
      }
      if (__shfl_sync(0xffffffffu, quit, 0)) break;
      continue;
    }
    seen_pending = -1;
    backoff = 128;
    for (int sub = 0; sub < got; sub += 32) {
    const int cnt = got - sub < 32 ? got - sub : 32;
    const unsigned long long fsub = first + static_cast<unsigned long long>(sub);
    // Read the claimed ids (a slot may still be in the middle of being written).
    int j = -1;
    if (lane < cnt) {
      volatile int* slot = a.queue + ((fsub + lane) % a.cap);
      int x = *slot;
      if (x == -1) {
        const unsigned long long t0 = global_ns();
        while ((x = *slot) == -1) {
          if (global_ns() - t0 > timeout) { atomicMax(&ctl->status, 4); break; }
          __nanosleep(32);
        }
      }
      j = x;
      if (j >= 0) {
        *slot = -1;
        // Leave the queue before taking the delta, so a message that lands
        // after the take re-enqueues the vertex instead of being stranded.
        atomicExch(a.inq + j, 0u);
        __threadfence();
      }
    }
    // Update: take Delta_j, fold it into v_j (atomically: the vertex may be
    // re-queued and updated by another warp meanwhile), form the message.
    Msg m{};
    int beg = 0, deg = 0;
    if (j >= 0) {
      beg = __ldg(a.rp + j);
      deg = __ldg(a.rp + j + 1) - beg;
      if constexpr (Op::kIsSum) {
        const D d = atomic_take(a.delta + j);
        if (d != D(0)) {
          atomicAdd(a.v + j, static_cast<double>(d));
          const double c = a.coef ? static_cast<double>(a.coef[j])
                                  : (deg ? a.damping / static_cast<double>(deg) : 0.0);
          m = static_cast<Msg>(c * static_cast<double>(d));
        }
      } else {
        const D d = __ldcg(a.delta + j);
        const unsigned int old = atomicMin(a.v + j, d);
        m = (d < old) ? d : kInfU32;
      }
      if (!Op::live(m)) deg = 0;
      else ++my_updates;
    }
    // Walk the batch's edges 32 at a time (prefix sum + owner search).
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - deg;
    my_pushes += deg;
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
      const Msg om = __shfl_sync(0xffffffffu, m, owner);
      bool want = false;
      int k = 0;
      if (t < total) {
        const typename Op::Edge ed = Op::load(a.edges, static_cast<int64_t>(ob) + (t - oe));
        k = ed.k;
        if constexpr (Op::kIsSum) {
          const D old = atomicAdd(a.delta + k, om);
          const double nw = fabs(static_cast<double>(old) + static_cast<double>(om));
          // re-activate when the receiver's delta crosses the threshold
          want = (fabs(static_cast<double>(old)) <= tau) && (nw > tau);
        } else {
          const uint32_t s = om + ed.w;
          const uint32_t nd = (s < om) ? kInfU32 : s;
          if (nd < __ldcg(a.delta + k)) {
            const uint32_t old = atomicMin(a.delta + k, nd);
            // re-activate when the receiver's distance can improve
            want = nd < old && nd < __ldcg(a.v + k);
          }
        }
        if (want) want = atomicExch(a.inq + k, 1u) == 0u;
      }
      enqueue_warp(a, want, k, lane);
    }
    }  // sub-batches
    // The batch is done: its pushes (and the enqueues they caused) are visible.
    __threadfence();
    if (lane == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->pending),
                static_cast<unsigned long long>(-static_cast<long long>(got)));
    }
  }
  my_updates = [&] {
    unsigned long long x = my_updates;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  }();
  my_pushes = [&] {
    unsigned long long x = my_pushes;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  }();
  if (lane == 0) {
    if (my_updates) atomicAdd(&ctl->updates, my_updates);
    if (my_pushes) atomicAdd(&ctl->pushes, my_pushes);
  }
}

// Exact termination check between launches, and the seed of the next one:
// sum |Delta| (or the pending count) over all vertices, then every vertex above
// the threshold enters the queue.  The last block decides (residual < eps,
// epoch cap, or an error status from the last launch) and sets the WHILE
// condition.
template <class Op, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_async_seed(AArgs<Op> a, cudaGraphConditionalHandle cond,
                                                       int use_cond) {
  using D = typename Op::D;
  AsyncCtl* ctl = a.ctl;
  volatile AsyncCtl* vc = ctl;
  const int lane = threadIdx.x & 31;
  const double tau = ctl->tau;
  const bool stop_now = vc->status != 0;
  double rsum = 0.0;
  unsigned long long npend = 0, nsel = 0;
  for (int base = blockIdx.x * BLOCK + (threadIdx.x & ~31); base < a.n; base += gridDim.x * BLOCK) {
    const int j = base + lane;
    bool sel = false;
    if (j < a.n) {
      const D d = a.delta[j];
      const typename Op::V vv = Op::kIsSum ? typename Op::V(0) : a.v[j];
      const bool pend = Op::pending(d, vv);
      npend += pend;
      if (Op::kIsSum) {
        const double p = Op::priority(d, vv);
        rsum += p;
        sel = pend && p > tau;
      } else {
        sel = pend;
      }
    }
    sel = sel && !stop_now;
    if (sel) sel = atomicExch(a.inq + j, 1u) == 0u;
    nsel += sel;
    enqueue_warp(a, sel, j, lane);
  }
  __shared__ double s_r[BLOCK / 32];
  __shared__ unsigned long long s_p[BLOCK / 32], s_s[BLOCK / 32];
  __shared__ int s_last;
  for (int o = 16; o > 0; o >>= 1) {
    rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
    npend += __shfl_xor_sync(0xffffffffu, npend, o);
    nsel += __shfl_xor_sync(0xffffffffu, nsel, o);
  }
  if (lane == 0) { s_r[threadIdx.x >> 5] = rsum; s_p[threadIdx.x >> 5] = npend; s_s[threadIdx.x >> 5] = nsel; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    unsigned long long p = 0, s = 0;
    for (int i = 0; i < BLOCK / 32; ++i) { r += s_r[i]; p += s_p[i]; s += s_s[i]; }
    if (r != 0.0) atomicAdd(&ctl->resid_acc, r);
    if (p) atomicAdd(&ctl->pend_acc, p);
    if (s) atomicAdd(&ctl->sel_acc, s);
    __threadfence();
    s_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  const double resid = Op::kIsSum ? vc->resid_acc : static_cast<double>(vc->pend_acc);
  const unsigned long long pend = vc->pend_acc;
  const unsigned long long sel = vc->sel_acc;
  ctl->residual = resid;
  unsigned cont = 0;
  if (stop_now) {
    // a launch reported a timeout or a full queue: keep its status
  } else if (Op::kIsSum ? (resid < vc->eps || pend == 0) : (pend == 0)) {
    ctl->status = 1;
  } else if (static_cast<long long>(vc->epochs) >= vc->max_epochs) {
    ctl->status = 2;
  } else {
    cont = 1;
    ctl->epochs = vc->epochs + 1;
    // nothing above the threshold although work remains: lower it (x0.1, to 0)
    if (Op::kIsSum && sel == 0) ctl->tau = (vc->tau < 1e-300) ? 0.0 : vc->tau * 0.1;
  }
  ctl->resid_acc = 0.0;
  ctl->pend_acc = 0;
  ctl->sel_acc = 0;
  ctl->ticket = 0;
  // Testing hook: a phantom pending item that nothing will ever complete, so
  // the next launch's idle warps wait until their timeout and report it.
  if (cont && vc->inject_stall) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->pending), 1ull);
  __threadfence();
  if (use_cond) cudaGraphSetConditional(cond, cont);
}

}  // namespace maiter
