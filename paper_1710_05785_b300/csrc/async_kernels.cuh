// Persistent asynchronous DAIC (Section 3.2, Eq. 5; Section 5.1).
//
// One launch processes vertices until the work is quiescent.  No CTA ever
// waits for another at a barrier: each CTA keeps its own work list in shared
// memory, updates the vertices on it, and puts the receivers whose delta just
// became worth an update on its next list - Maiter's update thread taking
// vertices from its queue while the receive thread accumulates messages, one
// of them per SM.
//
// Per edge the scatter is a fire-and-forget atomic (no returned value); the
// receiver is re-activated from a read of its delta just before: for + when
// that read was at or below the threshold tau and the read plus the message
// is above it, for min when the message improves the read distance and the
// receiver's state.  A per-vertex in-queue flag (exchanged only for those
// candidates) keeps a vertex on at most one list.  A stale read can miss an
// activation; the exact check between launches (k_async_seed) then finds the
// vertex still pending and seeds it again, so nothing is lost.
//
// A global ring of vertex ids (empty slot = -1; monotonic 64-bit head and
// tail) carries the seeds of a launch, the overflow of full local lists and
// the work busy CTAs hand to idle ones.  `busy` counts the CTAs that hold
// work: a CTA raises it before it claims from the ring and lowers it only
// when its lists are empty, after any hand-over, so "ring empty and no CTA
// busy, ring still empty" proves quiescence.
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

// The hot counters sit on cache lines of their own.
struct AsyncCtl {
  alignas(128) unsigned long long head;   // next ring index to claim
  alignas(128) unsigned long long tail;   // next ring index to reserve
  alignas(128) long long busy;            // CTAs holding work (+ an injected phantom)
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
  int inject_stall;              // testing: a phantom busy CTA per launch
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

// Warp-aggregated append of the lanes with `want` to the global ring:
// reserves slots, then writes each id once its slot is empty (bounded wait).
template <class Op>
__device__ __forceinline__ void ring_put_warp(const AArgs<Op>& a, bool want, int k, int lane) {
  const unsigned mask = __ballot_sync(0xffffffffu, want);
  if (!mask) return;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader)
    base = atomicAdd(&a.ctl->tail, static_cast<unsigned long long>(__popc(mask)));
  base = __shfl_sync(0xffffffffu, base, leader);
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
    __threadfence();   // the id is in the ring before this CTA can report itself idle
  }
}

constexpr int kAsyncList = 4096;   // ids per shared-memory work list
constexpr int kAsyncBig = 64;      // high-degree items a CTA scatters together
constexpr int kAsyncBigDeg = 1024; // out-degree from which an item is scattered by the CTA
constexpr int kAsyncClaim = 2048;  // ids claimed from the ring at once
constexpr int kAsyncShare = 512;   // a list longer than this hands half to the ring when it is empty

template <class Op, int BLOCK>
struct AsyncShared {
  int cur[kAsyncList];
  int nxt[kAsyncList];
  int big_j[kAsyncBig];
  typename Op::Msg big_m[kAsyncBig];
  int ncur, nnxt, nbig;
  int quit, got, share;
  unsigned long long first;
};

// Per edge: the scatter (fire-and-forget) and the re-activation test from the
// receiver's delta read just before it.  Returns the receiver to activate or -1.
template <class Op>
__device__ __forceinline__ int async_edge(const AArgs<Op>& a, int64_t e, typename Op::Msg m,
                                          double tau) {
  using D = typename Op::D;
  const typename Op::Edge ed = Op::load(a.edges, e);
  const int k = ed.k;
  bool want = false;
  if constexpr (Op::kIsSum) {
    const D old = __ldcg(a.delta + k);
    atomicAdd(a.delta + k, m);
    const double nw = fabs(static_cast<double>(old) + static_cast<double>(m));
    want = fabs(static_cast<double>(old)) <= tau && nw > tau;
  } else {
    const uint32_t s = m + ed.w;
    const uint32_t nd = (s < m) ? kInfU32 : s;
    if (nd < __ldcg(a.delta + k)) {
      atomicMin(a.delta + k, nd);
      want = nd < __ldcg(a.v + k);
    }
  }
  if (want) want = atomicExch(a.inq + k, 1u) == 0u;
  return want ? k : -1;
}

// Appends the lanes' ids (>= 0) to the next list; what does not fit goes to
// the ring.
template <class Op, int BLOCK>
__device__ __forceinline__ void list_put_warp(const AArgs<Op>& a, AsyncShared<Op, BLOCK>& sh,
                                              int k, int lane) {
  const unsigned mask = __ballot_sync(0xffffffffu, k >= 0);
  if (!mask) return;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&sh.nnxt, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  const int pos = base + __popc(mask & ((1u << lane) - 1u));
  const bool fits = k >= 0 && pos < kAsyncList;
  if (fits) sh.nxt[pos] = k;
  ring_put_warp(a, k >= 0 && !fits, k, lane);
}

template <class Op, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) k_async(AArgs<Op> a) {
  using Msg = typename Op::Msg;
  using D = typename Op::D;
  __shared__ AsyncShared<Op, BLOCK> sh;
  AsyncCtl* ctl = a.ctl;
  volatile AsyncCtl* vc = ctl;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int kWarps = BLOCK / 32;
  const double tau = ctl->tau;
  const unsigned long long timeout = ctl->timeout_ns;
  unsigned long long my_updates = 0, my_pushes = 0;
  // thread 0's view of the CTA: holding work (counted in busy) or not, and
  // the idle wait's bookkeeping (restarted whenever work moves anywhere)
  bool busy = false;
  unsigned long long idle_since = 0, seen_head = ~0ull, seen_tail = ~0ull;
  long long seen_busy = -1;
  unsigned backoff = 128;
  if (threadIdx.x == 0) { sh.ncur = 0; sh.nnxt = 0; sh.nbig = 0; }
  __syncthreads();

  for (;;) {
    // ---- take work: the CTA's list, else a claim from the ring
    if (threadIdx.x == 0) {
      sh.quit = vc->status >= 4;
      sh.got = 0;
      if (!sh.quit && sh.ncur == 0) {
        const unsigned long long t1 = vc->tail, h = vc->head;
        if (h < t1) {
          if (!busy) { atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->busy), 1ull); busy = true; }
          unsigned long long hh = h;
          for (int tries = 0; tries < 64; ++tries) {
            hh = vc->head;
            const unsigned long long t = vc->tail;
            if (hh >= t) break;
            const unsigned long long take =
                (t - hh) < static_cast<unsigned long long>(kAsyncClaim) ? (t - hh) : kAsyncClaim;
            if (atomicCAS(&ctl->head, hh, hh + take) == hh) {
              sh.got = static_cast<int>(take);
              sh.first = hh;
              break;
            }
            __nanosleep(32 + (tries & 7) * 16);
          }
        }
        if (sh.got == 0) {
          if (busy) {
            __threadfence();
            atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->busy),
                      static_cast<unsigned long long>(-1ll));
            busy = false;
          }
          // quiescent: ring empty, no CTA busy, and the ring still empty
          const unsigned long long ta = vc->tail, ha = vc->head;
          __threadfence();
          const long long b = vc->busy;
          __threadfence();
          const unsigned long long tb = vc->tail;
          if (ha == ta && ta == tb && b == 0) {
            sh.quit = 1;
          } else {
            const unsigned long long now = global_ns();
            if (ha != seen_head || ta != seen_tail || b != seen_busy) {
              seen_head = ha;
              seen_tail = ta;
              seen_busy = b;
              idle_since = now;
            } else if (now - idle_since > timeout) {
              atomicMax(&ctl->status, 4);
              sh.quit = 1;
            }
            if (!sh.quit) {
              __nanosleep(backoff);
              backoff = backoff < 8192u ? backoff * 2u : 8192u;
            }
          }
        } else {
          backoff = 128;
          seen_busy = -1;
        }
      }
    }
    __syncthreads();
    if (sh.quit) break;
    if (sh.ncur == 0 && sh.got == 0) continue;
    if (sh.got > 0) {
      // copy the claimed ids (a slot may still be in the middle of being written)
      for (int i = threadIdx.x; i < sh.got; i += BLOCK) {
        volatile int* slot = a.queue + ((sh.first + i) % a.cap);
        int x = *slot;
        if (x == -1) {
          const unsigned long long t0 = global_ns();
          while ((x = *slot) == -1) {
            if (global_ns() - t0 > timeout) { atomicMax(&ctl->status, 4); break; }
            __nanosleep(32);
          }
        }
        *slot = -1;
        sh.cur[i] = x;
      }
      __syncthreads();
      if (threadIdx.x == 0) sh.ncur = sh.got;
      __syncthreads();
    }
    const int ncur = sh.ncur;

    // ---- update the listed vertices, 32 per warp step
    for (int base = wid * 32; base < ncur; base += kWarps * 32) {
      const int i = base + lane;
      int j = -1;
      if (i < ncur) {
        j = sh.cur[i];
        if (j >= 0) {
          // leave the queue before taking the delta, so a message that lands
          // after the take re-activates the vertex instead of being stranded
          atomicExch(a.inq + j, 0u);
          __threadfence();
        }
      }
      Msg m{};
      int beg = 0, deg = 0;
      if (j >= 0) {
        beg = __ldg(a.rp + j);
        deg = __ldg(a.rp + j + 1) - beg;
        if constexpr (Op::kIsSum) {
          const D d = atomic_take(a.delta + j);
          if (d != D(0)) {
            // the vertex can be re-activated and updated on another SM meanwhile
            atomicAdd(a.v + j, static_cast<double>(d));
            if (deg) m = Op::message(j, deg, d, a.coef, a.damping);
          }
        } else {
          const D d = __ldcg(a.delta + j);
          const unsigned int old = atomicMin(a.v + j, d);
          m = (d < old) ? d : kInfU32;
        }
        if (!Op::live(m)) {
          deg = 0;
        } else {
          ++my_updates;
          my_pushes += deg;
          if (deg >= kAsyncBigDeg) {
            const int slot = atomicAdd(&sh.nbig, 1);
            if (slot < kAsyncBig) {
              sh.big_j[slot] = j;
              sh.big_m[slot] = m;
              deg = 0;   // the whole CTA scatters it below
            }
          }
        }
      }
      // walk the edges of the step's vertices 32 at a time (prefix sum + owner search)
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
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int probe = __shfl_sync(0xffffffffu, incl, owner + step - 1);
          if (probe <= t) owner += step;
        }
        const int ob = __shfl_sync(0xffffffffu, beg, owner);
        const int oe = __shfl_sync(0xffffffffu, excl, owner);
        const Msg om = __shfl_sync(0xffffffffu, m, owner);
        const int k = t < total ? async_edge(a, static_cast<int64_t>(ob) + (t - oe), om, tau) : -1;
        list_put_warp(a, sh, k, lane);
      }
    }
    __syncthreads();
    // ---- high-degree vertices: every thread of the CTA takes edges
    const int nbig = min(sh.nbig, kAsyncBig);
    for (int b = 0; b < nbig; ++b) {
      const int j = sh.big_j[b];
      const Msg m = sh.big_m[b];
      const int beg = __ldg(a.rp + j), end = __ldg(a.rp + j + 1);
      for (int e0 = beg; e0 < end; e0 += BLOCK) {
        const int e = e0 + static_cast<int>(threadIdx.x);
        const int k = e < end ? async_edge(a, static_cast<int64_t>(e), m, tau) : -1;
        list_put_warp(a, sh, k, lane);
      }
    }
    __syncthreads();
    // ---- the next list becomes the current one; a long list hands half of
    // its ids to the ring when the ring is empty, so idle CTAs get work
    if (threadIdx.x == 0) sh.share = min(sh.nnxt, kAsyncList) > kAsyncShare && vc->head >= vc->tail;
    __syncthreads();
    int nn = min(sh.nnxt, kAsyncList);
    if (sh.share) {
      const int keep = nn / 2;
      for (int i0 = keep; i0 < nn; i0 += BLOCK) {
        const int i = i0 + static_cast<int>(threadIdx.x);
        ring_put_warp(a, i < nn, i < nn ? sh.nxt[i] : 0, lane);
      }
      nn = keep;
    }
    for (int i = threadIdx.x; i < nn; i += BLOCK) sh.cur[i] = sh.nxt[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      sh.ncur = nn;
      sh.nnxt = 0;
      sh.nbig = 0;
    }
    __syncthreads();
  }
  // leaving with work would break the quiescence count; only a timeout or a
  // full ring gets here with busy still held (the launch is failed then)
  if (threadIdx.x == 0 && busy)
    atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->busy),
              static_cast<unsigned long long>(-1ll));
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
// the threshold enters the ring.  The last block decides (residual < eps,
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
    ring_put_warp(a, sel, j, lane);
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
    // a launch reported a timeout or a full ring: keep its status
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
  // Testing hook: a phantom busy CTA that never finishes, so the next
  // launch's idle CTAs wait until their timeout and report it.
  if (cont && vc->inject_stall) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->busy), 1ull);
  __threadfence();
  if (use_cond) cudaGraphSetConditional(cond, cont);
}

}  // namespace maiter
