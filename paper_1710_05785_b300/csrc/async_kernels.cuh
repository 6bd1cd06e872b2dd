// Persistent asynchronous DAIC (Section 3.2, Eq. 5; Section 5.1).
//
// One launch updates vertices until the work is quiescent, with no barrier
// between CTAs: the paper's round-robin workers.  Every CTA owns an
// interleaved share of the vertices (tiles of BLOCK consecutive ids, tile t
// to CTA t mod grid) and sweeps its tiles again and again; in a sweep every
// owned vertex that is pending is updated at once - v_j <- v_j (+) Delta_j by
// its owner alone, so without an atomic - and its messages are scattered
// with fire-and-forget atomics into the receivers' deltas, wherever they
// live.  Messages are accumulated on arrival (the receive thread of Section
// 5.1) and used by the receiver's owner in its next sweep, not in a round:
// no vertex waits for any other.  A vertex of out-degree >= kAsyncBigDeg is
// scattered by its whole CTA.
//
// Quiescence: `busy` counts the CTAs whose last sweep found work (set to the
// grid by the launch before).  A CTA whose sweep finds nothing leaves the
// count; one that finds work again rejoins it; a CTA that reads zero ends.
// A message that lands after its receiver's owner ended is caught by the
// exact check between launches (k_async_seed), which starts another launch,
// so nothing is lost.
//
// Sums update a vertex when |Delta_j| exceeds the launch's threshold theta, a
// fraction of the mean |Delta| the check before measured (never below the
// run's tau): updating on every trickle of mass would send many small
// messages where the synchronous form sends one.  Min updates every pending
// vertex (Delta_j < v_j).
//
// Every spin is bounded: an idle CTA that sees `busy` unchanged for
// timeout_ns records status 4 (timeout) and returns; the (v, Delta) state
// stays a valid DAIC state, since no taken delta is ever dropped.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_ops.cuh"

namespace maiter {

// The hot counter sits on a cache line of its own.
struct AsyncCtl {
  alignas(128) long long busy;            // CTAs whose last sweep found work (+ an injected phantom)
  alignas(128) unsigned int ticket;       // last-block election in k_async_seed
  int status;                    // 0 running, 1 converged, 2 epoch cap, 4 timeout
  double resid_acc;
  unsigned long long pend_acc;
  unsigned long long sel_acc;
  unsigned long long epochs;
  unsigned long long updates;    // vertex updates performed
  unsigned long long pushes;     // messages sent
  unsigned long long sweeps;     // CTA sweeps performed
  double residual;
  double tau;                    // lowest activation threshold (sums)
  double theta;                  // this launch's activation threshold (sums)
  double eps;
  long long max_epochs;
  unsigned long long timeout_ns; // longest wait without progress
  int grid;                      // CTAs of a launch (busy's start value)
  int inject_stall;              // testing: a phantom busy CTA per launch
};

// theta = max(tau, kAsyncMeanFrac x sum |Delta| / n) for a launch of sums.
// Below 1, so the largest |Delta| (at least the mean) exceeds it and every
// launch makes progress (at 1, a state whose deltas are all equal - the
// first one - would select nothing, launch after launch).
constexpr double kAsyncMeanFrac = 0.5;
static_assert(kAsyncMeanFrac < 1.0, "some delta must exceed the launch's threshold");

template <class Op>
struct AArgs {
  int n;
  const int* __restrict__ rp;
  EdgeCtx edges;
  const typename Op::C* coef;
  double damping;
  typename Op::V* v;
  typename Op::D* delta;
  AsyncCtl* ctl;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kAsyncBig = 64;      // high-degree vertices a CTA scatters together per tile
constexpr int kAsyncBigDeg = 1024; // out-degree from which a vertex is scattered by the CTA

// One edge's message: a fire-and-forget atomic into the receiver's delta
// (for min only when it improves the receiver's delta as read just before).
template <class Op>
__device__ __forceinline__ void async_edge(const AArgs<Op>& a, int64_t e, typename Op::Msg m) {
  const typename Op::Edge ed = Op::load(a.edges, e);
  if constexpr (Op::kIsSum) {
    atomicAdd(a.delta + ed.k, m);
  } else {
    const uint32_t s = m + ed.w;
    const uint32_t nd = (s < m) ? kInfU32 : s;
    if (nd < __ldcg(a.delta + ed.k)) atomicMin(a.delta + ed.k, nd);
  }
}

// 1024 threads per SM (four CTAs of 256): more independent sweepers than two
// CTAs of 512 (SSSP at R-MAT scale 20: 7.6 against 9.3 ms per 8 sources) and
// no spills (eight CTAs of 256 at 32 registers spill; 7.1 ms SSSP but 7 %
// slower PageRank).
template <class Op, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_async(AArgs<Op> a) {
  using Msg = typename Op::Msg;
  using D = typename Op::D;
  __shared__ int s_big_j[kAsyncBig];
  __shared__ Msg s_big_m[kAsyncBig];
  __shared__ int s_nbig, s_quit;
  AsyncCtl* ctl = a.ctl;
  volatile AsyncCtl* vc = ctl;
  const int lane = threadIdx.x & 31;
  const double theta = ctl->theta;
  const unsigned long long timeout = ctl->timeout_ns;
  const int ntiles = (a.n + BLOCK - 1) / BLOCK;
  unsigned long long my_updates = 0, my_pushes = 0, my_sweeps = 0;
  // thread 0's view of the CTA: counted in busy or not, and the idle wait's
  // bookkeeping (restarted whenever busy moves)
  bool counted = true;
  long long seen_busy = -1;
  unsigned long long idle_since = 0;
  if (threadIdx.x == 0) s_nbig = 0;
  __syncthreads();

  for (;;) {
    int found = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int j = t * BLOCK + static_cast<int>(threadIdx.x);
      Msg m{};
      int beg = 0, deg = 0;
      if (j < a.n) {
        const D d0 = __ldcg(a.delta + j);
        bool pend;
        if constexpr (Op::kIsSum) pend = fabs(static_cast<double>(d0)) > theta;
        else pend = d0 < a.v[j];
        if (pend) {
          found = 1;
          beg = __ldg(a.rp + j);
          deg = __ldg(a.rp + j + 1) - beg;
          if constexpr (Op::kIsSum) {
            // messages keep arriving: take the delta with an exchange
            const D d = atomic_take(a.delta + j);
            a.v[j] += static_cast<double>(d);   // the owner alone writes v_j
            if (deg) m = Op::message(j, deg, d, a.coef, a.damping);
          } else {
            a.v[j] = d0;   // Delta only falls: d0 < v_j
            m = d0;
          }
          ++my_updates;
          if (!Op::live(m)) {
            deg = 0;
          } else {
            my_pushes += deg;
            if (deg >= kAsyncBigDeg) {
              const int slot = atomicAdd(&s_nbig, 1);
              if (slot < kAsyncBig) {
                s_big_j[slot] = j;
                s_big_m[slot] = m;
                deg = 0;   // the whole CTA scatters it below
              }
            }
          }
        }
      }
      // the warp's vertices' edges, 32 at a time (prefix sum + owner search)
      int incl = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const int excl = incl - deg;
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int tt = t0 + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int probe = __shfl_sync(0xffffffffu, incl, owner + step - 1);
          if (probe <= tt) owner += step;
        }
        const int ob = __shfl_sync(0xffffffffu, beg, owner);
        const int oe = __shfl_sync(0xffffffffu, excl, owner);
        const Msg om = __shfl_sync(0xffffffffu, m, owner);
        if (tt < total) async_edge(a, static_cast<int64_t>(ob) + (tt - oe), om);
      }
      // high-degree vertices of the tile: every thread of the CTA takes edges
      // (one barrier a tile when there are none)
      if (__syncthreads_or(s_nbig > 0)) {
        const int nbig = min(s_nbig, kAsyncBig);
        for (int b = 0; b < nbig; ++b) {
          const int bj = s_big_j[b];
          const Msg bm = s_big_m[b];
          const int e1 = __ldg(a.rp + bj + 1);
          for (int e = __ldg(a.rp + bj) + static_cast<int>(threadIdx.x); e < e1; e += BLOCK)
            async_edge(a, static_cast<int64_t>(e), bm);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nbig = 0;
        __syncthreads();
      }
    }
    // the sweep is over: rejoin or leave the busy count, or end
    const int any = __syncthreads_or(found);
    if (threadIdx.x == 0) {
      ++my_sweeps;
      s_quit = vc->status >= 4;
      if (!s_quit) {
        if (any) {
          if (!counted) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->busy), 1ull);
            counted = true;
          }
          seen_busy = -1;
        } else {
          if (counted) {
            __threadfence();   // this CTA's messages are out before it leaves the count
            atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->busy),
                      static_cast<unsigned long long>(-1ll));
            counted = false;
          }
          const long long b = vc->busy;
          if (b <= 0) {
            s_quit = 1;
          } else {
            const unsigned long long now = global_ns();
            if (b != seen_busy) {
              seen_busy = b;
              idle_since = now;
            } else if (now - idle_since > timeout) {
              atomicMax(&ctl->status, 4);
              s_quit = 1;
            }

          }
        }
      }
    }
    __syncthreads();
    if (s_quit) break;
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
  if (threadIdx.x == 0) atomicAdd(&ctl->sweeps, my_sweeps);
}

// Exact termination check between launches: sum |Delta| (or the pending
// count) over all vertices.  The last block decides (residual < eps, epoch
// cap, or an error status from the last launch), sets the next launch's
// threshold and busy count, and sets the WHILE condition.
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
  for (int j = blockIdx.x * BLOCK + threadIdx.x; j < a.n; j += gridDim.x * BLOCK) {
    const D d = a.delta[j];
    const typename Op::V vv = Op::kIsSum ? typename Op::V(0) : a.v[j];
    const bool pend = Op::pending(d, vv);
    npend += pend;
    if (Op::kIsSum) {
      const double p = Op::priority(d, vv);
      rsum += p;
      nsel += pend && p > tau;
    } else {
      nsel += pend;
    }
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
    // a launch reported a timeout: keep its status
  } else if (Op::kIsSum ? (resid < vc->eps || pend == 0) : (pend == 0)) {
    ctl->status = 1;
  } else if (static_cast<long long>(vc->epochs) >= vc->max_epochs) {
    ctl->status = 2;
  } else {
    cont = 1;
    ctl->epochs = vc->epochs + 1;
    if (Op::kIsSum) {
      // nothing above the lowest threshold although work remains: lower it
      // (x0.1, to 0)
      if (sel == 0) ctl->tau = (vc->tau < 1e-300) ? 0.0 : vc->tau * 0.1;
      const double mean = kAsyncMeanFrac * resid / static_cast<double>(a.n);
      ctl->theta = mean > ctl->tau ? mean : ctl->tau;
    }
  }
  ctl->resid_acc = 0.0;
  ctl->pend_acc = 0;
  ctl->sel_acc = 0;
  ctl->ticket = 0;
  // every CTA of the next launch starts counted; the testing hook adds a
  // phantom that never leaves, so the idle CTAs wait until their timeout
  ctl->busy = static_cast<long long>(vc->grid) + ((cont && vc->inject_stall) ? 1 : 0);
  __threadfence();
  if (use_cond) cudaGraphSetConditional(cond, cont);
}

}  // namespace maiter
