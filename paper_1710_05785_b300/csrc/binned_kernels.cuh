// Binned engine for dense rounds of (+) with g_{j,k}(x) = c_j x (PageRank,
// personalised PageRank, Katz): every round delivers the messages of every
// vertex with a pending delta, like the synchronous DAIC of Section 3.2, but
// no edge needs an atomic in L2.  Messages are streamed into destination
// bins and each bin is summed in shared memory - the receive side of Eq. 5
// ("Delta_k <- Delta_k + sum of the messages that reached k") computed one
// block of receivers at a time.
//
// Static layout (built once per graph content, see binned_engine.cu):
//   cell   - 8192 consecutive senders; a cell's out-edges are cut into
//            chunks of at most 65536 edges;
//   bin    - 16384 consecutive receivers (their sums fit shared memory in
//            FP64);
//   segment (chunk c, bin b) - the edges of chunk c whose target lies in bin
//            b, padded to a multiple of 8 entries; a chunk's segments are
//            stored one after another in bin order, chunks one after another,
//            so chunk c owns the slot range [cb[c], cb[c+1]);
//   src_local[slot] - the sender of the edge, relative to its cell
//            (0xFFFF on padding);
//   dst_local[slot] - the receiver, relative to its bin (on padding, a value
//            >= 16384 that differs from its neighbours');
//   T[b][c] - first slot of segment (c, b); T[nbins][c] = cb[c+1], so the
//            segment ends at T[b+1][c].
//
// A round is two kernels:
//   k_bin_scatter - the termination decision (the progress check of Section
//            5.1, on the totals of the round before), then for every chunk:
//            stage the messages msg_v[j] = c_j Delta_j of its cell in shared
//            memory and write msg_e[slot] = msg_v[sender of slot] for every
//            slot - a sequential read of src_local and a sequential write;
//   k_bin_gather - for every bin: sum the messages of its segments into a
//            shared-memory array of 64-bit fixed-point integers (one slot
//            read, one integer atomic per run of equal receivers), then
//            for every receiver k of the bin: fold the delta the messages came
//            from into v_k (v_k <- v_k + Delta_k), store the new delta (the
//            sum), and its message c_k Delta_k for the next round; the FP64
//            residual sum |Delta| of the new deltas feeds the next decision.
// The sums are exact integers: every message is scaled by 2^s, s chosen per
// round so that the round's total message mass E = sum_j deg_j |m_j| (which
// bounds every receiver's sum) stays below 2^62; each message loses only the
// bits below 2^-s (truncation), far below its own FP32 / FP64 ulp.  Integer
// atomics on shared memory are native; floating-point ones are
// compare-and-swap loops on this part.
// Between kernels (v, Delta) is always a complete DAIC state: before the
// gather the messages in msg_e are a function of the pending deltas, which
// are still in Delta; after it they have been delivered and folded.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "daic_kernels.cuh"

namespace maiter {

constexpr int kBinShift = 14;                  // receivers per bin = 2^14
constexpr int kBinSize = 1 << kBinShift;
constexpr int kCellShift = 13;                 // senders per cell = 2^13
constexpr int kCellSize = 1 << kCellShift;
constexpr int kPieceEdges = 65536;             // edges per chunk at most
constexpr int kPad = 8;                        // segment padding (entries)
constexpr unsigned short kPadSrc = 0xFFFF;     // src_local of a padding slot
constexpr int kBinScatterBlock = 512;
constexpr int kBinMaxBins = 16384;             // n <= 2^28

struct BinArgs {
  int n;
  int nbins;
  int nchunks;
  const int* __restrict__ rp;            // n + 1 row offsets
  const void* coef;                      // per-source c_j (CT), or null: damping / outdeg
  double damping;
  double* v;                             // FP64 state
  void* delta;                           // DT[n]
  void* msg_v;                           // MT[n]: c_j Delta_j of every vertex
  void* msg_e;                           // MT[slots]: one message per slot
  void* cmsg;                            // MT[n]: c_j of every sender in the phase's
                                         // message precision (0 without out-edges),
                                         // written by the prime
  const int4* __restrict__ chunks;       // {e_begin, e_end, s_base, s_lo | s_hi << 16}
  const int* __restrict__ cb;            // nchunks + 1 slot offsets
  const int* __restrict__ T;             // (nbins + 1) x nchunks segment starts
  const uint4* __restrict__ src8;        // src_local, 8 per uint4
  const uint4* __restrict__ dst8;        // dst_local, 8 per uint4
  const int* __restrict__ step_base;     // nbins + 1: first group of each bin
  const unsigned* __restrict__ steps;    // per bin, its segments' 8-slot groups
                                         // (first slot / 8)
  DevCtl* ctl;
};

template <class CT>
__device__ __forceinline__ double bin_coef(const BinArgs& a, int j, int deg) {
  return a.coef ? static_cast<double>(static_cast<const CT*>(a.coef)[j])
                : a.damping / static_cast<double>(deg);
}

// Block-wide sum of (resid, act, push, mass) into set `ws` of the control
// block, one atomic per block per total.
template <int BLOCK>
__device__ __forceinline__ void bin_block_totals(DevCtl* ctl, unsigned ws, double resid,
                                                 unsigned long long act,
                                                 unsigned long long push, double mass) {
  __shared__ double s_r[BLOCK / 32], s_m[BLOCK / 32];
  __shared__ unsigned long long s_a[BLOCK / 32], s_p[BLOCK / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  resid = warp_sum(resid);
  mass = warp_sum(mass);
  act = warp_sum(act);
  push = warp_sum(push);
  if (lane == 0) { s_r[wid] = resid; s_m[wid] = mass; s_a[wid] = act; s_p[wid] = push; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, ms = 0.0;
    unsigned long long x = 0, y = 0;
    for (int i = 0; i < BLOCK / 32; ++i) { r += s_r[i]; ms += s_m[i]; x += s_a[i]; y += s_p[i]; }
    if (r != 0.0) atomicAdd(&ctl->resid_acc[ws], r);
    if (ms != 0.0) atomicAdd(&ctl->mass_acc[ws], ms);
    if (x) atomicAdd(&ctl->act_acc[ws], x);
    if (y) atomicAdd(&ctl->push_acc[ws], y);
  }
}

// Fixed point: x * 2^s as a 64-bit integer, truncated toward zero.  The
// scaling multiplies by exact powers of two (split in two factors so that
// each fits the type's exponent range), then one conversion; the caller
// guarantees |x| 2^s < 2^62.
struct BinScale {
  float f1, f2;      // 2^s = f1 f2 (FP32 messages)
  double d;          // 2^s (FP64 messages)
};
__device__ __forceinline__ long long bin_fix(float x, const BinScale& sc) {
  return __float2ll_rz((x * sc.f1) * sc.f2);
}
__device__ __forceinline__ long long bin_fix(double x, const BinScale& sc) {
  return __double2ll_rz(x * sc.d);
}

// The round's scale: E < 2^e (frexp), s = 62 - e, so E 2^s < 2^62; s is
// kept within [-250, 250] (sums below 2^-250 are zero to any precision used).
__device__ __forceinline__ int bin_scale(double mass) {
  if (!(mass > 0.0)) return 0;
  int e = 0;
  frexp(mass, &e);
  return max(-250, min(250, 62 - e));
}
__device__ __forceinline__ BinScale bin_scale_factors(int s) {
  BinScale r;
  const int h = s / 2;
  r.f1 = ldexpf(1.0f, h);
  r.f2 = ldexpf(1.0f, s - h);
  r.d = ldexp(1.0, s);
  return r;
}

// Primes a phase: msg_v[j] = c_j Delta_j for every vertex and the totals of
// Delta (residual, pending count, out-degree sum of pending vertices) into
// the set the next decision reads.  With `wide` (the switch of a mixed run
// from FP64 to FP32 deltas) Delta is first rounded once from the FP64
// warm-up deltas, and the control block is re-armed for the FP32 phase,
// which runs only if the warm-up ended by its residual test.
template <class DT, class MT, class CT>
__global__ void __launch_bounds__(256) k_bin_prime(BinArgs a, const double* __restrict__ wide,
                                                   cudaGraphConditionalHandle cond,
                                                   int use_cond) {
  DevCtl* ctl = a.ctl;
  const unsigned ws = ctl->scan_set;
  DT* delta = static_cast<DT*>(a.delta);
  MT* msg = static_cast<MT*>(a.msg_v);
  double resid = 0.0, mass = 0.0;
  unsigned long long act = 0, push = 0;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < a.n; j += gridDim.x * 256) {
    DT d;
    if (wide) {
      d = static_cast<DT>(wide[j]);
      delta[j] = d;
    } else {
      d = delta[j];
    }
    const int deg = __ldg(a.rp + j + 1) - __ldg(a.rp + j);
    // the coefficient once per phase, in the message precision (an FP64
    // divide per vertex and round would cost more than the round's sums)
    const MT cj = deg > 0 ? static_cast<MT>(bin_coef<CT>(a, j, deg)) : MT(0);
    static_cast<MT*>(a.cmsg)[j] = cj;
    const MT m = (d != DT(0)) ? cj * static_cast<MT>(d) : MT(0);
    msg[j] = m;
    resid += fabs(static_cast<double>(d));
    mass += static_cast<double>(deg) * fabs(static_cast<double>(m));
    act += (d != DT(0));
    push += (d != DT(0)) ? static_cast<unsigned long long>(deg) : 0ull;
  }
  bin_block_totals<256>(ctl, ws, resid, act, push, mass);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->push_set = ws;
    if (wide) {
      const int st = ctl->status;
      ctl->status = (st == 1) ? 0 : st;
      ctl->phase = (st == 1) ? 1 : 0;
      ctl->warm_rounds = ctl->rounds;
      ctl->warm_activations = ctl->activations;
      ctl->warm_pushes = ctl->pushes;
      ctl->switch_frac = 0.0;
      ctl->rounds_in[ws] = ctl->rounds;
      ctl->eps_in[ws] = ctl->eps;
      if (use_cond) cudaGraphSetConditional(cond, st == 1 ? 1u : 0u);
    }
  }
}

// The termination decision of one round, taken by thread 0 of every CTA of
// the scatter on the totals the last gather (or prime) wrote; every CTA
// decides alike, CTA 0 records the decision, clears the other set for the
// next gather and sets the WHILE condition.  Returns 1 to continue, 0 to stop
// (-1: a round after the stopping one in the same pass; nothing is recorded).
__device__ __forceinline__ int bin_decide(DevCtl* ctl, cudaGraphConditionalHandle cond,
                                          int use_cond) {
  if (ctl->status != 0) {
    // stopped before (by this test or by a kernel's error status): the loop ends
    if (blockIdx.x == 0 && use_cond) cudaGraphSetConditional(cond, 0u);
    return -1;
  }
  const unsigned ps = ctl->push_set;
  const double resid = ctl->resid_acc[ps];
  const unsigned long long act = ctl->act_acc[ps], psh = ctl->push_acc[ps];
  const unsigned long long rounds = ctl->rounds_in[ps];
  const double eps_eff = ctl->eps_in[ps];
  const long long max_rounds = ctl->max_rounds;
  const double eps = ctl->eps, switch_frac = ctl->switch_frac;
  double eps_now = eps_eff;
  if (rounds == 0) {
    eps_now = eps;
    if (switch_frac > 0.0 && switch_frac * resid > eps_now) eps_now = switch_frac * resid;
  }
  const bool converged = resid < eps_now || act == 0 || (rounds == 0 && switch_frac >= 1.0);
  int status = 0;
  if (converged) status = 1;
  else if (static_cast<long long>(rounds) >= max_rounds) status = 2;
  const unsigned cont = status == 0;
  if (blockIdx.x == 0) {
    const unsigned ns = ps ^ 1u;
    ctl->residual = resid;
    ctl->rounds_in[ns] = rounds + cont;
    ctl->eps_in[ns] = eps_now;
    if (cont) {
      ctl->rounds = rounds + 1;
      ctl->activations = ctl->activations + act;
      ctl->pushes = ctl->pushes + psh;
    } else {
      ctl->status = status;
    }
    ctl->resid_acc[ns] = 0.0;
    ctl->mass_acc[ns] = 0.0;
    ctl->act_acc[ns] = ctl->push_acc[ns] = ctl->pend_acc[ns] = 0;
    ctl->cnt[ns][0] = 0;                 // the gather's bin ticket
    ctl->scan_set = ns;
    if (use_cond) cudaGraphSetConditional(cond, cont);
  }
  return static_cast<int>(cont);
}

// 8 messages of one slot group, as stored in msg_e.
template <class MT> struct Msg8;
template <> struct Msg8<float> {
  using V = float4;
  static constexpr int kVec = 2;
  float4 x[2];
};
template <> struct Msg8<double> {
  using V = double2;
  static constexpr int kVec = 4;
  double2 x[4];
};

template <class MT>
__device__ __forceinline__ Msg8<MT> load_msg8(const MT* p) {
  using V = typename Msg8<MT>::V;
  Msg8<MT> r;
  const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
  for (int i = 0; i < Msg8<MT>::kVec; ++i) r.x[i] = __ldcs(q + i);
  return r;
}
template <class MT>
__device__ __forceinline__ void store_msg8(MT* p, const Msg8<MT>& r) {
  using V = typename Msg8<MT>::V;
  V* q = reinterpret_cast<V*>(p);
#pragma unroll
  for (int i = 0; i < Msg8<MT>::kVec; ++i) __stcs(q + i, r.x[i]);
}
template <class MT>
__device__ __forceinline__ MT msg8_get(const Msg8<MT>& r, int i) {
  return reinterpret_cast<const MT*>(&r)[i];
}
template <class MT>
__device__ __forceinline__ void msg8_set(Msg8<MT>& r, int i, MT x) {
  reinterpret_cast<MT*>(&r)[i] = x;
}

// Scatter: decision, then msg_e[slot] = msg_v[sender] for every slot.
template <class MT>
__global__ void __launch_bounds__(kBinScatterBlock) k_bin_scatter(BinArgs a,
                                                                  cudaGraphConditionalHandle cond,
                                                                  int use_cond) {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  __shared__ int s_go;
  extern __shared__ __align__(16) unsigned char bin_smem[];
  MT* s_msg = reinterpret_cast<MT*>(bin_smem);      // one cell's messages
  if (threadIdx.x == 0) s_go = bin_decide(a.ctl, cond, use_cond);
  __syncthreads();
  if (s_go <= 0) return;
  const MT* msg_v = static_cast<const MT*>(a.msg_v);
  MT* msg_e = static_cast<MT*>(a.msg_e);
  for (int c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
    const int4 ch = a.chunks[c];
    const int lo = ch.w & 0xFFFF, hi = ch.w >> 16;
    for (int i = lo + threadIdx.x; i <= hi; i += kBinScatterBlock)
      s_msg[i - lo] = msg_v[ch.z + i];
    __syncthreads();
    const int g0 = __ldg(a.cb + c) / kPad, g1 = __ldg(a.cb + c + 1) / kPad;
    // two groups of 8 slots in flight per thread
    for (int g = g0 + threadIdx.x; g < g1; g += 2 * kBinScatterBlock) {
      const int gb = g + kBinScatterBlock;
      const uint4 s0 = __ldcs(a.src8 + g);
      uint4 s1 = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
      if (gb < g1) s1 = __ldcs(a.src8 + gb);
      Msg8<MT> m0, m1;
      const unsigned short* p0 = reinterpret_cast<const unsigned short*>(&s0);
      const unsigned short* p1 = reinterpret_cast<const unsigned short*>(&s1);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        msg8_set(m0, i, p0[i] == kPadSrc ? MT(0) : s_msg[p0[i] - lo]);
        msg8_set(m1, i, p1[i] == kPadSrc ? MT(0) : s_msg[p1[i] - lo]);
      }
      store_msg8(msg_e + static_cast<int64_t>(g) * kPad, m0);
      if (gb < g1) store_msg8(msg_e + static_cast<int64_t>(gb) * kPad, m1);
    }
    __syncthreads();   // s_msg is reloaded for the next chunk
  }
}

constexpr int kBinGatherBlock = 1024;   // one CTA per SM: 128 KB of 64-bit sums

// acc[k] += x on a shared-memory word, as a reduction with no return value,
// addressed in the shared window (a generic-address atomic is slower).
__device__ __forceinline__ void bin_red(unsigned long long* acc, unsigned k, long long x) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(acc + k));
  asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(x) : "memory");
}

// The 8 slots of one group into the bin's sums: receivers of a sorted
// segment ascend, so equal receivers are adjacent and each run of them is
// added with one integer atomic.  Padding slots carry receivers >= kBinSize
// and zero messages: skipped.
template <class MT>
__device__ __forceinline__ void bin_group_add(unsigned long long* acc, const uint4& d,
                                              const Msg8<MT>& m, const BinScale& s) {
  const unsigned short* k = reinterpret_cast<const unsigned short*>(&d);
  unsigned rk = k[0];
  long long run = bin_fix(msg8_get(m, 0), s);
#pragma unroll
  for (int i = 1; i < 8; ++i) {
    const unsigned ki = k[i];
    const long long xi = bin_fix(msg8_get(m, i), s);
    if (ki == rk) {
      run += xi;
    } else {
      if (run != 0 && rk < kBinSize) bin_red(acc, rk, run);
      rk = ki;
      run = xi;
    }
  }
  if (run != 0 && rk < kBinSize) bin_red(acc, rk, run);
}

// Gather: per bin, sum the messages of its segments in shared memory, then
// fold the old deltas into v, store the new deltas and their messages, and
// accumulate the totals of the new deltas for the next decision.  A bin's
// segments are listed as 8-slot groups (built with the layout); each thread
// takes groups, two at a time, with one 16-byte load of receivers and the
// messages' vector loads per group.
template <class DT, class MT, class CT>
__global__ void __launch_bounds__(kBinGatherBlock, 1) k_bin_gather(BinArgs a) {
  constexpr int BLOCK = kBinGatherBlock;
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  DevCtl* ctl = a.ctl;
  if (ctl->status != 0) return;   // after the stopping round of this pass
  const unsigned ws = ctl->scan_set;
  // the messages of this round came from the deltas the set ws ^ 1 measured
  const int s_round = bin_scale(ctl->mass_acc[ws ^ 1u]);
  const BinScale sc = bin_scale_factors(s_round);
  const double unscale = ldexp(1.0, -s_round);
  extern __shared__ __align__(16) unsigned char bin_smem[];
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(bin_smem);
  __shared__ int s_bin;
  for (int k = threadIdx.x; k < kBinSize; k += BLOCK) acc[k] = 0ull;
  DT* delta = static_cast<DT*>(a.delta);
  MT* msg_v = static_cast<MT*>(a.msg_v);
  const MT* msg_e = static_cast<const MT*>(a.msg_e);
  double resid = 0.0, mass = 0.0;
  unsigned long long act = 0, push = 0;
  for (;;) {
    if (threadIdx.x == 0) s_bin = static_cast<int>(atomicAdd(&ctl->cnt[ws][0], 1u));
    __syncthreads();   // also orders the zeroing of acc before the sums
    const int b = s_bin;
    if (b >= a.nbins) break;
    const int q0 = __ldg(a.step_base + b), q1 = __ldg(a.step_base + b + 1);
    int q = q0 + threadIdx.x;
    for (; q + BLOCK < q1; q += 2 * BLOCK) {
      const unsigned g0 = __ldg(a.steps + q), g1 = __ldg(a.steps + q + BLOCK);
      const uint4 d0 = __ldcs(a.dst8 + g0), d1 = __ldcs(a.dst8 + g1);
      const Msg8<MT> m0 = load_msg8(msg_e + static_cast<int64_t>(g0) * kPad);
      const Msg8<MT> m1 = load_msg8(msg_e + static_cast<int64_t>(g1) * kPad);
      bin_group_add<MT>(acc, d0, m0, sc);
      bin_group_add<MT>(acc, d1, m1, sc);
    }
    if (q < q1) {
      const unsigned g0 = __ldg(a.steps + q);
      const uint4 d0 = __ldcs(a.dst8 + g0);
      const Msg8<MT> m0 = load_msg8(msg_e + static_cast<int64_t>(g0) * kPad);
      bin_group_add<MT>(acc, d0, m0, sc);
    }
    __syncthreads();
    const int j0 = b << kBinShift;
    const int cnt = min(kBinSize, a.n - j0);
    for (int k = threadIdx.x; k < cnt; k += BLOCK) {
      const int j = j0 + k;
      const long long x = static_cast<long long>(acc[k]);
      acc[k] = 0ull;
      const DT dnew = static_cast<DT>(static_cast<double>(x) * unscale);
      const DT dold = delta[j];
      if (dold != DT(0)) __stcs(a.v + j, __ldcs(a.v + j) + static_cast<double>(dold));
      delta[j] = dnew;
      const int deg = __ldg(a.rp + j + 1) - __ldg(a.rp + j);
      const MT m = (dnew != DT(0)) ? __ldg(static_cast<const MT*>(a.cmsg) + j) * static_cast<MT>(dnew)
                                   : MT(0);
      msg_v[j] = m;
      resid += fabs(static_cast<double>(dnew));
      mass += static_cast<double>(deg) * fabs(static_cast<double>(m));
      act += (dnew != DT(0));
      push += (dnew != DT(0)) ? static_cast<unsigned long long>(deg) : 0ull;
    }
    // acc is zero again once every thread is past the fold; the next
    // iteration's __syncthreads orders that before its sums
  }
  bin_block_totals<BLOCK>(ctl, ws, resid, act, push, mass);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->push_set = ws;
}

// ---------------------------------------------------------- layout build

// cell[k] = {first edge of cell k, number of its edges}.
static __global__ void k_bin_cells(const int* __restrict__ rp, int64_t n, int ncells,
                                   int2* __restrict__ cell) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncells; k += gridDim.x * blockDim.x) {
    const int64_t s0 = static_cast<int64_t>(k) << kCellShift;
    const int64_t s1 = min(n, s0 + kCellSize);
    cell[k] = make_int2(rp[s0], rp[s1] - rp[s0]);
  }
}

// The senders a chunk's edges come from, relative to its cell: lo = the
// sender of its first edge, hi = of its last (binary search on the offsets).
static __global__ void k_bin_span(const int* __restrict__ rp, int64_t n, int4* chunks,
                                  int nchunks) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
    int4 ch = chunks[c];
    const int s_end = static_cast<int>(min(n, static_cast<int64_t>(ch.z) + kCellSize));
    int src[2];
    const int e_of[2] = {ch.x, ch.y - 1};
    for (int q = 0; q < 2; ++q) {
      // largest j in [s_base, s_end) with rp[j] <= e
      int lo = ch.z, hi = s_end - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= e_of[q]) lo = mid; else hi = mid - 1;
      }
      src[q] = lo - ch.z;
    }
    ch.w = src[0] | (src[1] << 16);
    chunks[c] = ch;
  }
}

// Per chunk: how many of its edges go to each bin, padded, as a prefix over
// the bins: soff[c][b] (b = 0..nbins; soff[c][nbins] = the chunk's padded
// slot count).  One CTA per chunk, the histogram in shared memory.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_bin_hist(const int* __restrict__ col,
                                                    const int4* __restrict__ chunks, int nchunks,
                                                    int nbins, int* __restrict__ soff) {
  extern __shared__ __align__(16) unsigned char bin_smem[];
  int* hist = reinterpret_cast<int*>(bin_smem);
  __shared__ int s_part[BLOCK];
  const int per = (nbins + BLOCK - 1) / BLOCK;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    for (int b = threadIdx.x; b < nbins; b += BLOCK) hist[b] = 0;
    __syncthreads();
    const int4 ch = chunks[c];
    for (int e = ch.x + threadIdx.x; e < ch.y; e += BLOCK) atomicAdd(hist + (col[e] >> kBinShift), 1);
    __syncthreads();
    // exclusive prefix of the padded counts: each thread a run of `per` bins
    const int b0 = threadIdx.x * per;
    int run = 0;
    for (int b = b0; b < min(nbins, b0 + per); ++b) run += (hist[b] + kPad - 1) / kPad * kPad;
    s_part[threadIdx.x] = run;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int i = 0; i < BLOCK; ++i) { const int x = s_part[i]; s_part[i] = t; t += x; }
      soff[static_cast<int64_t>(c) * (nbins + 1) + nbins] = t;
    }
    __syncthreads();
    int o = s_part[threadIdx.x];
    for (int b = b0; b < min(nbins, b0 + per); ++b) {
      soff[static_cast<int64_t>(c) * (nbins + 1) + b] = o;
      o += (hist[b] + kPad - 1) / kPad * kPad;
    }
    __syncthreads();
  }
}

// T[b][c] = cb[c] + soff[c][b] for b = 0..nbins (T[nbins][c] = cb[c+1]).
static __global__ void k_bin_table(const int* __restrict__ soff, const int* __restrict__ cb,
                                   int nchunks, int nbins, int* __restrict__ T) {
  const int64_t total = static_cast<int64_t>(nbins + 1) * nchunks;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(i / nchunks), c = static_cast<int>(i % nchunks);
    T[i] = cb[c] + soff[static_cast<int64_t>(c) * (nbins + 1) + b];
  }
}

// Places every edge of a chunk into its segment: src_local (sender relative
// to the cell) and dst_local (receiver relative to the bin).  One CTA per
// chunk; per-bin cursors and the chunk's row offsets in shared memory.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_bin_place(const int* __restrict__ rp,
                                                     const int* __restrict__ col,
                                                     const int4* __restrict__ chunks, int nchunks,
                                                     int nbins, const int* __restrict__ soff,
                                                     const int* __restrict__ cb,
                                                     unsigned short* __restrict__ src_local,
                                                     unsigned short* __restrict__ dst_local) {
  extern __shared__ __align__(16) unsigned char bin_smem[];
  int* cursor = reinterpret_cast<int*>(bin_smem);
  int* srp = cursor + nbins;   // rp[s_base + lo .. s_base + hi + 1]
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int4 ch = chunks[c];
    const int lo = ch.w & 0xFFFF, hi = ch.w >> 16;
    const int base = cb[c];
    for (int b = threadIdx.x; b < nbins; b += BLOCK)
      cursor[b] = base + soff[static_cast<int64_t>(c) * (nbins + 1) + b];
    for (int i = threadIdx.x; i <= hi - lo + 1; i += BLOCK) srp[i] = rp[ch.z + lo + i];
    __syncthreads();
    for (int e = ch.x + threadIdx.x; e < ch.y; e += BLOCK) {
      // largest i in [0, hi - lo] with srp[i] <= e: the sender is lo + i
      int l = 0, h = hi - lo;
      while (l < h) {
        const int mid = (l + h + 1) >> 1;
        if (srp[mid] <= e) l = mid; else h = mid - 1;
      }
      const int k = col[e];
      const int pos = atomicAdd(cursor + (k >> kBinShift), 1);
      src_local[pos] = static_cast<unsigned short>(lo + l);
      dst_local[pos] = static_cast<unsigned short>(k & (kBinSize - 1));
    }
    __syncthreads();
  }
}

constexpr int kSortMax = 1024;   // longest segment sorted (longer ones stay unsorted)
constexpr int kSortBlock = 256;

// Sorts every segment's slots by receiver (then sender), one warp per
// segment, bitonic in shared memory; padding slots go last.  Segments longer
// than kSortMax are left as placed: the gather is correct on any order, the
// sort only lets it combine messages to the same receiver.
static __global__ void __launch_bounds__(kSortBlock) k_bin_sort(const int* __restrict__ T, int nchunks,
                                                         int nbins,
                                                         unsigned short* __restrict__ src_local,
                                                         unsigned short* __restrict__ dst_local) {
  __shared__ unsigned s_key[kSortBlock / 32][kSortMax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* buf = s_key[wid];
  const int64_t nseg = static_cast<int64_t>(nbins) * nchunks;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (kSortBlock / 32);
  for (int64_t p = blockIdx.x * static_cast<int64_t>(kSortBlock / 32) + wid; p < nseg; p += nw) {
    const int s0 = __ldg(T + p), s1 = __ldg(T + p + nchunks);
    const int L = s1 - s0;
    if (L <= 1 || L > kSortMax) continue;
    int N = 32;
    while (N < L) N <<= 1;
    for (int i = lane; i < N; i += 32) {
      unsigned k = 0xFFFFFFFFu;
      if (i < L) {
        const unsigned sv = src_local[s0 + i], dv = dst_local[s0 + i];
        k = ((dv | (sv == kPadSrc ? 0x8000u : 0u)) << 16) | sv;
      }
      buf[i] = k;
    }
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < N; i += 32) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned x = buf[i], y = buf[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              buf[i] = y;
              buf[ixj] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    for (int i = lane; i < L; i += 32) {
      const unsigned k = buf[i];
      const unsigned sv = k & 0xFFFFu;
      src_local[s0 + i] = static_cast<unsigned short>(sv);
      // padding gets a receiver id of its own outside the bin (its message is
      // zero and never added), so no two padding slots form a run
      dst_local[s0 + i] = static_cast<unsigned short>(
          sv == kPadSrc ? (kBinSize | (i & (kBinSize - 1))) : ((k >> 16) & 0x7FFFu));
    }
    __syncwarp();
  }
}

constexpr int kStepBlock = 1024;

// Per bin: the number of 8-slot groups of its segments (pass 0), then the
// groups' first slots / 8 from the bin's first entry on (pass 1).  One CTA per
// bin.
template <int PASS>
__global__ void __launch_bounds__(kStepBlock) k_bin_steps(const int* __restrict__ T, int nchunks,
                                                          int nbins, int* __restrict__ count,
                                                          const int* __restrict__ step_base,
                                                          unsigned* __restrict__ steps) {
  __shared__ int s_part[kStepBlock];
  const int per = (nchunks + kStepBlock - 1) / kStepBlock;
  for (int b = blockIdx.x; b < nbins; b += gridDim.x) {
    const int* Tb = T + static_cast<int64_t>(b) * nchunks;
    const int* Te = Tb + nchunks;
    const int c0 = threadIdx.x * per, c1 = min(nchunks, c0 + per);
    int run = 0;
    for (int c = c0; c < c1; ++c) run += (Te[c] - Tb[c]) / kPad;
    if (PASS == 0) {
      s_part[threadIdx.x] = run;
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < kStepBlock; ++i) t += s_part[i];
        count[b] = t;
      }
      __syncthreads();
      continue;
    }
    s_part[threadIdx.x] = run;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int i = 0; i < kStepBlock; ++i) { const int x = s_part[i]; s_part[i] = t; t += x; }
    }
    __syncthreads();
    int q = step_base[b] + s_part[threadIdx.x];
    for (int c = c0; c < c1; ++c)
      for (int s0 = Tb[c]; s0 < Te[c]; s0 += kPad) steps[q++] = static_cast<unsigned>(s0 / kPad);
    __syncthreads();
  }
}

}  // namespace maiter
