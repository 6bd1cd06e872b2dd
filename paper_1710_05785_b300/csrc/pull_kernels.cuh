// Receive-side engine for dense rounds of (+) with g_{j,k}(x) = c_j x
// (PageRank, personalised PageRank, Katz): in a round of the synchronous
// DAIC (Section 3.2) in which every vertex with a pending delta sends, the
// receive step of Eq. 5, Delta_k <- Delta_k + sum of the messages that
// reached k, is computed at the receiver: k reads the messages c_j Delta_j
// of its in-neighbours j through the transpose of the graph and sums them in
// registers.  No edge needs an atomic; per edge the round reads one sender
// rank (streamed) and one message (a random read of an array with one entry
// per sender, which stays in L2).
//
// Static layout (pull_engine.cu, once per graph content):
//   crp, csrc - the transpose in CSR form: the senders of every receiver;
//   receivers in groups of 32 consecutive vertices, one warp each: the
//     in-edges of a group's rows are contiguous and each carries its row
//     within the group (one byte); every lane takes 4 consecutive edges per
//     step (one 16-byte load of senders, one 4-byte load of rows), sums the
//     runs of equal rows among them in registers, and one segmented shuffle
//     scan over the lanes joins the runs that cross lanes;
//   rows with more in-edges than the layout's cut keep their edges in a tail
//     region after all the others (each row's part starting at a multiple of
//     4 slots) and are cut into chunks of the layout's chunk size, one warp
//     each: the warp's sum goes to an FP64 accumulator of the row by one
//     atomic, and the warp that adds the row's last chunk folds the row;
//   message slots: a round's messages are stored by sender rank (the
//     vertices of out-degree > 0 in id order; in R-MAT graphs about half of
//     all vertices), so that the two message arrays of a round, the one read
//     at random and the one written, stay in L2 together; a vertex's rank is
//     the count of senders before its word of 32 rows (sbase) plus the bits
//     below it in the word's sender mask (smask).
// A round is two kernels: k_pull_decide (one thread: the termination test of
// Section 5.1 on the totals of the round before, shared with the binned
// engine) and k_pull (sum, then fold: v_k <- v_k + Delta_k, Delta_k <- sum,
// message c_k Delta_k for the next round, and the totals of the new deltas).
// Messages alternate between two buffers by the control block's set: a round
// reads msg[ws ^ 1] and writes msg[ws].
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "binned_kernels.cuh"

namespace maiter {

constexpr int kPullBlock = 256;
// resident CTAs per SM the register budget allows (40 registers a thread for
// FP32 messages, 64 for FP64 ones)
template <class MT>
constexpr int pull_min_blocks() { return sizeof(MT) == 4 ? 6 : 4; }
// A layout's cut (in-edges of the largest row a group sums) and chunk (in-edges
// per chunk of a larger row) are parameters of its build: the scalar round
// (k_pull) sums rows of up to 2048 in-edges in groups and splits larger
// ones into 4096-edge chunks; the 64-query vector round (k_vec_pull, a warp
// per row) takes rows past 256 in-edges in 1024-edge chunks, spread over
// many warps.
constexpr int kPullCut = 2048;
constexpr int kPullChunk = 4096;
constexpr int kVecCut = 256;
constexpr int kVecChunk = 1024;
constexpr int kPullSteps = 2;       // 128-edge steps of a group whose loads are issued together
constexpr int kPullLargeSteps = 2;  // 128-edge steps of a chunk whose loads are issued together

struct PullArgs {
  int n;
  int ngroups;                            // ceil(n / 32)
  int nlarge;                             // chunk entries of the large rows
  const int* __restrict__ rp;             // out-edge offsets (out-degrees)
  const int* __restrict__ crp;            // n + 1: in-edge offsets of the small rows (a
                                          // large row has none here: its edges are in
                                          // the tail, reached through its chunks)
  const int* __restrict__ csrc;           // sender rank of every in-edge
  const unsigned char* __restrict__ crow; // m: row of every small-row in-edge within its
                                          // group of 32 (k mod 32)
  const unsigned* __restrict__ lbits;     // ceil(n / 32): bit k mod 32 of word k / 32 set
                                          // when row k is large
  const int4* __restrict__ large;         // {row, first edge, end edge, large row index}
  const int* __restrict__ large_nch;      // chunks of every large row
  double* lacc;                           // FP64 sum of every large row (zero between rounds)
  unsigned* lcnt;                         // chunks of every large row added this round
  const void* coef;                       // per-source c_j (CT), or null: damping / outdeg
  double damping;
  double* v;                              // FP64 state
  void* delta;                            // DT[n]
  void* msg[2];                           // MT[nsend] each: c_j Delta_j by sender rank,
                                          // alternating by set
  const int* __restrict__ sbase;          // ceil(n / 32): senders before every word of 32 rows
  const unsigned* __restrict__ smask;     // ceil(n / 32): bit r set when row 32 w + r sends
  void* cmsg;                             // MT[n]: c_j in the message precision (prime)
  DevCtl* ctl;
};

// Message slot of sender k (out-degree > 0): its rank among the senders.
__device__ __forceinline__ int sender_index(const int* __restrict__ sbase,
                                            const unsigned* __restrict__ smask, int k) {
  return __ldg(sbase + (k >> 5)) + __popc(__ldg(smask + (k >> 5)) & ((1u << (k & 31)) - 1u));
}

// Primes a phase: msg[ws][j] = c_j Delta_j and the totals of Delta into set
// ws (as k_bin_prime, with the message buffer of the set).
template <class DT, class MT, class CT>
__global__ void __launch_bounds__(256) k_pull_prime(PullArgs a, const double* __restrict__ wide,
                                                    cudaGraphConditionalHandle cond,
                                                    int use_cond) {
  DevCtl* ctl = a.ctl;
  const unsigned ws = ctl->scan_set;
  DT* delta = static_cast<DT*>(a.delta);
  MT* msg = static_cast<MT*>(a.msg[ws]);
  MT* cmsg = static_cast<MT*>(a.cmsg);
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
    double c = 0.0;
    if (deg > 0)
      c = a.coef ? static_cast<double>(static_cast<const CT*>(a.coef)[j])
                 : a.damping / static_cast<double>(deg);
    const MT cj = static_cast<MT>(c);
    cmsg[j] = cj;
    const MT m = (d != DT(0)) ? cj * static_cast<MT>(d) : MT(0);
    if (deg > 0) msg[sender_index(a.sbase, a.smask, j)] = m;
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

// The round's termination decision (one thread), then the WHILE condition.
static __global__ void k_pull_decide(DevCtl* ctl, cudaGraphConditionalHandle cond, int use_cond) {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  if (threadIdx.x == 0) bin_decide(ctl, cond, use_cond);
}

// Fold of receiver k with its new delta: v_k += Delta_k (old), Delta_k =
// sum, its message for the next round, and its share of the totals.
template <class DT, class MT>
__device__ __forceinline__ void pull_fold(const PullArgs& a, MT* msg_out, int k, double sum,
                                          double& resid, double& mass, unsigned long long& act,
                                          unsigned long long& push) {
  DT* delta = static_cast<DT*>(a.delta);
  const DT dnew = static_cast<DT>(sum);
  const DT dold = delta[k];
  if (dold != DT(0)) a.v[k] += static_cast<double>(dold);
  delta[k] = dnew;
  const int deg = __ldg(a.rp + k + 1) - __ldg(a.rp + k);
  const MT m = (dnew != DT(0)) ? __ldg(static_cast<const MT*>(a.cmsg) + k) * static_cast<MT>(dnew)
                               : MT(0);
  if (deg > 0) msg_out[sender_index(a.sbase, a.smask, k)] = m;
  resid += fabs(static_cast<double>(dnew));
  mass += static_cast<double>(deg) * fabs(static_cast<double>(m));
  act += (dnew != DT(0));
  push += (dnew != DT(0)) ? static_cast<unsigned long long>(deg) : 0ull;
}

__device__ __forceinline__ int int4_at(const int4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// One step of a group's warp over 128 slots, 4 consecutive ones per lane,
// k[i] the row of slot i within the group (-1 before the group's first
// edge, 32 from its end on: never written) and x[i] its message.  Rows are
// non-decreasing along the slots, so a row's slots are contiguous: within a
// lane, a run that is neither the lane's first (head) nor its last (tail)
// run lies in this lane alone and is added to its row at once; the head runs
// of lanes with the same first row are joined by a segmented suffix scan,
// and the first lane of such a segment also takes the tail of the lane
// before it when that tail is the same row.  Every row is added to by at
// most one lane per step.
template <class MT>
__device__ __forceinline__ void pull_group_step(MT* s_row, int lane, const int (&k)[4],
                                                const MT (&x)[4]) {
  MT head = MT(0), run = x[0];
  int rk = k[0];
  bool split = false;
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    if (k[i] != rk) {
      if (!split) head = run;
      else if (rk >= 0 && rk < 32) s_row[rk] += run;   // a run inside the lane
      split = true;
      run = x[i];
      rk = k[i];
    } else {
      run += x[i];
    }
  }
  if (!split) head = run;
  const MT tail = split ? run : MT(0);
  const int f = k[0], l = k[3];
  MT hv = head;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const MT y = __shfl_down_sync(0xffffffffu, hv, o);
    const int fy = __shfl_down_sync(0xffffffffu, f, o);
    if (lane + o < 32 && fy == f) hv += y;
  }
  const int fprev = __shfl_up_sync(0xffffffffu, f, 1);
  const int lprev = __shfl_up_sync(0xffffffffu, l, 1);
  const MT tprev = __shfl_up_sync(0xffffffffu, tail, 1);
  const int fnext = __shfl_down_sync(0xffffffffu, f, 1);
  if (lane == 0 || fprev != f) {
    if (lane > 0 && lprev == f) hv += tprev;
    if (f >= 0 && f < 32) s_row[f] += hv;
  }
  if (split && (lane == 31 || fnext != l) && l >= 0 && l < 32) s_row[l] += tail;
}

// One dense round: the large rows' chunks, then the groups of 32 rows, a
// warp each (no block barrier).  Sums in the message precision within a
// step, in MT per row across steps (FP64 across the large rows' chunks).
// The edge streams are read once a round: evict-first in L2 (__ldcs), so
// they do not push the message array (read at random) out of it.
template <class DT, class MT>
__global__ void __launch_bounds__(kPullBlock, pull_min_blocks<MT>()) k_pull(PullArgs a) {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  DevCtl* ctl = a.ctl;
  if (ctl->status != 0) return;   // the decision stopped the run
  const unsigned ws = ctl->scan_set;
  const MT* __restrict__ msg_in = static_cast<const MT*>(a.msg[ws ^ 1u]);
  MT* msg_out = static_cast<MT*>(a.msg[ws]);
  double resid = 0.0, mass = 0.0;
  unsigned long long act = 0, push = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ MT s_row[kPullBlock / 32][32];   // a group's row sums, one warp each
  const int gw = blockIdx.x * (kPullBlock / 32) + wid;
  const int nw = gridDim.x * (kPullBlock / 32);

  // large rows: a warp per chunk (its first slot a multiple of 4), the
  // chunk's sum added to the row's FP64 accumulator by one atomic; the warp
  // that adds the last chunk folds the row
  for (int c = gw; c < a.nlarge; c += nw) {
    const int4 ent = __ldg(a.large + c);
    MT x[4] = {MT(0), MT(0), MT(0), MT(0)};
    for (int e0 = ent.y + 4 * lane; e0 < ent.z; e0 += 128 * kPullLargeSteps) {
      int4 src[kPullLargeSteps];
#pragma unroll
      for (int u = 0; u < kPullLargeSteps; ++u) {
        const int e = e0 + 128 * u;
        src[u] = e < ent.z ? __ldcs(reinterpret_cast<const int4*>(a.csrc + e)) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < kPullLargeSteps; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (e0 + 128 * u + i < ent.z) x[i] += msg_in[int4_at(src[u], i)];
    }
    double t = static_cast<double>(x[0]) + static_cast<double>(x[1]) +
               static_cast<double>(x[2]) + static_cast<double>(x[3]);
    t = warp_sum(t);
    int last = 0;
    if (lane == 0) {
      atomicAdd(a.lacc + ent.w, t);
      __threadfence();
      last = atomicAdd(a.lcnt + ent.w, 1u) == static_cast<unsigned>(__ldg(a.large_nch + ent.w)) - 1u;
      if (last) {
        __threadfence();
        const double sum = __longlong_as_double(static_cast<long long>(
            atomicExch(reinterpret_cast<unsigned long long*>(a.lacc + ent.w), 0ull)));
        a.lcnt[ent.w] = 0u;
        pull_fold<DT, MT>(a, msg_out, ent.x, sum, resid, mass, act, push);
      }
    }
  }

  // groups of 32 rows, one warp each: the small rows' in-edges of a group
  // are contiguous, each tagged with its row; a step covers 128 slots from a
  // multiple of 4 at or below the group's first edge
  for (int gi = gw; gi < a.ngroups; gi += nw) {
    const int k = gi * 32 + lane;
    const int gb = __ldg(a.crp + gi * 32);
    const int ge = __ldg(a.crp + min(gi * 32 + 32, a.n));
    s_row[wid][lane] = MT(0);
    __syncwarp();
    for (int e0 = (gb & ~3) + 4 * lane; e0 - 4 * lane < ge; e0 += 128 * kPullSteps) {
      int4 src[kPullSteps];
      unsigned tag[kPullSteps];
#pragma unroll
      for (int h = 0; h < kPullSteps; ++h) {
        const int e = e0 + 128 * h;
        const bool in = e < ge;
        src[h] = in ? __ldcs(reinterpret_cast<const int4*>(a.csrc + e)) : make_int4(0, 0, 0, 0);
        tag[h] = in ? __ldcs(reinterpret_cast<const unsigned*>(a.crow + e)) : 0u;
      }
      MT x[kPullSteps][4];
      int r[kPullSteps][4];
#pragma unroll
      for (int h = 0; h < kPullSteps; ++h)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = e0 + 128 * h + i;
          r[h][i] = e < gb ? -1 : (e >= ge ? 32 : static_cast<int>((tag[h] >> (8 * i)) & 0xffu));
          x[h][i] = (e >= gb && e < ge) ? msg_in[int4_at(src[h], i)] : MT(0);
        }
#pragma unroll
      for (int h = 0; h < kPullSteps; ++h) {
        pull_group_step<MT>(s_row[wid], lane, r[h], x[h]);
        __syncwarp();
      }
    }
    const MT acc = s_row[wid][lane];
    __syncwarp();   // s_row is reset by the warp's next group
    const bool large = (__ldg(a.lbits + gi) >> lane) & 1u;
    if (k < a.n && !large)
      pull_fold<DT, MT>(a, msg_out, k, static_cast<double>(acc), resid, mass, act, push);
  }
  bin_block_totals<kPullBlock>(ctl, ws, resid, act, push, mass);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->push_set = ws;
}

// ---------------------------------------------------------- layout build

// ------------------------------------------------ layout build (device)
// The layout's four counts of row k: small-row in-edges, tail in-edges,
// chunks and large rows (one), scanned together as an int4 over the rows in
// three passes: tile totals, a scan of the tile totals (one CTA), and the
// tiles' own scans, which write the offsets.
constexpr int kPullScanBlock = 256;
constexpr int kPullScanItems = 8;
constexpr int kPullScanTile = kPullScanBlock * kPullScanItems;   // rows per tile

__device__ __forceinline__ int4 pull_counts(int d, int cut, int chunk) {
  const bool big = d > cut;
  return make_int4(big ? 0 : d, big ? (d + 3) & ~3 : 0, big ? (d + chunk - 1) / chunk : 0,
                   big ? 1 : 0);
}
__device__ __forceinline__ int4 add4(int4 a, int4 b) {
  return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ int4 shfl_up4(int4 v, int o) {
  return make_int4(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o),
                   __shfl_up_sync(0xffffffffu, v.z, o), __shfl_up_sync(0xffffffffu, v.w, o));
}
// Inclusive block scan of one int4 per thread; returns the block total too.
__device__ __forceinline__ int4 block_scan4(int4 v, int4* total) {
  __shared__ int4 s_w[kPullScanBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int4 t = shfl_up4(v, o);
    if (lane >= o) v = add4(v, t);
  }
  if (lane == 31) s_w[wid] = v;
  __syncthreads();
  int4 off = make_int4(0, 0, 0, 0), tot = make_int4(0, 0, 0, 0);
  for (int w = 0; w < kPullScanBlock / 32; ++w) {
    if (w < wid) off = add4(off, s_w[w]);
    tot = add4(tot, s_w[w]);
  }
  __syncthreads();   // s_w is reused by the caller's next scan
  *total = tot;
  return add4(v, off);
}

// Pass 1: every tile's total.
static __global__ void __launch_bounds__(kPullScanBlock) k_pull_tile_sums(const int* __restrict__ indeg,
                                                                          int n, int cut, int chunk,
                                                                          int4* __restrict__ sums) {
  const int base = blockIdx.x * kPullScanTile + threadIdx.x * kPullScanItems;
  int4 v = make_int4(0, 0, 0, 0);
#pragma unroll
  for (int i = 0; i < kPullScanItems; ++i)
    if (base + i < n) v = add4(v, pull_counts(__ldg(indeg + base + i), cut, chunk));
  int4 tot;
  block_scan4(v, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Pass 2 (one CTA): exclusive scan of the tile totals in place, and the
// grand total in sums[ntiles].
static __global__ void __launch_bounds__(kPullScanBlock) k_pull_scan_sums(int4* sums, int ntiles) {
  int4 carry = make_int4(0, 0, 0, 0);
  for (int b0 = 0; b0 < ntiles; b0 += kPullScanBlock) {
    const int b = b0 + threadIdx.x;
    const int4 v = b < ntiles ? sums[b] : make_int4(0, 0, 0, 0);
    int4 tot;
    const int4 inc = block_scan4(v, &tot);
    if (b < ntiles) sums[b] = add4(carry, make_int4(inc.x - v.x, inc.y - v.y, inc.z - v.z, inc.w - v.w));
    carry = add4(carry, tot);
  }
  if (threadIdx.x == 0) sums[ntiles] = carry;
}

// Pass 3: each tile's scan from its offset: crp (small-row offsets), the
// first slot of every row (its crp, or its tail offset after all small-row
// edges), the large-row flags and, for every large row, its chunk entries.
static __global__ void __launch_bounds__(kPullScanBlock) k_pull_offsets(
    const int* __restrict__ indeg, int n, int cut, int chunk, const int4* __restrict__ sums, int ntiles,
    int* __restrict__ crp, int* __restrict__ first, unsigned* __restrict__ lbits,
    int4* __restrict__ large, int* __restrict__ large_nch) {
  const int base = blockIdx.x * kPullScanTile + threadIdx.x * kPullScanItems;
  int d[kPullScanItems];
  int4 v = make_int4(0, 0, 0, 0);
#pragma unroll
  for (int i = 0; i < kPullScanItems; ++i) {
    d[i] = base + i < n ? __ldg(indeg + base + i) : 0;
    v = add4(v, pull_counts(d[i], cut, chunk));
  }
  int4 tot;
  const int4 inc = block_scan4(v, &tot);
  const int4 tile_off = sums[blockIdx.x];
  const int small_total = sums[ntiles].x;
  const int tail_base = (small_total + 3) & ~3;   // the tail's rows start at multiples of 4
  int4 run = add4(tile_off, make_int4(inc.x - v.x, inc.y - v.y, inc.z - v.z, inc.w - v.w));
  unsigned flags = 0u;
#pragma unroll
  for (int i = 0; i < kPullScanItems; ++i) {
    const int k = base + i;
    if (k >= n) break;
    const int4 c = pull_counts(d[i], cut, chunk);
    crp[k] = run.x;
    if (c.w) {
      flags |= 1u << i;
      const int tail = tail_base + run.y;
      first[k] = tail;
      large_nch[run.w] = c.z;
      for (int q = 0; q < c.z; ++q)
        large[run.z + q] = make_int4(k, tail + q * chunk, tail + min(d[i], (q + 1) * chunk), run.w);
    } else {
      first[k] = run.x;
    }
    run = add4(run, c);
  }
  if (base < n && base + kPullScanItems >= n) crp[n] = small_total;   // the thread of the last row
  // 32 consecutive rows = 4 threads' flags
  const int lane = threadIdx.x & 31;
  const unsigned sh = (lane & 3) * kPullScanItems;
  unsigned w = flags << sh;
  w |= __shfl_down_sync(0xffffffffu, w, 1);
  w |= __shfl_down_sync(0xffffffffu, w, 2);
  if ((lane & 3) == 0 && base < n) lbits[base >> 5] = w;
}

// In-degree of every vertex (cnt zeroed by the caller).
static __global__ void k_pull_indegree(const int* __restrict__ col, int64_t m, int* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicAdd(cnt + __ldg(col + e), 1);
}

// In-edge placement: csrc[cursor[k]++] = the rank of sender j for every
// edge j -> k (cursor starts at row k's first slot, in the small-row region
// or in the tail), and the slot's row within its group.
// A warp per sender, its lanes over the sender's out-edges (a sender of high
// out-degree is not one thread's loop).
static __global__ void k_pull_place(const int* __restrict__ rp, const int* __restrict__ col, int n,
                                    const int* __restrict__ sbase, const unsigned* __restrict__ smask,
                                    int* __restrict__ cursor, int* __restrict__ csrc,
                                    unsigned char* __restrict__ crow) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = w0; j < n; j += nw) {
    const int e0 = __ldg(rp + j), e1 = __ldg(rp + j + 1);
    if (e1 == e0) continue;
    const int tag = sender_index(sbase, smask, j);
    for (int e = e0 + lane; e < e1; e += 32) {
      const int k = __ldg(col + e);
      const int pos = atomicAdd(cursor + k, 1);
      csrc[pos] = tag;
      crow[pos] = static_cast<unsigned char>(k & 31);
    }
  }
}

// Sender masks and ranks: smask[w] bit r set when row 32 w + r has
// out-edges; sbase[w] the senders in words before w (an exclusive scan of
// the masks' popcounts, in the three passes of the offsets above).
static __global__ void k_send_masks(const int* __restrict__ rp, int n, unsigned* __restrict__ smask) {
  const int lane = threadIdx.x & 31;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k - lane < n; k += gridDim.x * blockDim.x) {
    const bool s = k < n && __ldg(rp + k + 1) > __ldg(rp + k);
    const unsigned b = __ballot_sync(0xffffffffu, s);
    if (lane == 0) smask[k >> 5] = b;
  }
}
static __global__ void __launch_bounds__(kPullScanBlock) k_send_tile_sums(const unsigned* __restrict__ smask,
                                                                          int nwords, int4* __restrict__ sums) {
  const int base = blockIdx.x * kPullScanTile + threadIdx.x * kPullScanItems;
  int c = 0;
#pragma unroll
  for (int i = 0; i < kPullScanItems; ++i)
    if (base + i < nwords) c += __popc(__ldg(smask + base + i));
  int4 tot;
  block_scan4(make_int4(c, 0, 0, 0), &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}
static __global__ void __launch_bounds__(kPullScanBlock) k_send_offsets(const unsigned* __restrict__ smask,
                                                                        int nwords, const int4* __restrict__ sums,
                                                                        int* __restrict__ sbase) {
  const int base = blockIdx.x * kPullScanTile + threadIdx.x * kPullScanItems;
  int c[kPullScanItems];
  int t = 0;
#pragma unroll
  for (int i = 0; i < kPullScanItems; ++i) {
    c[i] = base + i < nwords ? __popc(__ldg(smask + base + i)) : 0;
    t += c[i];
  }
  int4 tot;
  const int4 inc = block_scan4(make_int4(t, 0, 0, 0), &tot);
  int run = sums[blockIdx.x].x + inc.x - t;
#pragma unroll
  for (int i = 0; i < kPullScanItems; ++i) {
    if (base + i < nwords) sbase[base + i] = run;
    run += c[i];
  }
}

}  // namespace maiter
