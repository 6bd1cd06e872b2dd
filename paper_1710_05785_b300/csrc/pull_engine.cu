// Host side of the receive-side engine (MAITER_ENGINE_PULL): the transpose
// of a graph and its chunk list for rows of high in-degree, built on first
// use and after every maiter_graph_update, and the run - a CUDA graph
// prime ; WHILE { (decide ; pull) x 3 } per precision phase, the loop
// condition set by the decision kernel (no host round trip per round).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "pull_kernels.cuh"
#include "sync_phase.cuh"

namespace maiter {

namespace {

void free_layout(PullLayout* L) {
  if (!L) return;
  cudaFree(L->crp);
  cudaFree(L->csrc);
  cudaFree(L->crow);
  cudaFree(L->lbits);
  cudaFree(L->large);
  cudaFree(L->large_nch);
  cudaFree(L->lacc);
  cudaFree(L->lcnt);
  cudaFree(L->sbase);
  cudaFree(L->smask);
  cudaFree(L->t_indeg);
  cudaFree(L->t_first);
  cudaFree(L->t_sums);
  delete L;
}

}  // namespace

void free_pull(maiter_graph* g) {
  free_layout(g->pull);
  free_layout(g->pullv);
  g->pull = nullptr;
  g->pullv = nullptr;
}

void invalidate_pull(maiter_graph* g) {
  if (g->pull) g->pull->valid = false;
  if (g->pullv) g->pullv->valid = false;
}

namespace {

template <class T>
cudaError_t grow(T** p, size_t* cap, size_t need) {
  need = std::max<size_t>(need, 1);
  if (*p && *cap >= need) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, sizeof(T) * need);
  if (e == cudaSuccess) *cap = need;
  return e;
}

// Sender masks and ranks of g (every vertex of out-degree > 0 gets the next
// message slot in id order); L->nsend the number of senders.
cudaError_t sender_ranks(const maiter_graph* g, PullLayout* L, cudaStream_t st) {
  const int64_t n = g->n;
  const int nwords = static_cast<int>(std::max<int64_t>((n + 31) / 32, 1));
  const int ntiles = (nwords + kPullScanTile - 1) / kPullScanTile;
  L->nsend = 0;
  cudaError_t e = grow(&L->sbase, &L->sbase_cap, static_cast<size_t>(nwords));
  if (e == cudaSuccess) e = grow(&L->smask, &L->smask_cap, static_cast<size_t>(nwords));
  if (e != cudaSuccess || n == 0) return e;
  e = grow(&L->t_sums, &L->t_sums_cap, static_cast<size_t>(ntiles) + 1);
  int4* sums = L->t_sums;
  int4 tot = make_int4(0, 0, 0, 0);
  if (e == cudaSuccess) {
    k_send_masks<<<g->num_sms * 4, 256, 0, st>>>(g->rp, static_cast<int>(n), L->smask);
    k_send_tile_sums<<<ntiles, kPullScanBlock, 0, st>>>(L->smask, nwords, sums);
    k_pull_scan_sums<<<1, kPullScanBlock, 0, st>>>(sums, ntiles);
    k_send_offsets<<<ntiles, kPullScanBlock, 0, st>>>(L->smask, nwords, sums, L->sbase);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, sums + ntiles, sizeof(int4), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) L->nsend = tot.x;
  return e;
}

}  // namespace

// Builds (or rebuilds after an update) the transpose of g on stream st, on
// the device: the in-degrees, one int4 prefix scan over the rows (small-row
// offsets, tail offsets, chunk entries, large-row index) whose total is the
// one value read back (to size the chunk list), then the senders placed by
// one atomic cursor per receiver.
maiter_status ensure_pull(const maiter_graph* cg, cudaStream_t st, bool vec) {
  maiter_graph* g = const_cast<maiter_graph*>(cg);
  PullLayout*& slot = vec ? g->pullv : g->pull;
  if (slot && slot->valid) return MAITER_OK;
  if (!slot) slot = new PullLayout();
  PullLayout* L = slot;
  L->cut = vec ? kVecCut : kPullCut;
  L->chunk = vec ? kVecChunk : kPullChunk;
  const int64_t n = g->n, m = g->m;
  const int64_t nwords = (n + 31) / 32;
  const int ntiles = static_cast<int>((n + kPullScanTile - 1) / kPullScanTile);
  MAITER_CUDA(grow(&L->crp, &L->crp_cap, static_cast<size_t>(n + 1)));
  MAITER_CUDA(grow(&L->lbits, &L->lbits_cap, static_cast<size_t>(nwords)));
  const size_t n1 = static_cast<size_t>(std::max<int64_t>(n, 1));
  cudaError_t e = grow(&L->t_indeg, &L->t_indeg_cap, n1);
  if (e == cudaSuccess) e = grow(&L->t_first, &L->t_first_cap, n1);
  if (e == cudaSuccess) e = grow(&L->t_sums, &L->t_sums_cap, static_cast<size_t>(ntiles) + 1);
  int* indeg = L->t_indeg;
  int* first = L->t_first;
  int4* sums = L->t_sums;
  if (e == cudaSuccess) e = cudaMemsetAsync(indeg, 0, sizeof(int) * n1, st);
  if (e == cudaSuccess && m > 0) {
    k_pull_indegree<<<g->num_sms * 4, 256, 0, st>>>(g->col, m, indeg);
    e = cudaGetLastError();
  }
  int4 totals = make_int4(0, 0, 0, 0);   // small edges, tail edges, chunks, large rows
  if (e == cudaSuccess && n > 0) {
    k_pull_tile_sums<<<ntiles, kPullScanBlock, 0, st>>>(indeg, static_cast<int>(n), L->cut, L->chunk,
                                                         sums);
    k_pull_scan_sums<<<1, kPullScanBlock, 0, st>>>(sums, ntiles);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&totals, sums + ntiles, sizeof(int4), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(L->crp, 0, sizeof(int), st);
  }
  L->nlarge = totals.z;
  L->nlrows = totals.w;
  // edge slots: the small rows' in-edges, the tail from the next multiple of
  // 4 (each large row's part padded to a multiple of 4), and 16 slots of
  // slack for the kernels' 4-slot loads that end past the last edge
  const size_t slots = static_cast<size_t>((static_cast<int64_t>(totals.x) + 3) & ~int64_t{3}) +
                       static_cast<size_t>(totals.y) + 16;
  if (e == cudaSuccess) e = grow(&L->csrc, &L->csrc_cap, slots);
  if (e == cudaSuccess) e = grow(&L->crow, &L->crow_cap, slots);
  if (e == cudaSuccess) e = grow(&L->large, &L->large_cap, static_cast<size_t>(totals.z));
  if (e == cudaSuccess) e = grow(&L->large_nch, &L->lrow_cap, static_cast<size_t>(totals.w));
  if (e == cudaSuccess) {
    // lacc / lcnt: one entry per large row, zero between rounds
    const size_t nl = static_cast<size_t>(std::max(totals.w, 1));
    e = grow(&L->lacc, &L->lacc_cap, nl);
    if (e == cudaSuccess) e = grow(&L->lcnt, &L->lcnt_cap, nl);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->lacc, 0, sizeof(double) * nl, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->lcnt, 0, sizeof(unsigned) * nl, st);
  }
  if (e == cudaSuccess && n > 0) {
    k_pull_offsets<<<ntiles, kPullScanBlock, 0, st>>>(indeg, static_cast<int>(n), L->cut, L->chunk,
                                                       sums, ntiles,
                                                       L->crp, first, L->lbits, L->large,
                                                       L->large_nch);
    e = cudaGetLastError();
  }
  // the sender ranks reuse the scan's work array (in stream order, after the
  // offsets pass has read it)
  if (e == cudaSuccess) e = sender_ranks(g, L, st);
  if (e == cudaSuccess && n > 0) {
    k_pull_place<<<g->num_sms * 8, 256, 0, st>>>(g->rp, g->col, static_cast<int>(n), L->sbase,
                                                 L->smask, first, L->csrc, L->crow);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  MAITER_CUDA(e);
  L->valid = true;
  return MAITER_OK;
}

namespace {

// One precision phase: prime, then WHILE { (decide ; pull) x kRounds }.
template <class DT, class MT, class CT>
struct PullPhase {
  PullArgs a{};
  int pull_grid = 1, prime_grid = 1;
  static constexpr int kRounds = 3;

  static void* prime_fn() { return reinterpret_cast<void*>(&k_pull_prime<DT, MT, CT>); }
  void launch_prime(cudaStream_t s, const double* wide, cudaGraphConditionalHandle h,
                    int use_cond) const {
    k_pull_prime<DT, MT, CT><<<prime_grid, 256, 0, s>>>(a, wide, h, use_cond);
  }
  void launch_round(cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                    bool chained) const {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.blockDim = dim3(32);
    cfg.gridDim = dim3(1);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = chained ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_pull_decide, a.ctl, h, use_cond);
    cfg.blockDim = dim3(kPullBlock);
    cfg.gridDim = dim3(pull_grid);
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_pull<DT, MT>, a);
  }
  maiter_status add_to(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                       cudaGraphConditionalHandle h, cudaGraphNode_t* node) const {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    MAITER_CUDA(cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t cap;
    MAITER_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int u = 0; u < kRounds; ++u) launch_round(cap, h, 1, u > 0);
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(cap, &captured);
    }
    cudaStreamDestroy(cap);
    MAITER_CUDA(e);
    return MAITER_OK;
  }
  // Host-driven rounds with events around the pull (profiling mode).
  maiter_status host_loop(maiter_result* r, cudaStream_t st, cudaEvent_t* e,
                          maiter_stats& s) const {
    for (;;) {
      k_pull_decide<<<1, 32, 0, st>>>(a.ctl, cudaGraphConditionalHandle{}, 0);
      k_hold<<<1, 32, 0, st>>>(kHoldNs);
      MAITER_CUDA(cudaEventRecord(e[0], st));
      k_pull<DT, MT><<<pull_grid, kPullBlock, 0, st>>>(a);
      MAITER_CUDA(cudaEventRecord(e[1], st));
      MAITER_CUDA(cudaGetLastError());
      MAITER_CUDA(cudaMemcpyAsync(r->h_ctl, r->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
      MAITER_CUDA(cudaStreamSynchronize(st));
      if (r->h_ctl->status != 0) return MAITER_OK;   // the pull returned at once
      float t = 0.f;
      cudaEventElapsedTime(&t, e[0], e[1]);
      s.push_ms += t;
      s.push_launches++;
    }
  }
};

template <class DT, class MT, class CT>
void setup_phase(PullPhase<DT, MT, CT>& ph, const maiter_graph* g, maiter_result* r, void* delta,
                 const void* coef, double damping) {
  const PullLayout* L = g->pull;
  PullArgs& a = ph.a;
  a.n = static_cast<int>(g->n);
  a.ngroups = static_cast<int>((g->n + 31) / 32);
  a.nlarge = L->nlarge;
  a.rp = g->rp;
  a.crp = L->crp;
  a.csrc = L->csrc;
  a.crow = L->crow;
  a.lbits = L->lbits;
  a.large = L->large;
  a.large_nch = L->large_nch;
  a.lacc = L->lacc;
  a.lcnt = L->lcnt;
  a.coef = coef;
  a.damping = damping;
  a.v = static_cast<double*>(r->v);
  a.delta = delta;
  a.msg[0] = r->bin_msg_v;
  a.msg[1] = r->pull_msg;
  a.cmsg = r->bin_cmsg;
  a.sbase = L->sbase;
  a.smask = L->smask;
  a.ctl = r->ctl;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pull<DT, MT>, kPullBlock, 0);
  ph.pull_grid = g->num_sms * std::max(per_sm, 1);
  ph.prime_grid = std::max(1, std::min(static_cast<int>((g->n + 255) / 256), g->num_sms * 4));
}

}  // namespace

maiter_status run_pull(const maiter_graph* g, const maiter_run_params* p, maiter_result* r,
                       cudaStream_t st) {
  {
    maiter_status s = ensure_pull(g, st);
    if (s != MAITER_OK) return s;
  }
  const PullLayout* L = g->pull;
  const bool mixed = p->op == MAITER_OP_SUM_MIXED;
  {
    const size_t nv = static_cast<size_t>(std::max<int64_t>(g->n, 1));
    if (!r->bin_msg_v) MAITER_CUDA(cudaMalloc(&r->bin_msg_v, nv * sizeof(double)));
    if (!r->pull_msg) MAITER_CUDA(cudaMalloc(&r->pull_msg, nv * sizeof(double)));
    if (!r->bin_cmsg) MAITER_CUDA(cudaMalloc(&r->bin_cmsg, nv * sizeof(double)));
  }
  const void* coef = p->coef ? r->coef : nullptr;
  PullPhase<double, double, double> f64;
  PullPhase<double, double, float> warm;
  PullPhase<float, float, float> f32;
  if (mixed) {
    setup_phase(warm, g, r, r->delta_wide, coef, p->damping);
    setup_phase(f32, g, r, r->delta, coef, p->damping);
  } else {
    setup_phase(f64, g, r, r->delta, coef, p->damping);
  }
  const bool profile = (p->flags & MAITER_FLAG_PROFILE_KERNELS) != 0;
  // the executable graph bakes in its arguments: rebuilt when one changes
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](uint64_t x) { key = (key ^ x) * 1099511628211ull; };
  uint64_t dbits;
  std::memcpy(&dbits, &p->damping, sizeof(dbits));
  mix(0x9A11EDull);
  mix(static_cast<uint64_t>(p->op));
  mix(p->coef ? 1 : 0);
  mix(dbits);
  mix(static_cast<uint64_t>(L->nlarge));
  mix(reinterpret_cast<uintptr_t>(L->crp));
  mix(reinterpret_cast<uintptr_t>(L->csrc));
  mix(reinterpret_cast<uintptr_t>(L->crow));
  mix(reinterpret_cast<uintptr_t>(L->lbits));
  mix(reinterpret_cast<uintptr_t>(L->large));
  mix(reinterpret_cast<uintptr_t>(L->lacc));
  mix(reinterpret_cast<uintptr_t>(r->pull_msg));
  mix(reinterpret_cast<uintptr_t>(L->sbase));
  mix(reinterpret_cast<uintptr_t>(L->smask));
  if (!profile && (!r->exec || r->exec_key != key)) {
    if (r->exec) { cudaGraphExecDestroy(r->exec); r->exec = nullptr; }
    if (r->graph) { cudaGraphDestroy(r->graph); r->graph = nullptr; }
    r->exec_key = 0;
    MAITER_CUDA(cudaGraphCreate(&r->graph, 0));
    cudaGraphConditionalHandle h1;
    MAITER_CUDA(cudaGraphConditionalHandleCreate(&h1, r->graph, 1, cudaGraphCondAssignDefault));
    auto prime_node = [&](auto& ph, const double* wide, cudaGraphConditionalHandle h,
                          int use_cond, const cudaGraphNode_t* deps, size_t ndeps,
                          cudaGraphNode_t* out_node) -> maiter_status {
      void* args[] = {&ph.a, &wide, &h, &use_cond};
      cudaKernelNodeParams kp{};
      kp.func = ph.prime_fn();
      kp.gridDim = dim3(ph.prime_grid);
      kp.blockDim = dim3(256);
      kp.sharedMemBytes = 0;
      kp.kernelParams = args;
      MAITER_CUDA(cudaGraphAddKernelNode(out_node, r->graph, deps, ndeps, &kp));
      return MAITER_OK;
    };
    cudaGraphNode_t n0, n1;
    maiter_status s;
    if (mixed) {
      s = prime_node(warm, nullptr, h1, 0, nullptr, 0, &n0);
      if (s != MAITER_OK) return s;
      s = warm.add_to(r->graph, &n0, 1, h1, &n1);
      if (s != MAITER_OK) return s;
      cudaGraphConditionalHandle h2;
      MAITER_CUDA(cudaGraphConditionalHandleCreate(&h2, r->graph, 0, 0));
      cudaGraphNode_t n2, n3;
      s = prime_node(f32, static_cast<const double*>(r->delta_wide), h2, 1, &n1, 1, &n2);
      if (s != MAITER_OK) return s;
      s = f32.add_to(r->graph, &n2, 1, h2, &n3);
    } else {
      s = prime_node(f64, nullptr, h1, 0, nullptr, 0, &n0);
      if (s != MAITER_OK) return s;
      s = f64.add_to(r->graph, &n0, 1, h1, &n1);
    }
    if (s != MAITER_OK) return s;
    MAITER_CUDA(cudaGraphInstantiate(&r->exec, r->graph, 0));
    r->exec_key = key;
  }
  DevCtl c{};
  c.eps = p->eps;
  c.eps_in[0] = c.eps_in[1] = p->eps;
  c.switch_frac = mixed ? p->mixed_switch : 0.0;
  c.max_rounds = p->max_rounds > 0 ? p->max_rounds : 1000000;
  c.sched = p->sched;
  *r->h_ctl = c;
  MAITER_CUDA(cudaMemcpyAsync(r->ctl, r->h_ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, st));
  maiter_stats& s = r->stats;
  s = maiter_stats{};
  if (profile) {
    cudaEvent_t e[2];
    for (auto& x : e) MAITER_CUDA(cudaEventCreate(&x));
    MAITER_CUDA(cudaEventRecord(r->ev0, st));
    maiter_status ls;
    if (mixed) {
      warm.launch_prime(st, nullptr, cudaGraphConditionalHandle{}, 0);
      ls = warm.host_loop(r, st, e, s);
      if (ls == MAITER_OK) {
        f32.launch_prime(st, static_cast<const double*>(r->delta_wide),
                         cudaGraphConditionalHandle{}, 0);
        MAITER_CUDA(cudaGetLastError());
        MAITER_CUDA(cudaMemcpyAsync(r->h_ctl, r->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
        MAITER_CUDA(cudaStreamSynchronize(st));
        if (r->h_ctl->status == 0) ls = f32.host_loop(r, st, e, s);
      }
    } else {
      f64.launch_prime(st, nullptr, cudaGraphConditionalHandle{}, 0);
      ls = f64.host_loop(r, st, e, s);
    }
    MAITER_CUDA(cudaEventRecord(r->ev1, st));
    MAITER_CUDA(cudaStreamSynchronize(st));
    for (auto& x : e) cudaEventDestroy(x);
    if (ls != MAITER_OK) return ls;
  } else {
    MAITER_CUDA(cudaEventRecord(r->ev0, st));
    MAITER_CUDA(cudaGraphLaunch(r->exec, st));
    MAITER_CUDA(cudaEventRecord(r->ev1, st));
    MAITER_CUDA(cudaMemcpyAsync(r->h_ctl, r->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
    MAITER_CUDA(cudaStreamSynchronize(st));
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, r->ev0, r->ev1);
  const DevCtl& h = *r->h_ctl;
  s.rounds = static_cast<int64_t>(h.rounds);
  s.activations = static_cast<int64_t>(h.activations);
  s.edge_pushes = static_cast<int64_t>(h.pushes);
  if (mixed) {
    const bool switched = h.phase > 0;
    s.warm_rounds = static_cast<int64_t>(switched ? h.warm_rounds : h.rounds);
    s.warm_activations = static_cast<int64_t>(switched ? h.warm_activations : h.activations);
    s.warm_edge_pushes = static_cast<int64_t>(switched ? h.warm_pushes : h.pushes);
  }
  s.residual = h.residual;
  s.elapsed_ms = ms;
  s.converged = h.status == 1;
  // prime per phase, then whole passes of kRounds rounds (2 kernels each);
  // the pass that stops completes its remaining rounds, which return at once
  const int64_t phases = 1 + (h.phase > 0 ? 1 : 0);
  constexpr int64_t kPass = PullPhase<double, double, double>::kRounds;
  const int64_t decided = static_cast<int64_t>(h.rounds) + phases;
  const int64_t rounds_run = profile ? decided : kPass * ((decided + kPass - 1) / kPass);
  s.kernel_launches = phases + 2 * rounds_run + (profile ? decided : 0);
  s.status = h.status == 1 ? MAITER_OK : MAITER_ERR_NOT_CONVERGED;
  if (h.status != 1)
    set_error("round cap of %lld reached before the termination test held (residual %g)",
              (long long)c.max_rounds, h.residual);
  return static_cast<maiter_status>(s.status);
}

}  // namespace maiter
