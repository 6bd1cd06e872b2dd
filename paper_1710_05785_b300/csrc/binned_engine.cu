// Host side of the binned engine (MAITER_ENGINE_BINNED): the static layout
// of a graph's edges by (sender cell, receiver bin), built on the device on
// first use and after every maiter_graph_update, and the run - a CUDA graph
// prime ; WHILE { (scatter ; gather) x 3 } per precision phase, with the loop
// condition set by the scatter's CTA 0 (no host round trip per round).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "binned_kernels.cuh"
#include "sync_phase.cuh"

namespace maiter {

struct BinLayout {
  bool valid = false;
  uint64_t generation = 0;
  int nbins = 0;
  int nchunks = 0;
  int64_t slots = 0;                 // padded edge slots
  int4* chunks = nullptr;
  int* cb = nullptr;                 // nchunks + 1
  int* T = nullptr;                  // (nbins + 1) x nchunks
  unsigned short* src_local = nullptr;
  unsigned short* dst_local = nullptr;
  int* step_base = nullptr;          // nbins + 1
  unsigned* steps = nullptr;         // the 32-slot steps of every bin's segments
  int64_t nsteps = 0;
  size_t chunks_cap = 0, cb_cap = 0, t_cap = 0, src_cap = 0, dst_cap = 0, sb_cap = 0,
         steps_cap = 0;
};

void free_bins(maiter_graph* g) {
  if (!g->bins) return;
  BinLayout* L = g->bins;
  cudaFree(L->chunks);
  cudaFree(L->cb);
  cudaFree(L->T);
  cudaFree(L->src_local);
  cudaFree(L->dst_local);
  cudaFree(L->step_base);
  cudaFree(L->steps);
  delete L;
  g->bins = nullptr;
}

void invalidate_bins(maiter_graph* g) {
  if (g->bins) g->bins->valid = false;
}

namespace {

constexpr int kHistBlock = 1024;
constexpr int kPlaceBlock = 512;

// Grows a device buffer to at least `need` elements (contents not kept).
template <class T>
cudaError_t ensure(T** p, size_t* cap, size_t need) {
  if (*p && *cap >= need) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, sizeof(T) * std::max<size_t>(need, 1));
  if (e == cudaSuccess) *cap = std::max<size_t>(need, 1);
  return e;
}

maiter_status set_smem_limits() {
  static bool done = false;
  if (done) return MAITER_OK;
  MAITER_CUDA(cudaFuncSetAttribute(k_bin_hist<kHistBlock>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kBinMaxBins * 4));
  MAITER_CUDA(cudaFuncSetAttribute(k_bin_place<kPlaceBlock>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (kBinMaxBins + kCellSize + 1) * 4));
  MAITER_CUDA(cudaFuncSetAttribute(k_bin_scatter<double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kCellSize * 8));
  MAITER_CUDA(cudaFuncSetAttribute(k_bin_scatter<float>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kCellSize * 4));
  MAITER_CUDA(cudaFuncSetAttribute(k_bin_gather<double, double, double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kBinSize * 8));
  MAITER_CUDA(cudaFuncSetAttribute(k_bin_gather<double, double, float>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kBinSize * 8));
  MAITER_CUDA(cudaFuncSetAttribute(k_bin_gather<float, float, float>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kBinSize * 8));
  done = true;
  return MAITER_OK;
}

}  // namespace

// Builds (or rebuilds after an update) the layout of g on stream st.
maiter_status ensure_bins(const maiter_graph* cg, cudaStream_t st) {
  maiter_graph* g = const_cast<maiter_graph*>(cg);
  if (g->bins && g->bins->valid) return MAITER_OK;
  {
    maiter_status s = set_smem_limits();
    if (s != MAITER_OK) return s;
  }
  if (!g->bins) {
    g->bins = new (std::nothrow) BinLayout();
    MAITER_REQUIRE(g->bins, "host allocation failed");
  }
  BinLayout* L = g->bins;
  const int64_t n = g->n, m = g->m;
  const int64_t nbins64 = (n + kBinSize - 1) >> kBinShift;
  if (nbins64 > kBinMaxBins) {
    set_error("the binned engine serves at most %lld vertices (n = %lld)",
              (long long)kBinMaxBins * kBinSize, (long long)n);
    return MAITER_ERR_UNSUPPORTED;
  }
  L->nbins = static_cast<int>(nbins64);
  const int ncells = static_cast<int>((n + kCellSize - 1) >> kCellShift);
  // 1. edges per cell -> chunks (pieces of at most kPieceEdges edges)
  std::vector<int4> chunks;
  if (m > 0 && ncells > 0) {
    int2* d_cells = nullptr;
    MAITER_CUDA(cudaMalloc(&d_cells, sizeof(int2) * ncells));
    k_bin_cells<<<std::max(1, std::min(ncells / 256 + 1, g->num_sms * 4)), 256, 0, st>>>(
        g->rp, n, ncells, d_cells);
    std::vector<int2> cells(ncells);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cells.data(), d_cells, sizeof(int2) * ncells, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_cells);
    MAITER_CUDA(e);
    for (int k = 0; k < ncells; ++k) {
      const int first = cells[k].x, cnt = cells[k].y;
      for (int p = 0; p * static_cast<int64_t>(kPieceEdges) < cnt; ++p) {
        const int b = first + p * kPieceEdges;
        const int en = first + static_cast<int>(std::min<int64_t>(cnt, (p + 1) * int64_t(kPieceEdges)));
        chunks.push_back(make_int4(b, en, k << kCellShift, 0));
      }
    }
  }
  const int nchunks = static_cast<int>(chunks.size());
  L->nchunks = nchunks;
  MAITER_CUDA(ensure(&L->chunks, &L->chunks_cap, static_cast<size_t>(nchunks)));
  MAITER_CUDA(ensure(&L->cb, &L->cb_cap, static_cast<size_t>(nchunks) + 1));
  if (nchunks == 0) {
    L->slots = 0;
    int zero = 0;
    MAITER_CUDA(cudaMemcpyAsync(L->cb, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    MAITER_CUDA(ensure(&L->T, &L->t_cap, static_cast<size_t>(1)));
    MAITER_CUDA(ensure(&L->src_local, &L->src_cap, static_cast<size_t>(kPad)));
    MAITER_CUDA(ensure(&L->dst_local, &L->dst_cap, static_cast<size_t>(kPad)));
    MAITER_CUDA(ensure(&L->step_base, &L->sb_cap, static_cast<size_t>(L->nbins) + 1));
    MAITER_CUDA(cudaMemsetAsync(L->step_base, 0, sizeof(int) * (L->nbins + 1), st));
    MAITER_CUDA(ensure(&L->steps, &L->steps_cap, static_cast<size_t>(1)));
    L->nsteps = 0;
    MAITER_CUDA(cudaStreamSynchronize(st));
    L->valid = true;
    ++L->generation;
    return MAITER_OK;
  }
  MAITER_CUDA(cudaMemcpyAsync(L->chunks, chunks.data(), sizeof(int4) * nchunks,
                              cudaMemcpyHostToDevice, st));
  k_bin_span<<<std::max(1, std::min(nchunks / 256 + 1, g->num_sms * 4)), 256, 0, st>>>(
      g->rp, n, L->chunks, nchunks);
  MAITER_CUDA(cudaGetLastError());
  // 2. padded per-(chunk, bin) offsets
  int* soff = nullptr;
  const size_t soff_n = static_cast<size_t>(nchunks) * (L->nbins + 1);
  MAITER_CUDA(cudaMalloc(&soff, sizeof(int) * soff_n));
  auto fail = [&](cudaError_t e) {
    cudaFree(soff);
    set_error("binned layout: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;
  };
  const int grid = std::min(nchunks, g->num_sms * 2);
  k_bin_hist<kHistBlock><<<grid, kHistBlock, L->nbins * 4, st>>>(g->col, L->chunks, nchunks,
                                                                 L->nbins, soff);
  cudaError_t e = cudaGetLastError();
  std::vector<int> pc(nchunks);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(pc.data(), sizeof(int), soff + L->nbins, sizeof(int) * (L->nbins + 1),
                          sizeof(int), nchunks, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  // 3. chunk bases
  std::vector<int> cb(nchunks + 1);
  int64_t run = 0;
  for (int c = 0; c < nchunks; ++c) {
    cb[c] = static_cast<int>(std::min<int64_t>(run, INT32_MAX));
    run += pc[c];
  }
  if (run >= (int64_t(1) << 31)) {
    cudaFree(soff);
    set_error("binned layout: %lld padded slots exceed 2^31", (long long)run);
    return MAITER_ERR_UNSUPPORTED;
  }
  cb[nchunks] = static_cast<int>(run);
  L->slots = run;
  e = cudaMemcpyAsync(L->cb, cb.data(), sizeof(int) * (nchunks + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = ensure(&L->T, &L->t_cap, static_cast<size_t>(L->nbins + 1) * nchunks);
  if (e != cudaSuccess) return fail(e);
  if (e == cudaSuccess) e = ensure(&L->src_local, &L->src_cap, static_cast<size_t>(run));
  if (e == cudaSuccess) e = ensure(&L->dst_local, &L->dst_cap, static_cast<size_t>(run));
  if (e != cudaSuccess) return fail(e);
  // 4. segment table and slot contents
  k_bin_table<<<g->num_sms * 4, 256, 0, st>>>(soff, L->cb, nchunks, L->nbins, L->T);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemsetAsync(L->src_local, 0xFF, sizeof(unsigned short) * run, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(L->dst_local, 0, sizeof(unsigned short) * run, st);
  if (e != cudaSuccess) return fail(e);
  k_bin_place<kPlaceBlock><<<std::min(nchunks, g->num_sms * 2), kPlaceBlock,
                             (L->nbins + kCellSize + 1) * 4, st>>>(
      g->rp, g->col, L->chunks, nchunks, L->nbins, soff, L->cb, L->src_local, L->dst_local);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_bin_sort<<<g->num_sms * 4, kSortBlock, 0, st>>>(L->T, nchunks, L->nbins, L->src_local,
                                                      L->dst_local);
    e = cudaGetLastError();
  }
  // 5. per bin, the 32-slot steps of its segments
  std::vector<int> bin_steps(L->nbins);
  if (e == cudaSuccess) e = ensure(&L->step_base, &L->sb_cap, static_cast<size_t>(L->nbins) + 1);
  if (e == cudaSuccess) {
    k_bin_steps<0><<<std::min(L->nbins, g->num_sms * 2), kStepBlock, 0, st>>>(
        L->T, nchunks, L->nbins, L->step_base, nullptr, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bin_steps.data(), L->step_base, sizeof(int) * L->nbins,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  std::vector<int> sb(L->nbins + 1);
  int64_t q = 0;
  for (int b = 0; b < L->nbins; ++b) {
    sb[b] = static_cast<int>(q);
    q += bin_steps[b];
  }
  sb[L->nbins] = static_cast<int>(q);
  L->nsteps = q;
  e = cudaMemcpyAsync(L->step_base, sb.data(), sizeof(int) * (L->nbins + 1),
                      cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = ensure(&L->steps, &L->steps_cap, static_cast<size_t>(std::max<int64_t>(q, 1)));
  if (e == cudaSuccess) {
    k_bin_steps<1><<<std::min(L->nbins, g->num_sms * 2), kStepBlock, 0, st>>>(
        L->T, nchunks, L->nbins, nullptr, L->step_base, L->steps);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(soff);
  soff = nullptr;
  if (e != cudaSuccess) return fail(e);
  L->valid = true;
  ++L->generation;
  return MAITER_OK;
}

namespace {

// One precision phase: prime, then WHILE { (scatter ; gather) x kRounds }.
template <class DT, class MT, class CT>
struct BinPhase {
  BinArgs a{};
  int scatter_grid = 1, gather_grid = 1, prime_grid = 1;
  static constexpr int kRounds = 3;

  static void* prime_fn() { return reinterpret_cast<void*>(&k_bin_prime<DT, MT, CT>); }
  void launch_prime(cudaStream_t s, const double* wide, cudaGraphConditionalHandle h,
                    int use_cond) const {
    k_bin_prime<DT, MT, CT><<<prime_grid, 256, 0, s>>>(a, wide, h, use_cond);
  }
  void launch_round(cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                    bool chained) const {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.blockDim = dim3(kBinScatterBlock);
    cfg.gridDim = dim3(scatter_grid);
    cfg.dynamicSmemBytes = kCellSize * sizeof(MT);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = chained ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_bin_scatter<MT>, a, h, use_cond);
    cfg.blockDim = dim3(kBinGatherBlock);
    cfg.gridDim = dim3(gather_grid);
    cfg.dynamicSmemBytes = kBinSize * sizeof(unsigned long long);
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_bin_gather<DT, MT, CT>, a);
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
  // Host-driven rounds with events around each kernel (profiling mode).
  maiter_status host_loop(maiter_result* r, cudaStream_t st, cudaEvent_t* e,
                          maiter_stats& s) const {
    for (;;) {
      k_hold<<<1, 32, 0, st>>>(kHoldNs);
      MAITER_CUDA(cudaEventRecord(e[0], st));
      k_bin_scatter<MT><<<scatter_grid, kBinScatterBlock, kCellSize * sizeof(MT), st>>>(
          a, cudaGraphConditionalHandle{}, 0);
      MAITER_CUDA(cudaEventRecord(e[1], st));
      k_bin_gather<DT, MT, CT><<<gather_grid, kBinGatherBlock,
                                 kBinSize * sizeof(unsigned long long), st>>>(a);
      MAITER_CUDA(cudaEventRecord(e[2], st));
      MAITER_CUDA(cudaGetLastError());
      MAITER_CUDA(cudaMemcpyAsync(r->h_ctl, r->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
      MAITER_CUDA(cudaStreamSynchronize(st));
      if (r->h_ctl->status != 0) return MAITER_OK;   // this round's kernels returned at once
      float t1 = 0.f, t2 = 0.f;
      cudaEventElapsedTime(&t1, e[0], e[1]);
      cudaEventElapsedTime(&t2, e[1], e[2]);
      s.bin_scatter_ms += t1;
      s.bin_gather_ms += t2;
      s.push_ms += t1 + t2;
      s.push_launches++;
    }
  }
};

template <class DT, class MT, class CT>
void setup_phase(BinPhase<DT, MT, CT>& ph, const maiter_graph* g, maiter_result* r, void* delta,
                 const void* coef, double damping) {
  const BinLayout* L = g->bins;
  BinArgs& a = ph.a;
  a.n = static_cast<int>(g->n);
  a.nbins = L->nbins;
  a.nchunks = L->nchunks;
  a.rp = g->rp;
  a.coef = coef;
  a.damping = damping;
  a.v = static_cast<double*>(r->v);
  a.delta = delta;
  a.msg_v = r->bin_msg_v;
  a.msg_e = r->bin_msg_e;
  a.cmsg = r->bin_cmsg;
  a.chunks = L->chunks;
  a.cb = L->cb;
  a.T = L->T;
  a.src8 = reinterpret_cast<const uint4*>(L->src_local);
  a.dst8 = reinterpret_cast<const uint4*>(L->dst_local);
  a.step_base = L->step_base;
  a.steps = L->steps;
  a.ctl = r->ctl;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_scatter<MT>, kBinScatterBlock,
                                                kCellSize * sizeof(MT));
  ph.scatter_grid = std::max(1, std::min(L->nchunks, g->num_sms * std::max(per_sm, 1)));
  ph.gather_grid = std::max(1, std::min(L->nbins, g->num_sms));
  ph.prime_grid = std::max(1, std::min(static_cast<int>((g->n + 255) / 256), g->num_sms * 4));
}

}  // namespace

maiter_status run_binned(const maiter_graph* g, const maiter_run_params* p, maiter_result* r,
                         cudaStream_t st) {
  {
    maiter_status s = ensure_bins(g, st);
    if (s != MAITER_OK) return s;
  }
  const BinLayout* L = g->bins;
  const bool mixed = p->op == MAITER_OP_SUM_MIXED;
  {
    const size_t nv = static_cast<size_t>(std::max<int64_t>(g->n, 1));
    if (!r->bin_msg_v) MAITER_CUDA(cudaMalloc(&r->bin_msg_v, nv * sizeof(double)));
    if (!r->bin_cmsg) MAITER_CUDA(cudaMalloc(&r->bin_cmsg, nv * sizeof(double)));
    const size_t ne = static_cast<size_t>(std::max<int64_t>(L->slots, kPad));
    if (!r->bin_msg_e || r->bin_msg_e_cap < ne) {
      cudaFree(r->bin_msg_e);
      r->bin_msg_e = nullptr;
      r->bin_msg_e_cap = 0;
      MAITER_CUDA(cudaMalloc(&r->bin_msg_e, ne * sizeof(double)));
      r->bin_msg_e_cap = ne;
    }
  }
  const void* coef = p->coef ? r->coef : nullptr;
  BinPhase<double, double, double> f64;
  BinPhase<double, double, float> warm;
  BinPhase<float, float, float> f32;
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
  mix(0xB1AAEDull);
  mix(static_cast<uint64_t>(p->op));
  mix(p->coef ? 1 : 0);
  mix(dbits);
  mix(static_cast<uint64_t>(L->nchunks));
  mix(reinterpret_cast<uintptr_t>(L->T));
  mix(reinterpret_cast<uintptr_t>(L->src_local));
  mix(reinterpret_cast<uintptr_t>(L->dst_local));
  mix(reinterpret_cast<uintptr_t>(L->chunks));
  mix(reinterpret_cast<uintptr_t>(L->cb));
  mix(reinterpret_cast<uintptr_t>(r->bin_msg_e));
  mix(reinterpret_cast<uintptr_t>(L->steps));
  mix(reinterpret_cast<uintptr_t>(L->step_base));
  if (!profile && (!r->exec || r->exec_key != key)) {
    if (r->exec) { cudaGraphExecDestroy(r->exec); r->exec = nullptr; }
    if (r->graph) { cudaGraphDestroy(r->graph); r->graph = nullptr; }
    r->exec_key = 0;
    MAITER_CUDA(cudaGraphCreate(&r->graph, 0));
    cudaGraphConditionalHandle h1;
    MAITER_CUDA(cudaGraphConditionalHandleCreate(&h1, r->graph, 1, cudaGraphCondAssignDefault));
    // prime nodes: kernel nodes with their arguments
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
    cudaEvent_t e[3];
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
  s.slots = L->slots;
  // prime per phase, then whole passes of kRounds rounds (2 kernels each);
  // the pass that stops completes its remaining rounds, which return at once
  const int64_t phases = 1 + (h.phase > 0 ? 1 : 0);
  constexpr int64_t kPass = BinPhase<double, double, double>::kRounds;
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
