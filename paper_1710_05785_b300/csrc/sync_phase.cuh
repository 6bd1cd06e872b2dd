// Host-side pieces of the round engine shared by single runs (maiter_api.cu)
// and the dense batch (batch_engine.cu): launch shapes, trace sinks, and the
// Phase that adds / drives WHILE(cond) { ([select] ; k_scan ; k_push) x kRoundsPerPass }.
#pragma once
#include <algorithm>

#include "internal.h"

namespace maiter {

inline int grid_for(const void* fn, int block, int num_sms, int per_sm_cap) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm_cap > 0 && per_sm > per_sm_cap) per_sm = per_sm_cap;
  return num_sms * per_sm;
}

constexpr int kBlock = 256;
constexpr long long kPushEdgesPerCta = 2048;
// per-round hold of the host-driven (profiling) loop
constexpr unsigned long long kHoldNs = 40000;

// Device buffers that a traced run fills, one row per (record, sampled vertex).
struct TraceSink {
  const int* sample = nullptr;
  int ns = 0;
  int max_records = 0;
  int records = 0;
  float* feat = nullptr;
  double* dl = nullptr;
  double* vs = nullptr;
  unsigned* la = nullptr;
};

// One phase of the round loop, WHILE(cond) { [select] ; k_scan ; k_push }, for one
// operator: its kernel arguments and launch shapes.
template <class Op>
struct Phase {
  KArgs<Op> a{};
  int push_grid = 1, scan_grid = 1, hist_grid = 1;
  bool learned = false;               // LEARNED: the scan scores (k_scan<.., true>)

  void setup(const maiter_graph* g, maiter_result* r, void* delta, const void* coef,
             double damping, const Tuning& tu, bool topq, const MlpWeights* scorer = nullptr,
             bool track = false) {
    learned = scorer != nullptr;
    a.mlp = scorer;
    a.lstat = g->lstat;
    a.last_act = (scorer || track) ? r->last_act : nullptr;
    a.n = static_cast<int>(g->n);
    a.rp = g->rp;
    a.edges.col = g->col;
    a.edges.w = g->w;
    a.edges.ecoef = r->ecoef;
    a.edges.cw = g->cw;
    a.coef = static_cast<const typename Op::C*>(coef);
    a.damping = damping;
    a.v = static_cast<typename Op::V*>(r->v);
    a.delta = static_cast<typename Op::D*>(delta);
    for (int b = 0; b < 2; ++b) a.list[b] = r->list[b];
    a.large = r->large;
    a.large_d = static_cast<typename Op::D*>(r->large_d);
    a.large_cap = r->large_cap;
    a.ctl = r->ctl;
    a.topq = topq ? r->topq : nullptr;
    hist_grid = g->num_sms * 4;
    a.cut_warp = tu.cut_warp;
    a.cut_cta = tu.cut_cta;
    push_grid = grid_for(reinterpret_cast<const void*>(&k_push<Op, kBlock>), kBlock, g->num_sms,
                         tu.push_blocks_per_sm);
    scan_grid = grid_for(learned ? reinterpret_cast<const void*>(&k_scan<Op, kBlock, true>)
                                 : reinterpret_cast<const void*>(&k_scan<Op, kBlock>),
                         kBlock, g->num_sms, tu.scan_blocks_per_sm);
    // Small graphs: one push CTA per kPushEdgesPerCta edges (at least one per
    // SM) instead of a full grid of CTAs that would only take the decision
    // and leave (PageRank on 65K edges: 1.49 -> 1.41 ms).
    {
      const long long want = std::max<long long>(g->num_sms, g->m / kPushEdgesPerCta);
      if (want < push_grid) push_grid = static_cast<int>(want);
    }
    const int tile = kBlock * kScanItems;
    const int need = static_cast<int>((g->n + tile - 1) / tile);
    if (need < scan_grid) scan_grid = need > 0 ? need : 1;
  }

  // TOPFRAC: the three radix-select passes that fix the round's key threshold
  // (exact); LEARNED: the sampled threshold (the scan scores every vertex),
  // with `chained` a programmatic dependent of the push before it.
  void launch_select(cudaStream_t s, bool chained = false) const {
    if (!a.topq) return;
    TopqCtl* tq = const_cast<TopqCtl*>(a.topq);
    if (learned) {
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(kLearnedBlocks);
      cfg.blockDim = dim3(kLearnedBlock);
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = chained ? 1 : 0;
      cudaLaunchKernelEx(&cfg, k_learned_threshold<Op>, a, tq);
      return;
    }
    k_topq_hist<Op, kBlock, 0><<<hist_grid, kBlock, 0, s>>>(a, tq);
    k_topq_hist<Op, kBlock, 1><<<hist_grid, kBlock, 0, s>>>(a, tq);
    k_topq_hist<Op, kBlock, 2><<<hist_grid, kBlock, 0, s>>>(a, tq);
  }

  void launch_scan(cudaStream_t s) const {
    if (learned) k_scan<Op, kBlock, true><<<scan_grid, kBlock, 0, s>>>(a);
    else k_scan<Op, kBlock><<<scan_grid, kBlock, 0, s>>>(a);
  }

  // One round: [selection passes], frontier scan, then the push, whose CTAs
  // decide termination and set the WHILE condition.  With `chained`, the scan
  // is launched as a programmatic dependent of the kernel before it; the push
  // always is (of the scan): its CTAs are scheduled while the scan's retire
  // and wait in griddepcontrol.wait for the scan's writes.
  void launch_round(cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                    bool chained) const {
    launch_select(s, chained);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (learned) {
      // after the threshold kernel, whose writes griddepcontrol.wait shows
      cfg.gridDim = dim3(scan_grid);
      cudaLaunchKernelEx(&cfg, k_scan<Op, kBlock, true>, a);
    } else if (chained && !a.topq) {
      cfg.gridDim = dim3(scan_grid);
      cudaLaunchKernelEx(&cfg, k_scan<Op, kBlock>, a);
    } else {
      launch_scan(s);
    }
    cfg.gridDim = dim3(push_grid);
    cudaLaunchKernelEx(&cfg, k_push<Op, kBlock>, a, h, use_cond);
  }

  // Rounds per pass of the WHILE body: the scan and push that follow a
  // stopping round return at once (the control block's status is set), so a
  // pass may hold several rounds and the loop condition is tested once per
  // pass.  Three: the rounds left in the last pass cost two launches each,
  // and fewer passes mean fewer condition tests (measured against 2 and 4 on
  // SSSP, PageRank and components).
  static constexpr int kRoundsPerPass = 3;

  // Adds WHILE(h) { ([select] ; k_scan ; k_push) x kRoundsPerPass } after
  // `deps` (graph mode).
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
      for (int u = 0; u < kRoundsPerPass; ++u) launch_round(cap, h, 1, u > 0);
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(cap, &captured);
    }
    cudaStreamDestroy(cap);
    MAITER_CUDA(e);
    return MAITER_OK;
  }

  // Host-driven rounds with events around each launch (profiling mode), and
  // optionally a trace record of sampled vertices after every push.
  maiter_status host_loop(maiter_result* r, cudaStream_t st, cudaEvent_t* e, maiter_stats& s,
                          TraceSink* trace = nullptr) const {
    for (;;) {
      // the round's launches queue up behind the hold (the host syncs on
      // every round, so without it e[0] would fire while the GPU idles)
      k_hold<<<1, 32, 0, st>>>(kHoldNs);
      MAITER_CUDA(cudaEventRecord(e[0], st));
      launch_select(st);
      launch_scan(st);
      MAITER_CUDA(cudaEventRecord(e[1], st));
      k_push<Op, kBlock><<<push_grid, kBlock, 0, st>>>(a, cudaGraphConditionalHandle{}, 0);
      MAITER_CUDA(cudaEventRecord(e[2], st));
      if (trace && trace->records < trace->max_records) {
        const int64_t o = static_cast<int64_t>(trace->records) * trace->ns;
        k_trace<Op><<<(trace->ns + 255) / 256, 256, 0, st>>>(
            a, trace->sample, trace->ns, trace->feat + o * kMlpIn, trace->dl + o, trace->vs + o,
            trace->la + o);
        ++trace->records;
      }
      MAITER_CUDA(cudaGetLastError());
      MAITER_CUDA(cudaMemcpyAsync(r->h_ctl, r->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
      MAITER_CUDA(cudaStreamSynchronize(st));
      float t1 = 0.f, t2 = 0.f;
      cudaEventElapsedTime(&t1, e[0], e[1]);
      cudaEventElapsedTime(&t2, e[1], e[2]);
      s.scan_ms += t1;
      s.push_ms += t2;
      s.push_launches++;
      s.scan_launches++;
      if (r->h_ctl->status != 0) return MAITER_OK;
    }
  }
};

}  // namespace maiter
