// Host side of the persistent asynchronous engine: buffers, the CUDA graph
// WHILE(cond) { k_async_seed ; k_async }, and the profiling loop.
#include <cstring>

#include "internal.h"

namespace maiter {

constexpr int kAsyncBlock = 256;

void free_async(maiter_result* r) {
  if (r->aexec) cudaGraphExecDestroy(r->aexec);
  if (r->agraph) cudaGraphDestroy(r->agraph);
  cudaFree(r->actl);
  if (r->h_actl) cudaFreeHost(r->h_actl);
  r->aexec = nullptr;
  r->agraph = nullptr;
  r->actl = nullptr;
  r->h_actl = nullptr;
}

static maiter_status alloc_async(const maiter_graph*, maiter_result* r) {
  if (r->actl) return MAITER_OK;
  cudaError_t e = cudaMalloc(&r->actl, sizeof(AsyncCtl));
  if (e == cudaSuccess) e = cudaMallocHost(&r->h_actl, sizeof(AsyncCtl));
  if (e != cudaSuccess) {
    set_error("async buffers: %s", cudaGetErrorString(e));
    free_async(r);
    return e == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;
  }
  return MAITER_OK;
}

template <class Op>
struct AsyncPlan {
  AArgs<Op> a{};
  int grid = 1, seed_grid = 1;

  void setup(const maiter_graph* g, maiter_result* r, const void* coef, double damping) {
    a.n = static_cast<int>(g->n);
    a.rp = g->rp;
    a.edges.col = g->col;
    a.edges.cw = g->cw;
    a.edges.w = g->w;
    a.coef = static_cast<const typename Op::C*>(coef);
    a.damping = damping;
    a.v = static_cast<typename Op::V*>(r->v);
    a.delta = static_cast<typename Op::D*>(r->delta);
    a.ctl = r->actl;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, reinterpret_cast<const void*>(&k_async<Op, kAsyncBlock>), kAsyncBlock, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    // persistent: every CTA resident at once (an idle CTA waits for the others)
    grid = g->num_sms * per_sm;
    seed_grid = g->num_sms * 4;
    const int need = static_cast<int>((g->n + kAsyncBlock - 1) / kAsyncBlock);
    if (need < seed_grid) seed_grid = need > 0 ? need : 1;
  }

  void launch_epoch(cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) const {
    k_async_seed<Op, kAsyncBlock><<<seed_grid, kAsyncBlock, 0, s>>>(a, h, use_cond);
    k_async<Op, kAsyncBlock><<<grid, kAsyncBlock, 0, s>>>(a);
  }

  maiter_status build(maiter_result* r) const {
    if (r->aexec) { cudaGraphExecDestroy(r->aexec); r->aexec = nullptr; }
    if (r->agraph) { cudaGraphDestroy(r->agraph); r->agraph = nullptr; }
    MAITER_CUDA(cudaGraphCreate(&r->agraph, 0));
    cudaGraphConditionalHandle h;
    MAITER_CUDA(cudaGraphConditionalHandleCreate(&h, r->agraph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MAITER_CUDA(cudaGraphAddNode(&node, r->agraph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t cap;
    MAITER_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      launch_epoch(cap, h, 1);
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(cap, &captured);
    }
    cudaStreamDestroy(cap);
    MAITER_CUDA(e);
    MAITER_CUDA(cudaGraphInstantiate(&r->aexec, r->agraph, 0));
    return MAITER_OK;
  }
};

template <class Op>
static maiter_status run_async_op(const maiter_graph* g, const maiter_run_params* p,
                                  maiter_result* r, cudaStream_t st) {
  // r->coef holds the caller's coefficients, or c_j = damping / outdeg(j)
  // tabulated for this run (no FP64 divide per update)
  const void* coef = (p->coef || Op::kIsSum) ? r->coef : nullptr;
  AsyncPlan<Op> plan;
  plan.setup(g, r, coef, p->damping);
  const bool profile = (p->flags & MAITER_FLAG_PROFILE_KERNELS) != 0;
  uint64_t key = 0x9e3779b97f4a7c15ull ^ static_cast<uint64_t>(p->op);
  uint64_t dbits;
  std::memcpy(&dbits, &p->damping, sizeof(dbits));
  key = (key ^ dbits) * 1099511628211ull;
  key = (key ^ (p->coef ? 1u : 0u)) * 1099511628211ull;
  if (!profile && (!r->aexec || r->aexec_key != key)) {
    maiter_status s = plan.build(r);
    if (s != MAITER_OK) return s;
    r->aexec_key = key;
  }
  AsyncCtl c{};
  if (Op::kIsSum) {
    // All pending vertices: a vertex is worth an update once its delta
    // exceeds eps / (2n), so a quiescent launch leaves sum |Delta| <= eps / 2;
    // each launch raises that to a fraction of the mean delta (k_async_seed).
    c.tau = (p->sched == MAITER_SCHED_THRESHOLD) ? p->threshold
                                                 : p->eps / (2.0 * static_cast<double>(g->n));
    c.theta = c.tau;
  }
  c.grid = plan.grid;
  c.eps = p->eps;
  c.max_epochs = p->max_rounds > 0 ? p->max_rounds : 1000000;
  const long long tmo = p->timeout_ms > 0 ? p->timeout_ms : 10000;
  c.timeout_ns = static_cast<unsigned long long>(tmo) * 1000000ull;
  c.inject_stall = (p->flags & MAITER_FLAG_INJECT_STALL) ? 1 : 0;
  *r->h_actl = c;
  MAITER_CUDA(cudaMemcpyAsync(r->actl, r->h_actl, sizeof(AsyncCtl), cudaMemcpyHostToDevice, st));
  maiter_stats& s = r->stats;
  s = maiter_stats{};
  int64_t epochs_run = 0;
  MAITER_CUDA(cudaEventRecord(r->ev0, st));
  if (profile) {
    cudaEvent_t e[3];
    for (auto& x : e) MAITER_CUDA(cudaEventCreate(&x));
    for (;;) {
      MAITER_CUDA(cudaEventRecord(e[0], st));
      k_async_seed<Op, kAsyncBlock><<<plan.seed_grid, kAsyncBlock, 0, st>>>(
          plan.a, cudaGraphConditionalHandle{}, 0);
      MAITER_CUDA(cudaEventRecord(e[1], st));
      k_async<Op, kAsyncBlock><<<plan.grid, kAsyncBlock, 0, st>>>(plan.a);
      MAITER_CUDA(cudaEventRecord(e[2], st));
      MAITER_CUDA(cudaGetLastError());
      MAITER_CUDA(cudaMemcpyAsync(r->h_actl, r->actl, sizeof(AsyncCtl), cudaMemcpyDeviceToHost, st));
      MAITER_CUDA(cudaStreamSynchronize(st));
      float t1 = 0.f, t2 = 0.f;
      cudaEventElapsedTime(&t1, e[0], e[1]);
      cudaEventElapsedTime(&t2, e[1], e[2]);
      s.scan_ms += t1;
      s.push_ms += t2;
      s.scan_launches++;
      s.push_launches++;
      ++epochs_run;
      if (r->h_actl->status != 0) break;
    }
    for (auto& x : e) cudaEventDestroy(x);
  } else {
    MAITER_CUDA(cudaGraphLaunch(r->aexec, st));
  }
  MAITER_CUDA(cudaEventRecord(r->ev1, st));
  MAITER_CUDA(cudaMemcpyAsync(r->h_actl, r->actl, sizeof(AsyncCtl), cudaMemcpyDeviceToHost, st));
  MAITER_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, r->ev0, r->ev1);
  const AsyncCtl& h = *r->h_actl;
  s.rounds = static_cast<int64_t>(h.epochs);
  s.activations = static_cast<int64_t>(h.updates);
  s.edge_pushes = static_cast<int64_t>(h.pushes);
  s.residual = h.residual;
  s.elapsed_ms = ms;
  s.converged = h.status == 1;
  s.kernel_launches += 2 * (static_cast<int64_t>(h.epochs) + 1);
  if (h.status == 1) {
    s.status = MAITER_OK;
  } else if (h.status == 2) {
    s.status = MAITER_ERR_NOT_CONVERGED;
    set_error("epoch cap of %lld reached before the termination test held (residual %g)",
              (long long)c.max_epochs, h.residual);
  } else {
    s.status = MAITER_ERR_TIMEOUT;
    set_error("a bounded device wait of the asynchronous engine ran out (status %d); the "
              "state is a valid DAIC state and can be resumed", h.status);
  }
  return static_cast<maiter_status>(s.status);
}

maiter_status run_async(const maiter_graph* g, const maiter_run_params* p, maiter_result* r,
                        cudaStream_t st) {
  maiter_status s = alloc_async(g, r);
  if (s != MAITER_OK) return s;
  switch (p->op) {
    case MAITER_OP_SUM_F64: return run_async_op<OpSumF64>(g, p, r, st);
    case MAITER_OP_MIN_U32: return run_async_op<OpMinU32>(g, p, r, st);
    default:
      set_error("the asynchronous engine serves SUM_F64 and MIN_U32");
      return MAITER_ERR_UNSUPPORTED;
  }
}

}  // namespace maiter
