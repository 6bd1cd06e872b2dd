// Host side of the batched engine: query tables, query-major state, sparse
// frontiers, and the CUDA graph WHILE(cond) { k_b_take ; k_b_push } that
// advances every query of the batch in one launch.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "batch_kernels.cuh"
#include "pull_vec_kernels.cuh"
#include "sync_phase.cuh"

// Mode 3: personalised-PageRank queries of one graph, kVQ at a time, as one
// receive-side run with query vectors (pull_vec_kernels.cuh).
struct VGroup {
  int graph = 0;
  int nq = 0;
  int q[maiter::kVQ];                 // batch query of each slot
  maiter::PullVArgs a{};
  maiter::VCtl init{};
  int2* d_seeds = nullptr;            // (slot, vertex)
  float* d_seedval = nullptr;
  int nseeds = 0;
  int pull_grid = 1, prime_grid = 1, init_grid = 1;
};

struct maiter_batch {
  int device = 0;
  int nq = 0, ng = 0;
  std::vector<const maiter_graph*> graphs;
  std::vector<maiter::BQuery> hq;
  std::vector<int64_t> qn;                  // vertices of each query's graph
  std::vector<maiter::BItem> hseeds;
  int cut_large = 0, chunk = 0;
  maiter::BGraph* d_graphs = nullptr;
  maiter::BQuery* d_queries = nullptr;
  maiter::BItem* d_seeds = nullptr;
  double* v_sum = nullptr;
  double* d_sum = nullptr;
  uint32_t* v_min = nullptr;
  uint32_t* d_min = nullptr;
  unsigned* stamp = nullptr;
  maiter::BItem* items[2][maiter::kBOps] = {};
  unsigned cap[maiter::kBOps] = {};
  maiter::BChunk* chunks = nullptr;
  unsigned chunk_cap = 0;
  unsigned* qlast = nullptr;
  maiter::BCtl* ctl = nullptr;
  maiter::BCtl* h_ctl = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int exec_grid = 0;
  int64_t n_sum = 0, n_min = 0;
  // dense mode: one round-engine result per query, one WHILE branch each
  int mode = 0;
  std::vector<maiter_result*> qres;
  std::vector<int> seed_off, seed_cnt;
  int* d_qseeds = nullptr;
  maiter::DevCtl* h_ctls = nullptr;      // pinned, one per query
  int dense_grid_cap = 0;
  // mode 3: the query groups and each query's group and slot (-1: own branch)
  std::vector<VGroup> vg;
  std::vector<int> q_group, q_slot;
  maiter::VCtl* h_vctl = nullptr;        // pinned, one per group
  maiter_stats stats{};
};

namespace maiter {

constexpr int kBBlock = 256;

// Number of vertices of out-degree >= cut (sizes the large-item lists).
__global__ void k_count_large(const int* __restrict__ rp, int n, int cut, unsigned* out) {
  unsigned c = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    c += (rp[j + 1] - rp[j]) >= cut;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ------------------------------------------------------------- dense mode
// Every query is its own round-engine run (k_scan / k_push on its own v,
// Delta, frontier lists and control block) and one branch of a single CUDA
// graph: init -> seeds -> WHILE(cond_q) { k_scan ; k_push }.  Branches share
// nothing, so the GPU runs them concurrently, and each ends on its own exact
// termination test (sum |Delta| < eps_q, or no pending vertex).

template <class V, class D>
__global__ void k_dense_init(V* __restrict__ v, D* __restrict__ d, int64_t n, V vfill, D dfill,
                             DevCtl* ctl, DevCtl init) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    v[i] = vfill;
    d[i] = dfill;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *ctl = init;
}

template <class D>
__global__ void k_dense_seed(D* __restrict__ d, const int* __restrict__ seeds, int ns, D value) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ns) d[seeds[i]] = value;
}

static void free_vec(maiter_batch* b) {
  for (VGroup& G : b->vg) {
    cudaFree(G.a.v);
    cudaFree(G.a.delta);
    cudaFree(G.a.msg[0]);
    cudaFree(G.a.msg[1]);
    cudaFree(const_cast<float2*>(G.a.inv_deg));
    cudaFree(G.a.lacc);
    cudaFree(G.a.lcnt);
    cudaFree(G.a.ctl);
    cudaFree(G.d_seeds);
    cudaFree(G.d_seedval);
  }
  b->vg.clear();
  b->q_group.clear();
  b->q_slot.clear();
  if (b->h_vctl) cudaFreeHost(b->h_vctl);
  b->h_vctl = nullptr;
}

static void free_dense(maiter_batch* b) {
  free_vec(b);
  for (maiter_result* r : b->qres) maiter_result_destroy(r);
  b->qres.clear();
  cudaFree(b->d_qseeds);
  b->d_qseeds = nullptr;
  if (b->h_ctls) cudaFreeHost(b->h_ctls);
  b->h_ctls = nullptr;
}

// Mode 3: the seeds, damping and tolerances of every group's slots (also on
// a rerun with new values), into each group's seed arrays and initial
// control block.
static maiter_status vec_values(maiter_batch* b, const maiter_query* qs) {
  for (VGroup& G : b->vg) {
    VCtl c{};
    for (int s = 0; s < kVQ; ++s) c.conv_round[s] = -1;
    c.nq = G.nq;
    std::vector<int2> seeds;
    std::vector<float> vals;
    for (int s = 0; s < G.nq; ++s) {
      const maiter_query& Q = qs[G.q[s]];
      // half of the query's tolerance for the termination test, half left
      // to the FP32 rounding of its deltas and messages
      c.eps[s] = kVecEpsFrac * Q.eps;
      c.dq[s] = static_cast<float>(Q.damping);
      c.dq_lo[s] = static_cast<float>(Q.damping - static_cast<double>(c.dq[s]));
      const float init = static_cast<float>((1.0 - Q.damping) / static_cast<double>(Q.num_seeds));
      for (int i = 0; i < Q.num_seeds; ++i) {
        seeds.push_back(make_int2(s, Q.seeds[i]));
        vals.push_back(init);
      }
    }
    G.init = c;
    if (static_cast<int>(seeds.size()) != G.nseeds) {
      cudaFree(G.d_seeds);
      cudaFree(G.d_seedval);
      G.d_seeds = nullptr;
      G.d_seedval = nullptr;
      MAITER_CUDA(cudaMalloc(&G.d_seeds, sizeof(int2) * std::max<size_t>(seeds.size(), 1)));
      MAITER_CUDA(cudaMalloc(&G.d_seedval, sizeof(float) * std::max<size_t>(vals.size(), 1)));
      G.nseeds = static_cast<int>(seeds.size());
    }
    MAITER_CUDA(cudaMemcpy(G.d_seeds, seeds.data(), sizeof(int2) * seeds.size(), cudaMemcpyHostToDevice));
    MAITER_CUDA(cudaMemcpy(G.d_seedval, vals.data(), sizeof(float) * vals.size(), cudaMemcpyHostToDevice));
  }
  return MAITER_OK;
}

// Mode 3: personalised-PageRank queries grouped kVQ at a time per graph, and
// each group's query-minor state, messages and large-row accumulators.
static maiter_status vec_setup(maiter_batch* b, const maiter_query* qs) {
  const int nq = b->nq;
  b->q_group.assign(nq, -1);
  b->q_slot.assign(nq, -1);
  for (int gi = 0; gi < b->ng; ++gi) {
    for (int q = 0; q < nq; ++q) {
      if (qs[q].graph != gi || qs[q].op != MAITER_OP_SUM_F64) continue;
      if (b->vg.empty() || b->vg.back().graph != gi || b->vg.back().nq == kVQ) {
        b->vg.emplace_back();
        b->vg.back().graph = gi;
      }
      VGroup& G = b->vg.back();
      b->q_group[q] = static_cast<int>(b->vg.size()) - 1;
      b->q_slot[q] = G.nq;
      G.q[G.nq++] = q;
    }
  }
  for (VGroup& G : b->vg) {
    const maiter_graph* g = b->graphs[G.graph];
    maiter_status s = ensure_pull(g, nullptr, true);
    if (s != MAITER_OK) return s;
    const PullLayout* L = g->pullv;
    const size_t nv = static_cast<size_t>(std::max<int64_t>(g->n, 1)) * kVQ;
    PullVArgs& a = G.a;
    a.n = static_cast<int>(g->n);
    a.crp = L->crp;
    a.csrc = L->csrc;
    a.sbase = L->sbase;
    a.smask = L->smask;
    a.large = L->large;
    a.large_nch = L->large_nch;
    a.lbits = L->lbits;
    a.nlarge = L->nlarge;
    float2* inv = nullptr;
    cudaError_t e = cudaMalloc(&a.v, sizeof(double) * nv);
    if (e == cudaSuccess) e = cudaMalloc(&a.delta, sizeof(float) * nv);
    if (e == cudaSuccess) e = cudaMalloc(&a.msg[0], sizeof(float) * nv);
    if (e == cudaSuccess) e = cudaMalloc(&a.msg[1], sizeof(float) * nv);
    if (e == cudaSuccess) e = cudaMalloc(&inv, sizeof(float2) * std::max<int64_t>(g->n, 1));
    if (e == cudaSuccess)
      e = cudaMalloc(&a.lacc, sizeof(double) * kVQ * std::max(L->nlrows, 1));
    if (e == cudaSuccess) e = cudaMalloc(&a.lcnt, sizeof(unsigned) * std::max(L->nlrows, 1));
    if (e == cudaSuccess) e = cudaMalloc(&a.ctl, sizeof(VCtl));
    if (e == cudaSuccess)
      e = cudaMemset(a.lacc, 0, sizeof(double) * kVQ * std::max(L->nlrows, 1));
    if (e == cudaSuccess) e = cudaMemset(a.lcnt, 0, sizeof(unsigned) * std::max(L->nlrows, 1));
    a.inv_deg = inv;
    if (e != cudaSuccess) {
      set_error("batch allocation failed: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;
    }
    if (g->n > 0) k_vec_inv_deg<<<g->num_sms * 4, 256>>>(g->rp, static_cast<int>(g->n), inv);
    MAITER_CUDA(cudaGetLastError());
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vec_pull, kVBlock, 0);
    G.pull_grid = g->num_sms * std::max(per_sm, 1);
    G.prime_grid = std::max(1, std::min(static_cast<int>((g->n + 7) / 8), g->num_sms * 4));
    G.init_grid = std::max(1, std::min(static_cast<int>((static_cast<int64_t>(g->n) * kVQ + 255) / 256),
                                       g->num_sms * 8));
  }
  MAITER_CUDA(cudaMallocHost(&b->h_vctl, sizeof(VCtl) * std::max<size_t>(b->vg.size(), 1)));
  MAITER_CUDA(cudaDeviceSynchronize());
  return vec_values(b, qs);
}

static maiter_status dense_setup(maiter_batch* b, const maiter_query* qs) {
  const int nq = b->nq;
  b->qres.assign(nq, nullptr);
  b->seed_off.assign(nq, 0);
  b->seed_cnt.assign(nq, 0);
  std::vector<int> flat;
  for (int q = 0; q < nq; ++q) {
    const maiter_graph* g = b->graphs[qs[q].graph];
    // mode 3 runs the personalised-PageRank queries in groups (vec_setup)
    if (!(b->mode == 3 && qs[q].op == MAITER_OP_SUM_F64)) {
      maiter_status s = alloc_result(g, qs[q].op, &b->qres[q]);
      if (s != MAITER_OK) return s;
    }
    b->seed_off[q] = static_cast<int>(flat.size());
    b->seed_cnt[q] = qs[q].num_seeds;
    flat.insert(flat.end(), qs[q].seeds, qs[q].seeds + qs[q].num_seeds);
  }
  MAITER_CUDA(cudaMalloc(&b->d_qseeds, sizeof(int) * (flat.empty() ? 1 : flat.size())));
  MAITER_CUDA(cudaMemcpy(b->d_qseeds, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice));
  MAITER_CUDA(cudaMallocHost(&b->h_ctls, sizeof(DevCtl) * nq));
  MAITER_CUDA(cudaEventCreate(&b->ev0));
  MAITER_CUDA(cudaEventCreate(&b->ev1));
  if (b->mode == 3) return vec_setup(b, qs);
  return MAITER_OK;
}

// Mode 3: a group's branch, init -> seeds -> prime -> WHILE(h) { (decide ;
// pull) x 3 }, after `dep` (none: nullptr).
static maiter_status vec_add(cudaGraph_t graph, const VGroup& G, const VCtl& init,
                             cudaGraphNode_t* last) {
  PullVArgs a = G.a;
  VCtl ci = init;
  void* a1[] = {&a, &ci};
  cudaKernelNodeParams k1{};
  k1.func = reinterpret_cast<void*>(&k_vec_init);
  k1.gridDim = dim3(G.init_grid);
  k1.blockDim = dim3(256);
  k1.kernelParams = a1;
  cudaGraphNode_t n1, n2, n3, n4;
  MAITER_CUDA(cudaGraphAddKernelNode(&n1, graph, nullptr, 0, &k1));
  const int2* seeds = G.d_seeds;
  const float* vals = G.d_seedval;
  int ns = G.nseeds;
  void* a2[] = {&a, &seeds, &vals, &ns};
  cudaKernelNodeParams k2{};
  k2.func = reinterpret_cast<void*>(&k_vec_seed);
  k2.gridDim = dim3(std::max(1, (ns + 255) / 256));
  k2.blockDim = dim3(256);
  k2.kernelParams = a2;
  MAITER_CUDA(cudaGraphAddKernelNode(&n2, graph, &n1, 1, &k2));
  void* a3[] = {&a};
  cudaKernelNodeParams k3{};
  k3.func = reinterpret_cast<void*>(&k_vec_prime);
  k3.gridDim = dim3(G.prime_grid);
  k3.blockDim = dim3(kVBlock);
  k3.kernelParams = a3;
  MAITER_CUDA(cudaGraphAddKernelNode(&n3, graph, &n2, 1, &k3));
  cudaGraphConditionalHandle h;
  MAITER_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  MAITER_CUDA(cudaGraphAddNode(&n4, graph, &n3, nullptr, 1, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t cap;
  MAITER_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    for (int u = 0; u < 3; ++u) {
      cudaLaunchConfig_t cfg{};
      cfg.stream = cap;
      cfg.attrs = attr;
      cfg.gridDim = dim3(1);
      cfg.blockDim = dim3(kVQ);
      cfg.numAttrs = u > 0 ? 1 : 0;
      cudaLaunchKernelEx(&cfg, k_vec_decide, a.ctl, h, 1);
      cfg.gridDim = dim3(G.pull_grid);
      cfg.blockDim = dim3(kVBlock);
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_vec_pull, a);
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cap, &captured);
  }
  cudaStreamDestroy(cap);
  MAITER_CUDA(e);
  *last = n4;
  return MAITER_OK;
}

static VCtl vec_init(const VGroup& G, const maiter_batch_params* p) {
  VCtl c = G.init;
  c.max_rounds = p->max_rounds > 0 ? p->max_rounds : 1000000;
  return c;
}

template <class Op>
static Phase<Op> dense_phase(const maiter_batch* b, int q, const maiter_batch_params* p) {
  const BQuery& Q = b->hq[q];
  const maiter_graph* g = b->graphs[Q.graph];
  Tuning tu{};
  if (p->push_blocks_per_sm > 0) tu.push_blocks_per_sm = p->push_blocks_per_sm;
  Phase<Op> ph;
  maiter_result* r = b->qres[q];
  ph.setup(g, r, r->delta, nullptr, Q.damping, tu, false);
  // small graphs get small grids, so many queries run side by side
  const int want = static_cast<int>(std::min<int64_t>(std::max<int64_t>(g->m / 4096, 32), 1 << 30));
  if (want < ph.push_grid) ph.push_grid = want;
  return ph;
}

template <class V, class D>
static maiter_status dense_add_init(cudaGraph_t graph, const maiter_batch* b, int q, V vfill,
                                    D dfill, D seedval, const DevCtl& init, cudaGraphNode_t* last) {
  maiter_result* r = b->qres[q];
  const maiter_graph* g = b->graphs[b->hq[q].graph];
  V* v = static_cast<V*>(r->v);
  D* d = static_cast<D*>(r->delta);
  int64_t n = g->n;
  DevCtl* ctl = r->ctl;
  DevCtl ci = init;
  void* a1[] = {&v, &d, &n, &vfill, &dfill, &ctl, &ci};
  cudaKernelNodeParams k1{};
  k1.func = reinterpret_cast<void*>(&k_dense_init<V, D>);
  k1.gridDim = dim3(static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, g->num_sms * 2))));
  k1.blockDim = dim3(256);
  k1.kernelParams = a1;
  cudaGraphNode_t n1, n2;
  MAITER_CUDA(cudaGraphAddKernelNode(&n1, graph, nullptr, 0, &k1));
  const int* seeds = b->d_qseeds + b->seed_off[q];
  int ns = b->seed_cnt[q];
  D sv = seedval;
  void* a2[] = {&d, &seeds, &ns, &sv};
  cudaKernelNodeParams k2{};
  k2.func = reinterpret_cast<void*>(&k_dense_seed<D>);
  k2.gridDim = dim3((ns + 255) / 256);
  k2.blockDim = dim3(256);
  k2.kernelParams = a2;
  MAITER_CUDA(cudaGraphAddKernelNode(&n2, graph, &n1, 1, &k2));
  *last = n2;
  return MAITER_OK;
}

static DevCtl dense_ctl(const BQuery& Q, const maiter_batch_params* p, double eps) {
  DevCtl c{};
  c.eps = Q.op == 0 ? eps : 0.0;
  c.eps_in[0] = c.eps_in[1] = c.eps;
  c.max_rounds = p->max_rounds > 0 ? p->max_rounds : 1000000;
  c.sched = MAITER_SCHED_ALL;
  return c;
}

static maiter_status dense_build(maiter_batch* b, const maiter_batch_params* p,
                                 const std::vector<double>& eps) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  MAITER_CUDA(cudaGraphCreate(&b->graph, 0));
  // mode 2 chains the branches: query q's rounds start when query q - 1 has
  // stopped (its initialisation, which touches only its own buffers, may run
  // earlier)
  cudaGraphNode_t prev = nullptr;
  for (const VGroup& G : b->vg) {
    cudaGraphNode_t last;
    maiter_status s = vec_add(b->graph, G, vec_init(G, p), &last);
    if (s != MAITER_OK) return s;
  }
  for (int q = 0; q < b->nq; ++q) {
    if (!b->qres[q]) continue;   // in a mode-3 group
    const BQuery& Q = b->hq[q];
    const DevCtl init = dense_ctl(Q, p, eps[q]);
    cudaGraphNode_t deps[2], wnode;
    const size_t ndeps = (p->mode == 2 && prev) ? 2 : 1;
    deps[1] = prev;
    cudaGraphConditionalHandle h;
    MAITER_CUDA(cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault));
    maiter_status s;
    if (Q.op == 0) {
      s = dense_add_init<double, double>(b->graph, b, q, 0.0, 0.0, Q.init, init, &deps[0]);
      if (s == MAITER_OK)
        s = dense_phase<OpSumF64>(b, q, p).add_to(b->graph, deps, ndeps, h, &wnode);
    } else {
      s = dense_add_init<uint32_t, uint32_t>(b->graph, b, q, kInfU32, kInfU32, 0u, init, &deps[0]);
      if (s == MAITER_OK)
        s = dense_phase<OpMinU32>(b, q, p).add_to(b->graph, deps, ndeps, h, &wnode);
    }
    if (s != MAITER_OK) return s;
    prev = wnode;
  }
  MAITER_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return MAITER_OK;
}

static void free_batch_buffers(maiter_batch* b) {
  free_dense(b);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  cudaFree(b->d_graphs);
  cudaFree(b->d_queries);
  cudaFree(b->d_seeds);
  cudaFree(b->v_sum);
  cudaFree(b->d_sum);
  cudaFree(b->v_min);
  cudaFree(b->d_min);
  cudaFree(b->stamp);
  for (auto& s : b->items)
    for (auto& o : s) { cudaFree(o); o = nullptr; }
  cudaFree(b->chunks);
  cudaFree(b->qlast);
  cudaFree(b->ctl);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  b->d_graphs = nullptr; b->d_queries = nullptr; b->d_seeds = nullptr;
  b->v_sum = b->d_sum = nullptr; b->v_min = b->d_min = nullptr; b->stamp = nullptr;
  b->chunks = nullptr; b->qlast = nullptr; b->ctl = nullptr; b->h_ctl = nullptr;
  b->ev0 = b->ev1 = nullptr;
}

static BArgs batch_args(const maiter_batch* b) {
  BArgs a{};
  a.graphs = b->d_graphs;
  a.queries = b->d_queries;
  a.v_sum = b->v_sum;
  a.d_sum = b->d_sum;
  a.v_min = b->v_min;
  a.d_min = b->d_min;
  a.stamp = b->stamp;
  for (int s = 0; s < 2; ++s)
    for (int o = 0; o < kBOps; ++o) a.items[s][o] = b->items[s][o];
  for (int o = 0; o < kBOps; ++o) a.cap[o] = b->cap[o];
  a.chunks = b->chunks;
  a.chunk_cap = b->chunk_cap;
  a.qlast = b->qlast;
  a.ctl = b->ctl;
  a.cut_large = b->cut_large;
  a.chunk = b->chunk;
  return a;
}

// Validates the queries and builds the host tables; allocates device memory.
static maiter_status batch_setup(maiter_batch* b, const maiter_graph* const* graphs, int ng,
                                 const maiter_query* qs, int nq, const maiter_batch_params* p) {
  b->device = graphs[0]->device;
  b->ng = ng;
  b->nq = nq;
  b->mode = p->mode;
  b->graphs.assign(graphs, graphs + ng);
  b->cut_large = p->cut_large > 0 ? p->cut_large : 1024;
  b->chunk = p->chunk > 0 ? p->chunk : 1024;
  b->hq.resize(nq);
  b->qn.resize(nq);
  b->hseeds.clear();
  int64_t off[2] = {0, 0};
  int64_t m_op[2] = {0, 0};
  for (int q = 0; q < nq; ++q) {
    const maiter_query& Q = qs[q];
    const maiter_graph* g = graphs[Q.graph];
    const int op = Q.op == MAITER_OP_MIN_U32 ? 1 : 0;
    BQuery& bq = b->hq[q];
    bq.graph = Q.graph;
    bq.op = op;
    bq.off = off[op];
    bq.damping = Q.damping;
    bq.tau = op == 0 ? Q.eps / static_cast<double>(g->n) : 0.0;
    bq.init = op == 0 ? (1.0 - Q.damping) / static_cast<double>(Q.num_seeds) : 0.0;
    b->qn[q] = g->n;
    off[op] += g->n;
    m_op[op] += g->m;
    for (int s = 0; s < Q.num_seeds; ++s)
      b->hseeds.push_back(BItem{static_cast<unsigned>(q), Q.seeds[s]});
  }
  b->n_sum = off[0];
  b->n_min = off[1];
  if (b->mode != 1) return dense_setup(b, qs);
  // large-vertex counts per graph at this cut-off
  std::vector<unsigned> nlarge(ng, 0);
  {
    unsigned* d_cnt = nullptr;
    MAITER_CUDA(cudaMalloc(&d_cnt, sizeof(unsigned) * ng));
    MAITER_CUDA(cudaMemset(d_cnt, 0, sizeof(unsigned) * ng));
    for (int i = 0; i < ng; ++i)
      k_count_large<<<graphs[i]->num_sms * 2, 256>>>(graphs[i]->rp, static_cast<int>(graphs[i]->n),
                                                     b->cut_large, d_cnt + i);
    cudaError_t e = cudaMemcpy(nlarge.data(), d_cnt, sizeof(unsigned) * ng, cudaMemcpyDeviceToHost);
    cudaFree(d_cnt);
    MAITER_CUDA(e);
  }
  int64_t large_op[2] = {0, 0};
  for (int q = 0; q < nq; ++q) large_op[b->hq[q].op] += nlarge[b->hq[q].graph];
  // Capacities: each (query, vertex) sits at most once in a min frontier (round
  // stamps) and at most twice in a sum frontier (it can cross the threshold
  // again after its own update); overflow is detected and reported.
  for (int o = 0; o < kBOps; ++o) {
    const int64_t n_op = o == 0 ? off[0] : off[1];
    const int64_t mult = o == 0 ? 2 : 1;
    const int64_t c0 = n_op * mult + 1024;
    MAITER_REQUIRE(c0 < (int64_t(1) << 32),
                   "batch too large: %lld (query, vertex) states", (long long)n_op);
    b->cap[o] = static_cast<unsigned>(c0);
  }
  const int64_t ccap = (large_op[0] * 2 + large_op[1]) + (m_op[0] * 2 + m_op[1]) / b->chunk + 64;
  MAITER_REQUIRE(ccap < (int64_t(1) << 32), "batch too large for the chunk list");
  b->chunk_cap = static_cast<unsigned>(ccap);

  std::vector<BGraph> hg(ng);
  for (int i = 0; i < ng; ++i)
    hg[i] = BGraph{graphs[i]->rp, graphs[i]->col, graphs[i]->w, static_cast<int>(graphs[i]->n), 0};
  cudaError_t e = cudaSuccess;
  auto A = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes > 0 ? bytes : 1);
  };
  A(reinterpret_cast<void**>(&b->d_graphs), sizeof(BGraph) * ng);
  A(reinterpret_cast<void**>(&b->d_queries), sizeof(BQuery) * nq);
  A(reinterpret_cast<void**>(&b->d_seeds), sizeof(BItem) * b->hseeds.size());
  A(reinterpret_cast<void**>(&b->v_sum), sizeof(double) * b->n_sum);
  A(reinterpret_cast<void**>(&b->d_sum), sizeof(double) * b->n_sum);
  A(reinterpret_cast<void**>(&b->v_min), sizeof(uint32_t) * b->n_min);
  A(reinterpret_cast<void**>(&b->d_min), sizeof(uint32_t) * b->n_min);
  A(reinterpret_cast<void**>(&b->stamp), sizeof(unsigned) * b->n_min);
  for (int s = 0; s < 2; ++s)
    for (int o = 0; o < kBOps; ++o)
      A(reinterpret_cast<void**>(&b->items[s][o]), sizeof(BItem) * b->cap[o]);
  A(reinterpret_cast<void**>(&b->chunks), sizeof(BChunk) * b->chunk_cap);
  A(reinterpret_cast<void**>(&b->qlast), sizeof(unsigned) * nq);
  A(reinterpret_cast<void**>(&b->ctl), sizeof(BCtl));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_ctl, sizeof(BCtl));
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_graphs, hg.data(), sizeof(BGraph) * ng, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_queries, b->hq.data(), sizeof(BQuery) * nq, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->hseeds.empty())
    e = cudaMemcpy(b->d_seeds, b->hseeds.data(), sizeof(BItem) * b->hseeds.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error("batch allocation failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;
  }
  return MAITER_OK;
}

static int batch_grid(const maiter_batch* b, const maiter_batch_params* p) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, reinterpret_cast<const void*>(&k_b_push<kBBlock>), kBBlock, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (p->push_blocks_per_sm > 0 && per_sm > p->push_blocks_per_sm) per_sm = p->push_blocks_per_sm;
  return b->graphs[0]->num_sms * per_sm;
}

static maiter_status batch_build_graph(maiter_batch* b, int grid) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  const BArgs a = batch_args(b);
  MAITER_CUDA(cudaGraphCreate(&b->graph, 0));
  cudaGraphConditionalHandle h;
  MAITER_CUDA(cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  MAITER_CUDA(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t cap;
  MAITER_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    k_b_take<kBBlock><<<grid, kBBlock, 0, cap>>>(a);
    k_b_push<kBBlock><<<grid, kBBlock, 0, cap>>>(a, h, 1);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cap, &captured);
  }
  cudaStreamDestroy(cap);
  MAITER_CUDA(e);
  MAITER_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->exec_grid = grid;
  return MAITER_OK;
}

// Dense mode: rebuild the graph when the queries' parameters change, launch
// it once, then read every query's control block.
static maiter_status dense_run(maiter_batch* b, const maiter_batch_params* p,
                               const maiter_query* qs) {
  cudaStream_t st = static_cast<cudaStream_t>(p->stream);
  std::vector<double> eps(b->nq);
  uint64_t sig = 1469598103934665603ull;
  auto mix = [&](uint64_t x) { sig = (sig ^ x) * 1099511628211ull; };
  for (int q = 0; q < b->nq; ++q) {
    eps[q] = qs[q].eps;
    uint64_t bits;
    std::memcpy(&bits, &qs[q].eps, 8);
    mix(bits);
    std::memcpy(&bits, &qs[q].damping, 8);
    mix(bits);
    for (int s = 0; s < qs[q].num_seeds; ++s) mix(static_cast<uint64_t>(qs[q].seeds[s]));
  }
  mix(static_cast<uint64_t>(p->max_rounds));
  mix(static_cast<uint64_t>(p->push_blocks_per_sm));
  mix(static_cast<uint64_t>(p->mode));
  const bool profile = (p->flags & MAITER_FLAG_PROFILE_KERNELS) != 0;
  if (!profile && (!b->exec || b->exec_grid != static_cast<int>(sig & 0x7fffffff))) {
    maiter_status s = dense_build(b, p, eps);
    if (s != MAITER_OK) return s;
    b->exec_grid = static_cast<int>(sig & 0x7fffffff);
  }
  maiter_stats& s = b->stats;
  s = maiter_stats{};
  MAITER_CUDA(cudaEventRecord(b->ev0, st));
  if (profile) {
    // queries one after another, each host-driven with events per kernel
    cudaEvent_t e[3];
    for (auto& x : e) MAITER_CUDA(cudaEventCreate(&x));
    for (const VGroup& G : b->vg) {
      // a group host-driven: events around each pull
      k_vec_init<<<G.init_grid, 256, 0, st>>>(G.a, vec_init(G, p));
      k_vec_seed<<<std::max(1, (G.nseeds + 255) / 256), 256, 0, st>>>(G.a, G.d_seeds, G.d_seedval,
                                                                        G.nseeds);
      k_vec_prime<<<G.prime_grid, kVBlock, 0, st>>>(G.a);
      for (;;) {
        k_vec_decide<<<1, kVQ, 0, st>>>(G.a.ctl, cudaGraphConditionalHandle{}, 0);
        k_hold<<<1, 32, 0, st>>>(kHoldNs);
        MAITER_CUDA(cudaEventRecord(e[0], st));
        k_vec_pull<<<G.pull_grid, kVBlock, 0, st>>>(G.a);
        MAITER_CUDA(cudaEventRecord(e[1], st));
        MAITER_CUDA(cudaGetLastError());
        VCtl* hc = b->h_vctl;
        MAITER_CUDA(cudaMemcpyAsync(hc, G.a.ctl, sizeof(VCtl), cudaMemcpyDeviceToHost, st));
        MAITER_CUDA(cudaStreamSynchronize(st));
        if (hc->status != 0) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, e[0], e[1]);
        s.push_ms += t;
        s.push_launches++;
      }
    }
    for (int q = 0; q < b->nq; ++q) {
      if (!b->qres[q]) continue;   // in a mode-3 group
      const BQuery& Q = b->hq[q];
      maiter_result* r = b->qres[q];
      const maiter_graph* g = b->graphs[Q.graph];
      const DevCtl init = dense_ctl(Q, p, eps[q]);
      const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((g->n + 255) / 256, g->num_sms * 2)));
      const int ns = b->seed_cnt[q];
      if (Q.op == 0) {
        k_dense_init<double, double><<<grid, 256, 0, st>>>(static_cast<double*>(r->v),
            static_cast<double*>(r->delta), g->n, 0.0, 0.0, r->ctl, init);
        k_dense_seed<double><<<(ns + 255) / 256, 256, 0, st>>>(static_cast<double*>(r->delta),
            b->d_qseeds + b->seed_off[q], ns, Q.init);
        maiter_status ls = dense_phase<OpSumF64>(b, q, p).host_loop(r, st, e, s);
        if (ls != MAITER_OK) return ls;
      } else {
        k_dense_init<uint32_t, uint32_t><<<grid, 256, 0, st>>>(static_cast<uint32_t*>(r->v),
            static_cast<uint32_t*>(r->delta), g->n, kInfU32, kInfU32, r->ctl, init);
        k_dense_seed<uint32_t><<<(ns + 255) / 256, 256, 0, st>>>(static_cast<uint32_t*>(r->delta),
            b->d_qseeds + b->seed_off[q], ns, 0u);
        maiter_status ls = dense_phase<OpMinU32>(b, q, p).host_loop(r, st, e, s);
        if (ls != MAITER_OK) return ls;
      }
    }
    for (auto& x : e) cudaEventDestroy(x);
  } else {
    MAITER_CUDA(cudaGraphLaunch(b->exec, st));
  }
  MAITER_CUDA(cudaEventRecord(b->ev1, st));
  for (int q = 0; q < b->nq; ++q)
    if (b->qres[q])
      MAITER_CUDA(cudaMemcpyAsync(b->h_ctls + q, b->qres[q]->ctl, sizeof(DevCtl),
                                  cudaMemcpyDeviceToHost, st));
  for (size_t i = 0; i < b->vg.size(); ++i)
    MAITER_CUDA(cudaMemcpyAsync(b->h_vctl + i, b->vg[i].a.ctl, sizeof(VCtl),
                                cudaMemcpyDeviceToHost, st));
  MAITER_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  s.elapsed_ms = ms;
  int worst = 1;
  for (size_t i = 0; i < b->vg.size(); ++i) {
    const VCtl& h = b->h_vctl[i];
    const VGroup& G = b->vg[i];
    const maiter_graph* g = b->graphs[G.graph];
    s.rounds = std::max<int64_t>(s.rounds, static_cast<int64_t>(h.rounds));
    // every round updates every vertex of every slot in use
    s.activations += static_cast<int64_t>(h.rounds) * g->n * G.nq;
    s.edge_pushes += static_cast<int64_t>(h.rounds) * g->m * G.nq;
    // init, seeds, prime, then per round a decision and a pull (the graph
    // runs whole passes of three rounds; profiling adds a hold per round)
    const int64_t ran = static_cast<int64_t>(h.rounds) + 1;
    s.kernel_launches += 3 + (profile ? 3 * ran : 2 * 3 * ((ran + 2) / 3));
    if (h.status != 1) worst = h.status;
  }
  for (int q = 0; q < b->nq; ++q) {
    if (!b->qres[q]) continue;
    const DevCtl& h = b->h_ctls[q];
    s.rounds = std::max<int64_t>(s.rounds, static_cast<int64_t>(h.rounds));
    s.activations += static_cast<int64_t>(h.activations);
    s.edge_pushes += static_cast<int64_t>(h.pushes);
    s.residual = std::max(s.residual, h.residual);
    // init + seed, then per round a scan and a push (and the profiling
    // loop's hold); the graph's WHILE body runs whole passes of
    // kRoundsPerPass rounds, the last of them ending in the stopping round
    const int64_t ran = static_cast<int64_t>(h.rounds) + 1;
    constexpr int64_t kPass = Phase<OpMinU32>::kRoundsPerPass;
    s.kernel_launches += 2 + (profile ? 3 * ran : 2 * kPass * ((ran + kPass - 1) / kPass));
    if (h.status != 1) worst = h.status;
  }
  s.converged = worst == 1;
  if (worst == 1) {
    s.status = MAITER_OK;
  } else if (worst == 2) {
    s.status = MAITER_ERR_NOT_CONVERGED;
    set_error("round cap reached before every query converged");
  } else {
    s.status = MAITER_ERR_OOM;
    set_error("a frontier outgrew its capacity");
  }
  return static_cast<maiter_status>(s.status);
}

static maiter_status batch_run(maiter_batch* b, const maiter_batch_params* p) {
  DeviceGuard guard(b->device);
  cudaStream_t st = static_cast<cudaStream_t>(p->stream);
  const int grid = batch_grid(b, p);
  const bool profile = (p->flags & MAITER_FLAG_PROFILE_KERNELS) != 0;
  if (!profile && (!b->exec || b->exec_grid != grid)) {
    maiter_status s = batch_build_graph(b, grid);
    if (s != MAITER_OK) return s;
  }
  // identities everywhere (0 for +, infinity for min), then the seeds
  MAITER_CUDA(cudaMemsetAsync(b->v_sum, 0, sizeof(double) * b->n_sum, st));
  MAITER_CUDA(cudaMemsetAsync(b->d_sum, 0, sizeof(double) * b->n_sum, st));
  MAITER_CUDA(cudaMemsetAsync(b->v_min, 0xFF, sizeof(uint32_t) * b->n_min, st));
  MAITER_CUDA(cudaMemsetAsync(b->d_min, 0xFF, sizeof(uint32_t) * b->n_min, st));
  MAITER_CUDA(cudaMemsetAsync(b->stamp, 0, sizeof(unsigned) * b->n_min, st));
  MAITER_CUDA(cudaMemsetAsync(b->qlast, 0, sizeof(unsigned) * b->nq, st));
  BCtl c{};
  c.rset = 0;
  c.wset = 1;
  c.max_rounds = p->max_rounds > 0 ? p->max_rounds : 1000000;
  *b->h_ctl = c;
  MAITER_CUDA(cudaMemcpyAsync(b->ctl, b->h_ctl, sizeof(BCtl), cudaMemcpyHostToDevice, st));
  const BArgs a = batch_args(b);
  const int nseeds = static_cast<int>(b->hseeds.size());
  MAITER_CUDA(cudaEventRecord(b->ev0, st));
  if (nseeds > 0)
    k_b_seed<<<(nseeds + 255) / 256, 256, 0, st>>>(a, b->d_seeds, nseeds);
  MAITER_CUDA(cudaGetLastError());
  maiter_stats& s = b->stats;
  s = maiter_stats{};
  if (profile) {
    cudaEvent_t e[3];
    for (auto& x : e) MAITER_CUDA(cudaEventCreate(&x));
    for (;;) {
      MAITER_CUDA(cudaEventRecord(e[0], st));
      k_b_take<kBBlock><<<grid, kBBlock, 0, st>>>(a);
      MAITER_CUDA(cudaEventRecord(e[1], st));
      k_b_push<kBBlock><<<grid, kBBlock, 0, st>>>(a, cudaGraphConditionalHandle{}, 0);
      MAITER_CUDA(cudaEventRecord(e[2], st));
      MAITER_CUDA(cudaGetLastError());
      MAITER_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
      MAITER_CUDA(cudaStreamSynchronize(st));
      float t1 = 0.f, t2 = 0.f;
      cudaEventElapsedTime(&t1, e[0], e[1]);
      cudaEventElapsedTime(&t2, e[1], e[2]);
      s.scan_ms += t1;   // the take/expand kernel
      s.push_ms += t2;
      s.scan_launches++;
      s.push_launches++;
      if (b->h_ctl->status != 0) break;
    }
    for (auto& x : e) cudaEventDestroy(x);
  } else if (nseeds > 0) {
    MAITER_CUDA(cudaGraphLaunch(b->exec, st));
  }
  MAITER_CUDA(cudaEventRecord(b->ev1, st));
  MAITER_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
  MAITER_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  const BCtl& h = *b->h_ctl;
  s.rounds = static_cast<int64_t>(h.rounds);
  s.activations = static_cast<int64_t>(h.updates);
  s.edge_pushes = static_cast<int64_t>(h.pushes);
  s.residual = 0.0;
  s.elapsed_ms = ms;
  const int status = nseeds == 0 ? 1 : h.status;
  s.converged = status == 1;
  s.kernel_launches = (nseeds > 0 ? 1 : 0) + 2 * static_cast<int64_t>(h.rounds);
  if (status == 1) {
    s.status = MAITER_OK;
  } else if (status == 2) {
    s.status = MAITER_ERR_NOT_CONVERGED;
    set_error("round cap reached before every query converged");
  } else {
    s.status = MAITER_ERR_OOM;
    set_error("a batch frontier outgrew its capacity");
  }
  return static_cast<maiter_status>(s.status);
}

}  // namespace maiter

using namespace maiter;

extern "C" {

void maiter_batch_params_default(maiter_batch_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->max_rounds = 1000000;
  p->cut_large = 1024;
  p->chunk = 1024;
  p->push_blocks_per_sm = 0;
}

void maiter_batch_destroy(maiter_batch* b) {
  if (!b) return;
  DeviceGuard guard(b->device);
  free_batch_buffers(b);
  delete b;
}

maiter_status maiter_run_batch(const maiter_graph* const* graphs, int32_t num_graphs,
                               const maiter_query* queries, int32_t num_queries,
                               const maiter_batch_params* p, maiter_batch** out) {
  set_error("%s", "");
  cudaGetLastError();
  MAITER_REQUIRE(graphs && queries && p && out, "maiter_run_batch: NULL argument");
  MAITER_REQUIRE(num_graphs >= 1 && num_queries >= 1, "need at least one graph and one query");
  for (int i = 0; i < num_graphs; ++i) {
    MAITER_REQUIRE(graphs[i], "graph %d is NULL", i);
    MAITER_REQUIRE(!graphs[i]->invalid, "graph %d: its last update failed validation", i);
    MAITER_REQUIRE(graphs[i]->device == graphs[0]->device, "all graphs must be on one device");
  }
  MAITER_REQUIRE(p->cut_large >= 0 && p->chunk >= 0 && (p->chunk == 0 || p->chunk >= 32),
                 "cut_large >= 0 and chunk = 0 or >= 32");
  MAITER_REQUIRE((p->flags & ~MAITER_FLAG_PROFILE_KERNELS) == 0, "unknown flags 0x%x", p->flags);
  MAITER_REQUIRE(p->mode >= 0 && p->mode <= 3 && p->reserved == 0, "mode must be 0, 1, 2 or 3");
  for (int q = 0; q < num_queries; ++q) {
    const maiter_query& Q = queries[q];
    MAITER_REQUIRE(Q.graph >= 0 && Q.graph < num_graphs, "query %d: graph %d out of range", q, Q.graph);
    MAITER_REQUIRE(Q.op == MAITER_OP_SUM_F64 || Q.op == MAITER_OP_MIN_U32,
                   "query %d: op must be SUM_F64 (personalised PageRank) or MIN_U32 (SSSP)", q);
    MAITER_REQUIRE(Q.num_seeds >= 1 && Q.seeds, "query %d: needs at least one seed", q);
    const maiter_graph* g = graphs[Q.graph];
    for (int s = 0; s < Q.num_seeds; ++s)
      MAITER_REQUIRE(Q.seeds[s] >= 0 && Q.seeds[s] < g->n, "query %d: seed out of range", q);
    if (Q.op == MAITER_OP_SUM_F64) {
      MAITER_REQUIRE(std::isfinite(Q.damping) && Q.damping >= 0.0 && Q.damping < 1.0,
                     "query %d: damping must lie in [0, 1)", q);
      MAITER_REQUIRE(std::isfinite(Q.eps) && Q.eps > 0.0, "query %d: eps must be > 0", q);
    } else {
      MAITER_REQUIRE(g->w || g->m == 0, "query %d: SSSP needs edge weights", q);
    }
  }
  DeviceGuard guard(graphs[0]->device);
  maiter_batch* b = *out;
  bool fresh = false;
  // Reuse when the batch has the same shape; rebuild otherwise.
  bool same = b && b->nq == num_queries && b->ng == num_graphs && b->mode == p->mode &&
              b->cut_large == (p->cut_large > 0 ? p->cut_large : 1024) &&
              b->chunk == (p->chunk > 0 ? p->chunk : 1024);
  if (same) {
    for (int i = 0; i < num_graphs && same; ++i) same = b->graphs[i] == graphs[i];
    for (int q = 0; q < num_queries && same; ++q) {
      const maiter_query& Q = queries[q];
      same = b->hq[q].graph == Q.graph && b->hq[q].op == (Q.op == MAITER_OP_MIN_U32 ? 1 : 0);
      if (same && b->mode != 1) same = b->seed_cnt[q] == Q.num_seeds;
    }
  }
  if (!same) {
    if (!b) {
      b = new (std::nothrow) maiter_batch();
      MAITER_REQUIRE(b, "host allocation failed");
      fresh = true;
    } else {
      free_batch_buffers(b);
    }
    maiter_status s = batch_setup(b, graphs, num_graphs, queries, num_queries, p);
    if (s != MAITER_OK) {
      if (fresh) maiter_batch_destroy(b);
      return s;
    }
  } else if (b->mode != 1) {
    // dense, same shape: refresh damping / seed values and the seed ids
    std::vector<int> flat;
    for (int q = 0; q < num_queries; ++q) {
      const maiter_query& Q = queries[q];
      BQuery& bq = b->hq[q];
      bq.damping = Q.damping;
      bq.init = bq.op == 0 ? (1.0 - Q.damping) / static_cast<double>(Q.num_seeds) : 0.0;
      flat.insert(flat.end(), Q.seeds, Q.seeds + Q.num_seeds);
    }
    MAITER_CUDA(cudaMemcpy(b->d_qseeds, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice));
    if (b->mode == 3) {
      maiter_status s = vec_values(b, queries);
      if (s != MAITER_OK) return s;
    }
  } else {
    // same shape: refresh thresholds, seeds and damping
    b->hseeds.clear();
    for (int q = 0; q < num_queries; ++q) {
      const maiter_query& Q = queries[q];
      BQuery& bq = b->hq[q];
      bq.damping = Q.damping;
      bq.tau = bq.op == 0 ? Q.eps / static_cast<double>(b->qn[q]) : 0.0;
      bq.init = bq.op == 0 ? (1.0 - Q.damping) / static_cast<double>(Q.num_seeds) : 0.0;
      for (int s = 0; s < Q.num_seeds; ++s)
        b->hseeds.push_back(BItem{static_cast<unsigned>(q), Q.seeds[s]});
    }
    cudaFree(b->d_seeds);
    b->d_seeds = nullptr;
    MAITER_CUDA(cudaMalloc(&b->d_seeds, sizeof(BItem) * (b->hseeds.empty() ? 1 : b->hseeds.size())));
    MAITER_CUDA(cudaMemcpy(b->d_seeds, b->hseeds.data(), sizeof(BItem) * b->hseeds.size(),
                           cudaMemcpyHostToDevice));
    MAITER_CUDA(cudaMemcpy(b->d_queries, b->hq.data(), sizeof(BQuery) * num_queries,
                           cudaMemcpyHostToDevice));
  }
  maiter_status s = b->mode != 1 ? dense_run(b, p, queries) : batch_run(b, p);
  if (s == MAITER_OK || s == MAITER_ERR_NOT_CONVERGED) {
    *out = b;
  } else if (fresh) {
    maiter_batch_destroy(b);
  }
  return s;
}

maiter_status maiter_batch_get_state(const maiter_batch* b, int32_t query, void* out, int64_t count) {
  set_error("%s", "");
  MAITER_REQUIRE(b && out, "NULL argument");
  MAITER_REQUIRE(query >= 0 && query < b->nq, "query %d out of range", query);
  MAITER_REQUIRE(count == b->qn[query], "count %lld != n %lld of the query's graph",
                 (long long)count, (long long)b->qn[query]);
  DeviceGuard guard(b->device);
  const BQuery& q = b->hq[query];
  const size_t bytes = (q.op == 0 ? sizeof(double) : sizeof(uint32_t)) * count;
  if (b->mode == 3 && b->q_group[query] >= 0) {
    // the query's column of its group's query-minor state
    const VGroup& G = b->vg[b->q_group[query]];
    MAITER_CUDA(cudaMemcpy2D(out, sizeof(double), G.a.v + b->q_slot[query], sizeof(double) * kVQ,
                             sizeof(double), static_cast<size_t>(count), cudaMemcpyDefault));
  } else if (b->mode != 1)
    MAITER_CUDA(cudaMemcpy(out, b->qres[query]->v, bytes, cudaMemcpyDefault));
  else if (q.op == 0)
    MAITER_CUDA(cudaMemcpy(out, b->v_sum + q.off, bytes, cudaMemcpyDefault));
  else
    MAITER_CUDA(cudaMemcpy(out, b->v_min + q.off, bytes, cudaMemcpyDefault));
  return MAITER_OK;
}

maiter_status maiter_batch_get_stats(const maiter_batch* b, maiter_stats* out) {
  set_error("%s", "");
  MAITER_REQUIRE(b && out, "NULL argument");
  *out = b->stats;
  return MAITER_OK;
}

maiter_status maiter_batch_query_rounds(const maiter_batch* b, int32_t* out, int32_t count) {
  set_error("%s", "");
  MAITER_REQUIRE(b && out && count == b->nq, "need num_queries entries");
  DeviceGuard guard(b->device);
  if (b->mode != 1) {
    // dense: the rounds each query's own loop ran (its control block); a
    // mode-3 query: the round at which its residual fell below its eps
    for (int q = 0; q < count; ++q)
      out[q] = (b->mode == 3 && b->q_group[q] >= 0)
                   ? b->h_vctl[b->q_group[q]].conv_round[b->q_slot[q]]
                   : static_cast<int32_t>(b->h_ctls[q].rounds);
    return MAITER_OK;
  }
  MAITER_CUDA(cudaMemcpy(out, b->qlast, sizeof(int32_t) * count, cudaMemcpyDeviceToHost));
  return MAITER_OK;
}

}  // extern "C"
