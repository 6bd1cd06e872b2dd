// C ABI of libmaiter: graph upload and validation, result management, and the
// round-synchronous engine whose round loop is a CUDA graph with a device-side
// WHILE condition.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "internal.h"

namespace maiter {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// Every entry point starts here: clear this thread's message and any
// non-sticky CUDA error left by an earlier unchecked runtime call, so a later
// cudaGetLastError() reports only this call's launches.
static void begin_call() {
  g_err[0] = '\0';
  cudaGetLastError();
}

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------ graph validation

// Checks the CSR and narrows row_ptr to int32.  Bit 0: row_ptr[0] != 0 or not
// non-decreasing or row_ptr[n] != m; bit 1: a target outside [0, n).
__global__ void k_validate_rowptr(const int64_t* __restrict__ rp64, int64_t n, int64_t m,
                                  int* __restrict__ rp32, unsigned* flag) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i <= n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t x = rp64[i];
    bool bad = x < 0 || x > m;
    if (i == 0) bad |= (x != 0);
    if (i == n) bad |= (x != m);
    if (i < n) bad |= (rp64[i + 1] < x);
    if (bad) atomicOr(flag, 1u);
    rp32[i] = static_cast<int>(x);
  }
}

__global__ void k_validate_col(const int* __restrict__ col, int64_t m, int64_t n, unsigned* flag) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int k = col[e];
    if (k < 0 || k >= n) atomicOr(flag, 2u);
  }
}

// (target, weight) pairs of a weighted graph, so the min operators read each
// edge with one 8-byte load.
__global__ void k_interleave(const int* __restrict__ col, const uint32_t* __restrict__ w,
                             int64_t m, uint2* __restrict__ cw) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    cw[e] = make_uint2(static_cast<uint32_t>(col[e]), w[e]);
}

}  // namespace maiter

using namespace maiter;

extern "C" {

const char* maiter_last_error(void) { return g_err; }

const char* maiter_version(void) { return "maiter-b300 0.1 (sm_103a)"; }

maiter_status maiter_device_info(int device, char* name, int32_t len, int32_t* num_sms) {
  begin_call();
  MAITER_REQUIRE(name && len > 0 && num_sms, "NULL argument");
  int ndev = 0;
  MAITER_CUDA(cudaGetDeviceCount(&ndev));
  MAITER_REQUIRE(device >= 0 && device < ndev, "device %d out of range", device);
  cudaDeviceProp prop{};
  MAITER_CUDA(cudaGetDeviceProperties(&prop, device));
  std::snprintf(name, static_cast<size_t>(len), "%s", prop.name);
  *num_sms = prop.multiProcessorCount;
  return MAITER_OK;
}

void maiter_params_default(maiter_run_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->op = MAITER_OP_SUM_F64;
  p->g = MAITER_G_SCALE_BY_SRC;
  p->sched = MAITER_SCHED_ALL;
  p->engine = MAITER_ENGINE_SYNC;
  p->coef = nullptr;
  p->damping = 0.8;
  p->source = -1;
  p->threshold = 0.0;
  p->top_frac = 0.01;
  p->eps = 1e-8;
  p->mixed_switch = 0.01;
  p->max_rounds = 1000000;
  p->timeout_ms = 0;
  p->stream = nullptr;
}

void maiter_graph_destroy(maiter_graph* g) {
  if (!g) return;
  DeviceGuard guard(g->device);
  cudaFree(g->rp);
  cudaFree(g->col);
  cudaFree(g->w);
  cudaFree(g->cw);
  cudaFree(g->rp64);
  cudaFree(g->flag);
  cudaFree(g->lstat);
  free_bins(g);
  free_pull(g);
  delete g;
}

maiter_status maiter_graph_create(int64_t n, int64_t m, const int64_t* row_ptr,
                                  const int32_t* col, const uint32_t* w, int device,
                                  maiter_graph** out) {
  begin_call();
  MAITER_REQUIRE(out, "maiter_graph_create: out is NULL");
  *out = nullptr;
  MAITER_REQUIRE(n >= 0 && n < (int64_t(1) << 31) - 1, "n = %lld out of range [0, 2^31-1)",
                 (long long)n);
  MAITER_REQUIRE(m >= 0 && m < (int64_t(1) << 31), "m = %lld out of range [0, 2^31)",
                 (long long)m);
  MAITER_REQUIRE(row_ptr, "row_ptr is NULL");
  MAITER_REQUIRE(m == 0 || col, "col is NULL with m > 0");
  int ndev = 0;
  MAITER_CUDA(cudaGetDeviceCount(&ndev));
  MAITER_REQUIRE(device >= 0 && device < ndev, "device %d out of range (%d devices)", device, ndev);
  DeviceGuard guard(device);

  maiter_graph* g = new (std::nothrow) maiter_graph();
  MAITER_REQUIRE(g, "host allocation failed");
  g->device = device;
  g->n = n;
  g->m = m;
  cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, device);

  int64_t* rp64 = nullptr;
  unsigned* flag = nullptr;
  auto fail = [&](maiter_status s) {
    cudaFree(rp64);
    cudaFree(flag);
    maiter_graph_destroy(g);
    return s;
  };
#define GC_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                       \
      return fail(e_ == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA); \
    }                                                                                  \
  } while (0)
  GC_CUDA(cudaMalloc(&g->rp, sizeof(int) * (n + 1)));
  GC_CUDA(cudaMalloc(&g->col, sizeof(int) * (m > 0 ? m : 1)));
  if (w) GC_CUDA(cudaMalloc(&g->w, sizeof(uint32_t) * (m > 0 ? m : 1)));
  if (w) GC_CUDA(cudaMalloc(&g->cw, sizeof(uint2) * (m > 0 ? m : 1)));
  GC_CUDA(cudaMalloc(&rp64, sizeof(int64_t) * (n + 1)));
  GC_CUDA(cudaMalloc(&flag, sizeof(unsigned)));
  GC_CUDA(cudaMemset(flag, 0, sizeof(unsigned)));
  GC_CUDA(cudaMemcpy(rp64, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault));
  if (m > 0) GC_CUDA(cudaMemcpy(g->col, col, sizeof(int) * m, cudaMemcpyDefault));
  if (w && m > 0) GC_CUDA(cudaMemcpy(g->w, w, sizeof(uint32_t) * m, cudaMemcpyDefault));
  const int blocks = g->num_sms * 4;
  k_validate_rowptr<<<blocks, 256>>>(rp64, n, m, g->rp, flag);
  if (m > 0) k_validate_col<<<blocks, 256>>>(g->col, m, n, flag);
  if (w && m > 0) k_interleave<<<blocks, 256>>>(g->col, g->w, m, g->cw);
  GC_CUDA(cudaGetLastError());
  unsigned h_flag = 0;
  GC_CUDA(cudaMemcpy(&h_flag, flag, sizeof(unsigned), cudaMemcpyDeviceToHost));
#undef GC_CUDA
  if (h_flag & 1u) {
    set_error("row_ptr must start at 0, be non-decreasing and end at m = %lld", (long long)m);
    return fail(MAITER_ERR_INVALID_ARG);
  }
  if (h_flag & 2u) {
    set_error("col holds a target outside [0, n = %lld)", (long long)n);
    return fail(MAITER_ERR_INVALID_ARG);
  }
  cudaFree(rp64);
  cudaFree(flag);
  *out = g;
  return MAITER_OK;
}

maiter_status maiter_graph_update(maiter_graph* g, const int64_t* row_ptr, const int32_t* col,
                                  const uint32_t* w, void* stream) {
  begin_call();
  MAITER_REQUIRE(g && row_ptr, "maiter_graph_update: NULL argument");
  MAITER_REQUIRE(g->m == 0 || col, "col is NULL with m > 0");
  MAITER_REQUIRE((w != nullptr) == (g->w != nullptr),
                 "weights must be given exactly when the graph has them");
  DeviceGuard guard(g->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = g->n, m = g->m;
  if (!g->rp64) MAITER_CUDA(cudaMalloc(&g->rp64, sizeof(int64_t) * (n + 1)));
  if (!g->flag) MAITER_CUDA(cudaMalloc(&g->flag, sizeof(unsigned)));
  g->invalid = true;   // until this content has been validated
  MAITER_CUDA(cudaMemsetAsync(g->flag, 0, sizeof(unsigned), st));
  MAITER_CUDA(cudaMemcpyAsync(g->rp64, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, st));
  if (m > 0) MAITER_CUDA(cudaMemcpyAsync(g->col, col, sizeof(int) * m, cudaMemcpyDefault, st));
  if (w && m > 0) MAITER_CUDA(cudaMemcpyAsync(g->w, w, sizeof(uint32_t) * m, cudaMemcpyDefault, st));
  const int blocks = g->num_sms * 4;
  k_validate_rowptr<<<blocks, 256, 0, st>>>(g->rp64, n, m, g->rp, g->flag);
  if (m > 0) k_validate_col<<<blocks, 256, 0, st>>>(g->col, m, n, g->flag);
  if (w && m > 0) k_interleave<<<blocks, 256, 0, st>>>(g->col, g->w, m, g->cw);
  MAITER_CUDA(cudaGetLastError());
  unsigned h_flag = 0;
  MAITER_CUDA(cudaMemcpyAsync(&h_flag, g->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  MAITER_CUDA(cudaStreamSynchronize(st));
  // contents changed: derived data is recomputed on its next use (a free
  // only when there is something to free: cudaFree waits for the device)
  if (g->lstat) {
    cudaFree(g->lstat);
    g->lstat = nullptr;
  }
  g->wf32 = 0;
  invalidate_bins(g);
  invalidate_pull(g);
  if (h_flag & 1u) {
    set_error("row_ptr must start at 0, be non-decreasing and end at m = %lld", (long long)m);
    return MAITER_ERR_INVALID_ARG;
  }
  if (h_flag & 2u) {
    set_error("col holds a target outside [0, n = %lld)", (long long)n);
    return MAITER_ERR_INVALID_ARG;
  }
  g->invalid = false;
  return MAITER_OK;
}

void maiter_result_destroy(maiter_result* r) {
  if (!r) return;
  DeviceGuard guard(r->device);
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->graph) cudaGraphDestroy(r->graph);
  cudaFree(r->v);
  cudaFree(r->delta);
  cudaFree(r->delta_wide);
  cudaFree(r->coef);
  cudaFree(r->ecoef);
  for (int b = 0; b < 2; ++b) cudaFree(r->list[b]);
  cudaFree(r->large);
  cudaFree(r->large_d);
  cudaFree(r->ctl);
  cudaFree(r->topq);
  cudaFree(r->last_act);
  cudaFree(r->bin_msg_v);
  cudaFree(r->bin_cmsg);
  cudaFree(r->bin_msg_e);
  cudaFree(r->pull_msg);
  free_async(r);
  if (r->h_ctl) cudaFreeHost(r->h_ctl);
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
  delete r;
}

}  // extern "C"

namespace maiter {

static bool is_min_op(int op) { return op == MAITER_OP_MIN_U32 || op == MAITER_OP_MIN_F32; }
static bool is_order_op(int op) { return is_min_op(op) || op == MAITER_OP_MAX_I32; }
static size_t state_bytes(int op) { return is_order_op(op) ? 4 : 8; }
static size_t delta_bytes(int op) { return op == MAITER_OP_SUM_F64 ? 8 : 4; }
static size_t coef_bytes(int op) { return op == MAITER_OP_SUM_F64 ? 8 : 4; }

// Round-engine and asynchronous sums with g = c_j x and no caller
// coefficients: c_j = damping / outdeg(j) is tabulated once per run
// (k_degree_coef).
static bool derived_coef(const maiter_run_params* p) {
  return !p->coef && (p->engine == MAITER_ENGINE_SYNC || p->engine == MAITER_ENGINE_ASYNC) &&
         p->g == MAITER_G_SCALE_BY_SRC &&
         (p->op == MAITER_OP_SUM_F64 || p->op == MAITER_OP_SUM_MIXED);
}

template <class C>
static __global__ void k_degree_coef(const int* __restrict__ rp, int64_t n, double damping,
                                     C* __restrict__ coef) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int deg = rp[j + 1] - rp[j];
    coef[j] = deg > 0 ? static_cast<C>(damping / static_cast<double>(deg)) : C(0);
  }
}

maiter_status alloc_result(const maiter_graph* g, int op, maiter_result** out) {
  maiter_result* r = new (std::nothrow) maiter_result();
  MAITER_REQUIRE(r, "host allocation failed");
  r->g = g;
  r->device = g->device;
  r->op = op;
  r->n = g->n;
  const size_t n = static_cast<size_t>(g->n > 0 ? g->n : 1);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&r->v, n * state_bytes(op));
  if (e == cudaSuccess) e = cudaMalloc(&r->delta, n * delta_bytes(op));
  if (e == cudaSuccess && op == MAITER_OP_SUM_MIXED) e = cudaMalloc(&r->delta_wide, n * sizeof(double));
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&r->list[b], n * sizeof(int));
  // every large vertex contributes ceil(deg / kChunk) <= deg / kChunk + 1 entries
  r->large_cap = static_cast<unsigned>(n + static_cast<size_t>(g->m) / kChunk + 1);
  if (e == cudaSuccess) e = cudaMalloc(&r->large, sizeof(int2) * r->large_cap);
  if (e == cudaSuccess) e = cudaMalloc(&r->large_d, sizeof(double) * r->large_cap);
  if (e == cudaSuccess) e = cudaMalloc(&r->ctl, sizeof(DevCtl));
  if (e == cudaSuccess) e = cudaMallocHost(&r->h_ctl, sizeof(DevCtl));
  if (e == cudaSuccess) e = cudaEventCreate(&r->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&r->ev1);
  if (e != cudaSuccess) {
    set_error("result allocation failed: %s", cudaGetErrorString(e));
    maiter_result_destroy(r);
    return e == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;
  }
  *out = r;
  return MAITER_OK;
}

}  // namespace maiter

#include "sync_phase.cuh"

namespace maiter {

// The mixed-precision run is two phases: FP64 deltas until the residual has
// fallen to mixed_switch x its first value, one rounding of every delta to
// FP32, then FP32 deltas to the end.  Both phases keep v and the residual
// reduction in FP64.
struct RunPlan {
  bool mixed = false;
  Phase<OpSumF64> f64;
  Phase<OpSumWarm> warm;
  Phase<OpSumMixed> f32;
  Phase<OpMinU32> umin;
  Phase<OpMinF32> fmin;
  Phase<OpSumEdge> fedge;
  Phase<OpMaxI32> imax;
  bool edge = false;      // SUM_F64 with one coefficient per edge
};

// Float weights must be finite and >= 0 (sign bit clear, exponent not all
// ones); checked once per graph, on the first float-distance run.
static __global__ void k_check_f32(const uint32_t* __restrict__ w, int64_t m, unsigned* bad) {
  unsigned b = 0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    b |= (w[e] >= 0x7F800000u) ? 1u : 0u;   // negative, +-inf or NaN
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1u);
}

static maiter_status check_float_weights(const maiter_graph* g) {
  maiter_graph* mg = const_cast<maiter_graph*>(g);
  if (mg->wf32 == 0) {
    unsigned* bad = nullptr;
    MAITER_CUDA(cudaMalloc(&bad, sizeof(unsigned)));
    MAITER_CUDA(cudaMemset(bad, 0, sizeof(unsigned)));
    k_check_f32<<<g->num_sms * 4, 256>>>(g->w, g->m, bad);
    unsigned h = 0;
    cudaError_t e = cudaMemcpy(&h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    MAITER_CUDA(e);
    mg->wf32 = h ? 2 : 1;
  }
  MAITER_REQUIRE(mg->wf32 == 1, "float weights must be finite and >= 0");
  return MAITER_OK;
}

// The graph-static scorer features (from the in- and out-degrees), computed
// once and kept with the graph.
static maiter_status ensure_learn_static(const maiter_graph* g) {
  if (g->lstat) return MAITER_OK;
  maiter_graph* mg = const_cast<maiter_graph*>(g);
  const int64_t n1 = g->n > 0 ? g->n : 1;
  int* indeg = nullptr;
  MAITER_CUDA(cudaMalloc(&indeg, sizeof(int) * n1));
  cudaError_t e = cudaMalloc(&mg->lstat, sizeof(uint2) * n1);
  if (e == cudaSuccess) e = cudaMemset(indeg, 0, sizeof(int) * n1);
  if (e == cudaSuccess && g->m > 0) {
    k_indegree<<<g->num_sms * 4, 256>>>(g->col, g->m, indeg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && g->n > 0) {
    k_learn_static<<<g->num_sms * 4, 256>>>(g->rp, indeg, static_cast<int>(g->n), mg->lstat);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(indeg);
  if (e != cudaSuccess) {
    cudaFree(mg->lstat);
    mg->lstat = nullptr;
  }
  MAITER_CUDA(e);
  return MAITER_OK;
}

static maiter_status setup_plan(const maiter_graph* g, const maiter_run_params* p,
                                maiter_result* r, const Tuning& tu, RunPlan* plan,
                                bool track = false) {
  const void* coef = (p->coef || derived_coef(p)) ? r->coef : nullptr;
  const bool learned = p->sched == MAITER_SCHED_LEARNED;
  const bool topq = p->sched == MAITER_SCHED_TOPFRAC || learned;
  if (topq && !r->topq) {
    MAITER_CUDA(cudaMalloc(&r->topq, sizeof(TopqCtl)));
    MAITER_CUDA(cudaMemset(r->topq, 0, sizeof(TopqCtl)));
  }
  if ((learned || track) && !r->last_act)
    MAITER_CUDA(cudaMalloc(&r->last_act, sizeof(unsigned) * (g->n > 0 ? g->n : 1)));
  if (learned || track) {
    maiter_status s = ensure_learn_static(g);
    if (s != MAITER_OK) return s;
  }
  const MlpWeights* W = learned ? mlp_device_weights(p->scorer) : nullptr;
  switch (p->op) {
    case MAITER_OP_SUM_F64:
      if (p->g == MAITER_G_SCALE_BY_EDGE) {
        plan->edge = true;
        plan->fedge.setup(g, r, r->delta, nullptr, 0.0, tu, topq, W, track);
      } else {
        plan->f64.setup(g, r, r->delta, coef, p->damping, tu, topq, W, track);
      }
      break;
    case MAITER_OP_SUM_MIXED:
      plan->mixed = true;
      plan->warm.setup(g, r, r->delta_wide, coef, p->damping, tu, topq, W, track);
      plan->f32.setup(g, r, r->delta, coef, p->damping, tu, topq, W, track);
      break;
    case MAITER_OP_MAX_I32:
      plan->imax.setup(g, r, r->delta, nullptr, 0.0, tu, topq, W, track);
      break;
    case MAITER_OP_MIN_F32:
      plan->fmin.setup(g, r, r->delta, nullptr, 0.0, tu, topq, W, track);
      plan->fmin.a.bucket = p->sched == MAITER_SCHED_BUCKET;
      break;
    default:
      plan->umin.setup(g, r, r->delta, nullptr, 0.0, tu, topq, W, track);
      plan->umin.a.bucket = p->sched == MAITER_SCHED_BUCKET;
      break;
  }
  return MAITER_OK;
}

static int conversion_grid(const maiter_graph* g) { return g->num_sms * 4; }

// Builds the executable graph of a run: WHILE{round} for one phase, or
// WHILE{round FP64} -> k_to_f32 -> WHILE{round FP32} for mixed precision.
// Each body pass scans, then pushes; the push decides whether another pass
// follows, so a phase whose first scan finds nothing to do pushes nothing.
static maiter_status build_graph(const maiter_graph* g, maiter_result* r, int op,
                                 const RunPlan& plan) {
  if (r->exec) { cudaGraphExecDestroy(r->exec); r->exec = nullptr; }
  if (r->graph) { cudaGraphDestroy(r->graph); r->graph = nullptr; }
  MAITER_CUDA(cudaGraphCreate(&r->graph, 0));
  cudaGraphConditionalHandle h1;
  MAITER_CUDA(cudaGraphConditionalHandleCreate(&h1, r->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNode_t n1;
  maiter_status s;
  if (plan.edge) s = plan.fedge.add_to(r->graph, nullptr, 0, h1, &n1);
  else if (op == MAITER_OP_SUM_F64) s = plan.f64.add_to(r->graph, nullptr, 0, h1, &n1);
  else if (op == MAITER_OP_SUM_MIXED) s = plan.warm.add_to(r->graph, nullptr, 0, h1, &n1);
  else if (op == MAITER_OP_MIN_F32) s = plan.fmin.add_to(r->graph, nullptr, 0, h1, &n1);
  else if (op == MAITER_OP_MAX_I32) s = plan.imax.add_to(r->graph, nullptr, 0, h1, &n1);
  else s = plan.umin.add_to(r->graph, nullptr, 0, h1, &n1);
  if (s != MAITER_OK) return s;
  if (op == MAITER_OP_SUM_MIXED) {
    cudaGraphConditionalHandle h2;
    MAITER_CUDA(cudaGraphConditionalHandleCreate(&h2, r->graph, 0, 0));
    const double* d64 = static_cast<const double*>(r->delta_wide);
    float* d32 = static_cast<float*>(r->delta);
    int64_t n = g->n;
    DevCtl* ctl = r->ctl;
    int use_cond = 1;
    void* args[] = {&d64, &d32, &n, &ctl, &h2, &use_cond};
    cudaKernelNodeParams kp{};
    kp.func = reinterpret_cast<void*>(&k_to_f32);
    kp.gridDim = dim3(conversion_grid(g));
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    cudaGraphNode_t kn, n3;
    MAITER_CUDA(cudaGraphAddKernelNode(&kn, r->graph, &n1, 1, &kp));
    s = plan.f32.add_to(r->graph, &kn, 1, h2, &n3);
    if (s != MAITER_OK) return s;
  }
  MAITER_CUDA(cudaGraphInstantiate(&r->exec, r->graph, 0));
  return MAITER_OK;
}

static maiter_status run_sync(const maiter_graph* g, const maiter_run_params* p,
                              maiter_result* r, cudaStream_t st, TraceSink* trace = nullptr) {
  Tuning tu{};
  if (p->cut_warp > 0) tu.cut_warp = p->cut_warp;
  if (p->cut_cta > 0) tu.cut_cta = p->cut_cta;
  if (p->push_blocks_per_sm > 0) tu.push_blocks_per_sm = p->push_blocks_per_sm;
  RunPlan plan;
  {
    maiter_status ps = setup_plan(g, p, r, tu, &plan, trace != nullptr);
    if (ps != MAITER_OK) return ps;
  }
  if (r->last_act && (p->sched == MAITER_SCHED_LEARNED || trace))
    MAITER_CUDA(cudaMemsetAsync(r->last_act, 0, sizeof(unsigned) * g->n, st));
  // The executable graph bakes in the kernel arguments; rebuild it only when
  // one of them changes.
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](uint64_t x) { key = (key ^ x) * 1099511628211ull; };
  uint64_t dbits;
  std::memcpy(&dbits, &p->damping, sizeof(dbits));
  mix(static_cast<uint64_t>(p->op));
  mix(p->coef ? 1 : 0);
  mix(static_cast<uint64_t>(p->g));
  mix(dbits);
  mix(static_cast<uint64_t>(tu.cut_warp));
  mix(static_cast<uint64_t>(tu.cut_cta));
  mix(static_cast<uint64_t>(p->sched));
  mix(static_cast<uint64_t>(reinterpret_cast<uintptr_t>(p->scorer)));
  mix(static_cast<uint64_t>(tu.push_blocks_per_sm));
  const bool profile = (p->flags & MAITER_FLAG_PROFILE_KERNELS) != 0 || trace != nullptr;
  if (!profile && (!r->exec || r->exec_key != key)) {
    maiter_status s = build_graph(g, r, p->op, plan);
    if (s != MAITER_OK) return s;
    r->exec_key = key;
  }
  DevCtl c{};
  c.tau = (p->sched == MAITER_SCHED_THRESHOLD || p->sched == MAITER_SCHED_BUCKET) ? p->threshold
                                                                                : 0.0;
  c.minpend_acc[0] = c.minpend_acc[1] = kInfU32;
  c.bucket_width = (p->sched == MAITER_SCHED_BUCKET) ? p->threshold : 0.0;
  c.eps = p->eps;
  c.eps_in[0] = c.eps_in[1] = p->eps;
  c.switch_frac = plan.mixed ? p->mixed_switch : 0.0;
  c.max_rounds = p->max_rounds > 0 ? p->max_rounds : 1000000;
  c.sched = p->sched;
  *r->h_ctl = c;
  if (r->topq && (p->sched == MAITER_SCHED_TOPFRAC || p->sched == MAITER_SCHED_LEARNED)) {
    // histograms and tickets start at zero; q for this run
    MAITER_CUDA(cudaMemsetAsync(r->topq, 0, sizeof(TopqCtl), st));
    MAITER_CUDA(cudaMemcpyAsync(&r->topq->frac, &p->top_frac, sizeof(double),
                                cudaMemcpyHostToDevice, st));
  }
  MAITER_CUDA(cudaMemcpyAsync(r->ctl, r->h_ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, st));
  maiter_stats& s = r->stats;
  s = maiter_stats{};
  float ms = 0.f;
  if (profile) {
    // Host-driven loop: the same kernels and launch shapes as the graph body,
    // each bracketed by events on the launching stream.
    cudaEvent_t e[3];
    for (auto& x : e) MAITER_CUDA(cudaEventCreate(&x));
    MAITER_CUDA(cudaEventRecord(r->ev0, st));
    maiter_status ls;
    if (p->op == MAITER_OP_SUM_F64) {
      ls = plan.edge ? plan.fedge.host_loop(r, st, e, s, trace)
                     : plan.f64.host_loop(r, st, e, s, trace);
    } else if (p->op == MAITER_OP_SUM_MIXED) {
      ls = plan.warm.host_loop(r, st, e, s);
      if (ls == MAITER_OK) {
        k_to_f32<<<conversion_grid(g), 256, 0, st>>>(static_cast<const double*>(r->delta_wide),
                                                     static_cast<float*>(r->delta), g->n,
                                                     r->ctl, cudaGraphConditionalHandle{}, 0);
        MAITER_CUDA(cudaGetLastError());
        MAITER_CUDA(cudaMemcpyAsync(r->h_ctl, r->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
        MAITER_CUDA(cudaStreamSynchronize(st));
        if (r->h_ctl->status == 0) ls = plan.f32.host_loop(r, st, e, s);
      }
    } else if (p->op == MAITER_OP_MIN_F32) {
      ls = plan.fmin.host_loop(r, st, e, s, trace);
    } else if (p->op == MAITER_OP_MAX_I32) {
      ls = plan.imax.host_loop(r, st, e, s, trace);
    } else {
      ls = plan.umin.host_loop(r, st, e, s, trace);
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
  cudaEventElapsedTime(&ms, r->ev0, r->ev1);
  const DevCtl& h = *r->h_ctl;
  s.rounds = static_cast<int64_t>(h.rounds);
  s.activations = static_cast<int64_t>(h.activations);
  s.edge_pushes = static_cast<int64_t>(h.pushes);
  if (plan.mixed) {
    // the warm-up phase is the whole run if it never switched to FP32
    const bool switched = h.phase > 0;
    s.warm_rounds = static_cast<int64_t>(switched ? h.warm_rounds : h.rounds);
    s.warm_activations = static_cast<int64_t>(switched ? h.warm_activations : h.activations);
    s.warm_edge_pushes = static_cast<int64_t>(switched ? h.warm_pushes : h.pushes);
  }
  s.residual = h.residual;
  s.elapsed_ms = ms;
  s.converged = h.status == 1;
  // every phase that ran ends with one scan that did not continue
  const int64_t phases = 1 + (h.phase > 0 ? 1 : 0);
  // + 3 radix passes (TOPFRAC), + the sampled threshold (LEARNED), + the
  // hold that starts every round of the host-driven profiling loop
  const int per_round = ((p->sched == MAITER_SCHED_TOPFRAC) ? 5
                         : (p->sched == MAITER_SCHED_LEARNED) ? 3 : 2) + (profile ? 1 : 0);
  // graph mode runs whole passes of kRoundsPerPass rounds: the pass that
  // decides to stop completes its remaining rounds (which push nothing)
  constexpr int64_t kPass = Phase<OpSumF64>::kRoundsPerPass;
  const int64_t rounds_run =
      profile ? static_cast<int64_t>(h.rounds) + phases
              : kPass * ((static_cast<int64_t>(h.rounds) + phases + kPass - 1) / kPass);
  s.kernel_launches += per_round * rounds_run + (plan.mixed ? 1 : 0);
  s.status = h.status == 1 ? MAITER_OK : MAITER_ERR_NOT_CONVERGED;
  if (h.status == 3) {
    set_error("a large-vertex chunk list outgrew its capacity (residual %g)", h.residual);
  } else if (h.status != 1) {
    set_error("round cap of %lld reached before the termination test held (residual %g)",
              (long long)c.max_rounds, h.residual);
  }
  return static_cast<maiter_status>(s.status);
}

// Initial v and Delta: copies when given, else the defaults of Table 1.
template <class V, class D>
static maiter_status init_state(const maiter_graph* g, const maiter_run_params* p, void* vbuf,
                                void* dbuf, bool is_sum, cudaStream_t st, int* launches,
                                uint32_t inf = kInfU32) {
  const int64_t n = g->n;
  if (n == 0) return MAITER_OK;
  const int blocks = g->num_sms * 4;
  V* v = static_cast<V*>(vbuf);
  D* d = static_cast<D*>(dbuf);
  if (p->v0) {
    MAITER_CUDA(cudaMemcpyAsync(v, p->v0, sizeof(V) * n, cudaMemcpyDefault, st));
  } else {
    k_fill<V><<<blocks, 256, 0, st>>>(v, n, is_sum ? V(0) : V(inf));
    ++*launches;
  }
  if (p->delta0) {
    MAITER_CUDA(cudaMemcpyAsync(d, p->delta0, sizeof(D) * n, cudaMemcpyDefault, st));
  } else if (is_sum) {
    k_fill<D><<<blocks, 256, 0, st>>>(d, n, static_cast<D>(1.0 - p->damping));
    ++*launches;
  } else {
    k_fill<D><<<blocks, 256, 0, st>>>(d, n, D(inf));
    k_fill<D><<<1, 32, 0, st>>>(d + p->source, 1, D(0));
    *launches += 2;
  }
  MAITER_CUDA(cudaGetLastError());
  return MAITER_OK;
}

static __global__ void k_iota(int32_t* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] = static_cast<int32_t>(i);
}

// Max labels: copies when given, else v = -1 and Delta_j = j (Table 1).
static maiter_status init_labels(const maiter_graph* g, const maiter_run_params* p,
                                 maiter_result* r, cudaStream_t st, int* launches) {
  const int64_t n = g->n;
  if (n == 0) return MAITER_OK;
  const int blocks = g->num_sms * 4;
  int32_t* v = static_cast<int32_t*>(r->v);
  int32_t* d = static_cast<int32_t*>(r->delta);
  if (p->v0) {
    MAITER_CUDA(cudaMemcpyAsync(v, p->v0, sizeof(int32_t) * n, cudaMemcpyDefault, st));
  } else {
    k_fill<int32_t><<<blocks, 256, 0, st>>>(v, n, -1);
    ++*launches;
  }
  if (p->delta0) {
    MAITER_CUDA(cudaMemcpyAsync(d, p->delta0, sizeof(int32_t) * n, cudaMemcpyDefault, st));
  } else {
    k_iota<<<blocks, 256, 0, st>>>(d, n);
    ++*launches;
  }
  MAITER_CUDA(cudaGetLastError());
  return MAITER_OK;
}

static maiter_status run_op(const maiter_graph* g, const maiter_run_params* p, maiter_result* r,
                            cudaStream_t st, TraceSink* trace = nullptr) {
  int init_launches = 0;
  maiter_status s;
  switch (p->op) {
    case MAITER_OP_SUM_F64:
      s = init_state<double, double>(g, p, r->v, r->delta, true, st, &init_launches);
      break;
    case MAITER_OP_SUM_MIXED:
      s = init_state<double, double>(g, p, r->v, r->delta_wide, true, st, &init_launches);
      break;
    case MAITER_OP_MAX_I32:   // v = -1, Delta_j = j (Table 1, connected components)
      s = init_labels(g, p, r, st, &init_launches);
      break;
    case MAITER_OP_MIN_F32:   // +inf everywhere, 0.0f (bits 0) at the source
      s = init_state<uint32_t, uint32_t>(g, p, r->v, r->delta, false, st, &init_launches,
                                         OpMinF32::kNone);
      break;
    default:
      s = init_state<uint32_t, uint32_t>(g, p, r->v, r->delta, false, st, &init_launches);
      break;
  }
  if (s != MAITER_OK) return s;
  if (p->g == MAITER_G_SCALE_BY_EDGE) {
    if (!r->ecoef) MAITER_CUDA(cudaMalloc(&r->ecoef, sizeof(double) * (g->m > 0 ? g->m : 1)));
    if (g->m > 0)
      MAITER_CUDA(cudaMemcpyAsync(r->ecoef, p->coef, sizeof(double) * g->m, cudaMemcpyDefault, st));
  } else if (p->coef && g->n > 0) {
    if (!r->coef) MAITER_CUDA(cudaMalloc(&r->coef, coef_bytes(r->op) * g->n));
    MAITER_CUDA(cudaMemcpyAsync(r->coef, p->coef, coef_bytes(r->op) * g->n, cudaMemcpyDefault, st));
  } else if (derived_coef(p) && g->n > 0) {
    // c_j = damping / outdeg(j) once per run: the update then reads c_j
    // instead of dividing in FP64 at every vertex update (FP64 arithmetic is
    // slow on this part)
    if (!r->coef) MAITER_CUDA(cudaMalloc(&r->coef, coef_bytes(r->op) * g->n));
    if (r->op == MAITER_OP_SUM_F64)
      k_degree_coef<double><<<conversion_grid(g), 256, 0, st>>>(g->rp, g->n, p->damping,
                                                                static_cast<double*>(r->coef));
    else
      k_degree_coef<float><<<conversion_grid(g), 256, 0, st>>>(g->rp, g->n, p->damping,
                                                               static_cast<float*>(r->coef));
    MAITER_CUDA(cudaGetLastError());
    ++init_launches;
  }
  if (g->n == 0) {
    r->stats = maiter_stats{};
    r->stats.converged = 1;
    r->stats.kernel_launches = init_launches;
    return MAITER_OK;
  }
  s = (p->engine == MAITER_ENGINE_ASYNC)    ? run_async(g, p, r, st)
      : (p->engine == MAITER_ENGINE_BINNED) ? run_binned(g, p, r, st)
      : (p->engine == MAITER_ENGINE_PULL)   ? run_pull(g, p, r, st)
                                            : run_sync(g, p, r, st, trace);
  r->stats.kernel_launches += init_launches;
  return s;
}

}  // namespace maiter

namespace maiter {

static maiter_status run_impl(const maiter_graph* g, const maiter_run_params* p, maiter_result** out,
                              TraceSink* trace) {
  MAITER_REQUIRE(g && p && out, "maiter_run: NULL argument");
  MAITER_REQUIRE(!g->invalid, "the graph's last update failed validation");
  MAITER_REQUIRE(p->op >= MAITER_OP_SUM_F64 && p->op <= MAITER_OP_MAX_I32, "unknown op %d", p->op);
  const bool is_sum = !is_order_op(p->op);
  if (p->op == MAITER_OP_MAX_I32 &&
      (p->engine != MAITER_ENGINE_SYNC || p->sched == MAITER_SCHED_LEARNED ||
       p->sched == MAITER_SCHED_BUCKET)) {
    set_error("max labels run on the round engine with ALL, THRESHOLD or TOPFRAC");
    return MAITER_ERR_UNSUPPORTED;
  }
  if (p->op == MAITER_OP_MIN_F32 &&
      (p->engine != MAITER_ENGINE_SYNC || p->sched == MAITER_SCHED_LEARNED)) {
    set_error("float distances run on the round engine with a fixed schedule");
    return MAITER_ERR_UNSUPPORTED;
  }
  MAITER_REQUIRE(p->sched >= MAITER_SCHED_ALL && p->sched <= MAITER_SCHED_BUCKET,
                 "unknown sched %d", p->sched);
  if (p->sched == MAITER_SCHED_BUCKET) {
    MAITER_REQUIRE(!is_sum, "BUCKET scheduling orders distances: min only");
    MAITER_REQUIRE(std::isfinite(p->threshold) && p->threshold > 0.0,
                   "BUCKET scheduling needs a bucket width threshold > 0");
    if (p->engine != MAITER_ENGINE_SYNC) {
      set_error("BUCKET scheduling runs on the round engine");
      return MAITER_ERR_UNSUPPORTED;
    }
  }
  if (p->sched == MAITER_SCHED_LEARNED) {
    MAITER_REQUIRE(p->scorer, "LEARNED scheduling needs params.scorer");
    MAITER_REQUIRE(mlp_device(p->scorer) == g->device, "the scorer lives on another device");
    if (p->engine != MAITER_ENGINE_SYNC) {
      set_error("learned scheduling runs on the round engine");
      return MAITER_ERR_UNSUPPORTED;
    }
    MAITER_REQUIRE(p->top_frac > 0.0 && p->top_frac <= 1.0, "top_frac must lie in (0, 1]");
  }
  MAITER_REQUIRE(p->engine == MAITER_ENGINE_SYNC || p->engine == MAITER_ENGINE_ASYNC ||
                     p->engine == MAITER_ENGINE_BINNED || p->engine == MAITER_ENGINE_PULL,
                 "unknown engine %d", p->engine);
  if ((p->engine == MAITER_ENGINE_BINNED || p->engine == MAITER_ENGINE_PULL) &&
      (!is_sum || p->g != MAITER_G_SCALE_BY_SRC || p->sched != MAITER_SCHED_ALL || trace ||
       (p->flags & MAITER_FLAG_INJECT_STALL))) {
    set_error("the binned and receive-side engines run sums with g = SCALE_BY_SRC and "
              "schedule ALL");
    return MAITER_ERR_UNSUPPORTED;
  }
  MAITER_REQUIRE(p->timeout_ms >= 0, "timeout_ms must be >= 0");
  MAITER_REQUIRE(p->cut_warp >= 0 && p->cut_cta >= 0 && p->push_blocks_per_sm >= 0 &&
                     p->reserved1 == 0,
                 "tuning fields must be >= 0 (0 = default)");
  MAITER_REQUIRE(p->cut_warp == 0 || p->cut_cta == 0 || p->cut_warp <= p->cut_cta,
                 "cut_warp must not exceed cut_cta");
  if (p->engine == MAITER_ENGINE_ASYNC && p->sched == MAITER_SCHED_TOPFRAC) {
    set_error("the asynchronous engine schedules by threshold; use the sync engine for TOPFRAC");
    return MAITER_ERR_UNSUPPORTED;
  }
  MAITER_REQUIRE((p->flags & ~(MAITER_FLAG_PROFILE_KERNELS | MAITER_FLAG_INJECT_STALL)) == 0 &&
                     p->reserved0 == 0,
                 "unknown flags 0x%x", p->flags);
  if (is_sum) {
    MAITER_REQUIRE(p->g == MAITER_G_SCALE_BY_SRC ||
                       (p->g == MAITER_G_SCALE_BY_EDGE && p->op == MAITER_OP_SUM_F64),
                   "sum ops take g = MAITER_G_SCALE_BY_SRC (or SCALE_BY_EDGE with SUM_F64)");
    MAITER_REQUIRE(p->g != MAITER_G_SCALE_BY_EDGE || p->coef || g->m == 0,
                   "g = SCALE_BY_EDGE needs m per-edge coefficients");
    if (p->g == MAITER_G_SCALE_BY_EDGE &&
        (p->engine != MAITER_ENGINE_SYNC || p->sched == MAITER_SCHED_LEARNED)) {
      set_error("per-edge coefficients run on the round engine with a fixed schedule");
      return MAITER_ERR_UNSUPPORTED;
    }
    MAITER_REQUIRE(p->coef || std::isfinite(p->damping),
                   "damping must be finite when coef is NULL");
    MAITER_REQUIRE(std::isfinite(p->eps) && p->eps >= 0.0, "eps must be finite and >= 0");
    MAITER_REQUIRE(p->op != MAITER_OP_SUM_MIXED || (p->mixed_switch >= 0.0 && p->mixed_switch <= 1.0),
                   "mixed_switch must lie in [0, 1]");
    MAITER_REQUIRE(p->sched != MAITER_SCHED_THRESHOLD ||
                       (std::isfinite(p->threshold) && p->threshold >= 0.0),
                   "threshold must be finite and >= 0");
  } else if (p->op == MAITER_OP_MAX_I32) {
    MAITER_REQUIRE(p->g == MAITER_G_IDENTITY, "max takes g = MAITER_G_IDENTITY");
  } else {
    MAITER_REQUIRE(p->g == MAITER_G_ADD_EDGE, "min takes g = MAITER_G_ADD_EDGE");
    MAITER_REQUIRE(g->w || g->m == 0, "min with g = x + w needs edge weights");
    MAITER_REQUIRE(p->delta0 || (p->source >= 0 && p->source < g->n),
                   "min without delta0 needs a source in [0, n)");
  }
  MAITER_REQUIRE(p->sched != MAITER_SCHED_TOPFRAC || (p->top_frac > 0.0 && p->top_frac <= 1.0),
                 "top_frac must lie in (0, 1]");
  DeviceGuard guard(g->device);
  if (p->op == MAITER_OP_MIN_F32 && g->m > 0) {
    maiter_status ws = check_float_weights(g);
    if (ws != MAITER_OK) return ws;
  }
  maiter_result* r = *out;
  bool fresh = false;
  if (r) {
    MAITER_REQUIRE(r->g == g && r->op == p->op,
                   "the result passed for reuse belongs to another graph or op");
  } else {
    maiter_status s = alloc_result(g, p->op, &r);
    if (s != MAITER_OK) return s;
    fresh = true;
  }
  cudaStream_t st = static_cast<cudaStream_t>(p->stream);
  maiter_status s = run_op(g, p, r, st, trace);
  if (s == MAITER_OK || s == MAITER_ERR_NOT_CONVERGED || s == MAITER_ERR_TIMEOUT) {
    *out = r;
  } else if (fresh) {
    maiter_result_destroy(r);
  }
  return s;
}

}  // namespace maiter

extern "C" {

maiter_status maiter_run(const maiter_graph* g, const maiter_run_params* p, maiter_result** out) {
  begin_call();
  return run_impl(g, p, out, nullptr);
}

maiter_status maiter_trace(const maiter_graph* g, const maiter_run_params* p,
                           const int32_t* sample, int32_t num_sample, int32_t max_records,
                           float* features, double* delta, double* v, uint32_t* last_update,
                           int32_t* records, maiter_result** out) {
  begin_call();
  MAITER_REQUIRE(g && p && sample && features && delta && v && last_update && records && out,
                 "maiter_trace: NULL argument");
  MAITER_REQUIRE(num_sample > 0 && max_records > 0, "num_sample and max_records must be > 0");
  MAITER_REQUIRE(p->op == MAITER_OP_SUM_F64 || p->op == MAITER_OP_MIN_U32,
                 "traces are recorded for SUM_F64 and MIN_U32 runs");
  MAITER_REQUIRE(p->engine == MAITER_ENGINE_SYNC && p->sched != MAITER_SCHED_LEARNED,
                 "traces come from the round engine with a fixed schedule");
  for (int i = 0; i < num_sample; ++i)
    MAITER_REQUIRE(sample[i] >= 0 && sample[i] < g->n, "sample id out of range");
  DeviceGuard guard(g->device);
  const size_t rows = static_cast<size_t>(num_sample) * static_cast<size_t>(max_records);
  TraceSink sink;
  int* d_sample = nullptr;
  cudaError_t e = cudaMalloc(&d_sample, sizeof(int) * num_sample);
  if (e == cudaSuccess) e = cudaMalloc(&sink.feat, sizeof(float) * kMlpIn * rows);
  if (e == cudaSuccess) e = cudaMalloc(&sink.dl, sizeof(double) * rows);
  if (e == cudaSuccess) e = cudaMalloc(&sink.vs, sizeof(double) * rows);
  if (e == cudaSuccess) e = cudaMalloc(&sink.la, sizeof(unsigned) * rows);
  if (e == cudaSuccess) e = cudaMemcpy(d_sample, sample, sizeof(int) * num_sample, cudaMemcpyHostToDevice);
  maiter_status s = MAITER_ERR_CUDA;
  if (e == cudaSuccess) {
    sink.sample = d_sample;
    sink.ns = num_sample;
    sink.max_records = max_records;
    s = run_impl(g, p, out, &sink);
    const size_t got = static_cast<size_t>(sink.records) * num_sample;
    if (s == MAITER_OK || s == MAITER_ERR_NOT_CONVERGED) {
      e = cudaMemcpy(features, sink.feat, sizeof(float) * kMlpIn * got, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(delta, sink.dl, sizeof(double) * got, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(v, sink.vs, sizeof(double) * got, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(last_update, sink.la, sizeof(unsigned) * got, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        set_error("trace copy failed: %s", cudaGetErrorString(e));
        s = MAITER_ERR_CUDA;
      }
      *records = sink.records;
    }
  } else {
    set_error("trace buffers: %s", cudaGetErrorString(e));
    s = e == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;
  }
  cudaFree(d_sample);
  cudaFree(sink.feat);
  cudaFree(sink.dl);
  cudaFree(sink.vs);
  cudaFree(sink.la);
  return s;
}

static maiter_status copy_out(const maiter_result* r, const void* src, size_t elem, void* out,
                              int64_t count) {
  MAITER_REQUIRE(r && out, "NULL argument");
  MAITER_REQUIRE(count == r->n, "count %lld != n %lld", (long long)count, (long long)r->n);
  if (count == 0) return MAITER_OK;
  DeviceGuard guard(r->device);
  MAITER_CUDA(cudaMemcpy(out, src, elem * count, cudaMemcpyDefault));
  return MAITER_OK;
}

maiter_status maiter_get_state(const maiter_result* r, void* out, int64_t count) {
  begin_call();
  MAITER_REQUIRE(r, "NULL result");
  return copy_out(r, r->v, state_bytes(r->op), out, count);
}

maiter_status maiter_get_delta(const maiter_result* r, void* out, int64_t count) {
  begin_call();
  MAITER_REQUIRE(r, "NULL result");
  return copy_out(r, r->delta, delta_bytes(r->op), out, count);
}

maiter_status maiter_get_stats(const maiter_result* r, maiter_stats* out) {
  begin_call();
  MAITER_REQUIRE(r && out, "NULL argument");
  *out = r->stats;
  return MAITER_OK;
}

}  // extern "C"
