// Host-side internals shared by the translation units of libmaiter.
#pragma once
#include <cstdint>
#include <cstdio>
#include <string>

#include <cuda_runtime.h>

#include "../../include/maiter.h"
#include "daic_kernels.cuh"
#include "async_kernels.cuh"
#include "topq_kernels.cuh"
#include "learned_kernels.cuh"

namespace maiter {

void set_error(const char* fmt, ...);

#define MAITER_CUDA(call)                                                              \
  do {                                                                                 \
    cudaError_t err_ = (call);                                                         \
    if (err_ != cudaSuccess) {                                                         \
      ::maiter::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(err_),    \
                          __FILE__, __LINE__);                                         \
      return err_ == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;     \
    }                                                                                  \
  } while (0)

#define MAITER_REQUIRE(cond, ...)                     \
  do {                                                \
    if (!(cond)) {                                    \
      ::maiter::set_error(__VA_ARGS__);               \
      return MAITER_ERR_INVALID_ARG;                  \
    }                                                 \
  } while (0)

// Restores the calling thread's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

bool is_device_pointer(const void* p);

// Degree cut-offs of the push kernel's three granularities and launch shape.
struct Tuning {
  int cut_warp = 32;    // out-degree below this: warp-gathered small path
  int cut_cta = 512;    // out-degree at or above this: one CTA per kChunk edges
  int push_blocks_per_sm = 0;   // 0 = occupancy maximum
  int scan_blocks_per_sm = 0;   // 0 = occupancy maximum
};

}  // namespace maiter

namespace maiter {
struct BinLayout;   // binned engine: the edges by (sender cell, receiver bin)

// Receive-side engine: the transpose of a graph and its chunk list for rows of
// high in-degree (pull_engine.cu builds it; the batch engine reads it too).
struct PullLayout {
  bool valid = false;
  int cut = 0, chunk = 0;  // largest row of a group; in-edges per chunk of a larger row
  int nlarge = 0;          // chunk entries
  int nlrows = 0;          // rows cut into chunks
  int* crp = nullptr;      // n + 1: offsets of the small rows' in-edges
  int* csrc = nullptr;     // m: small rows' in-edges, then the large rows' (tail)
  unsigned char* crow = nullptr;   // m: row within its group of every in-edge
  unsigned* lbits = nullptr;       // ceil(n / 32) large-row flags
  int4* large = nullptr;   // nlarge entries
  int* large_nch = nullptr;
  double* lacc = nullptr;
  unsigned* lcnt = nullptr;
  // message slots by sender rank (senders: the vertices of out-degree > 0)
  int nsend = 0;
  int* sbase = nullptr;            // ceil(n / 32): senders before every word of 32 rows
  unsigned* smask = nullptr;       // ceil(n / 32): the word's senders, one bit per row
  // the build's work arrays, kept between builds: a rebuild after an update
  // allocates and frees nothing (cudaFree would wait for the whole device,
  // including another stream's upload)
  int* t_indeg = nullptr;
  int* t_first = nullptr;
  int4* t_sums = nullptr;
  size_t crp_cap = 0, csrc_cap = 0, crow_cap = 0, lbits_cap = 0, large_cap = 0, lrow_cap = 0,
         sbase_cap = 0, smask_cap = 0, lacc_cap = 0, lcnt_cap = 0, t_indeg_cap = 0, t_first_cap = 0,
         t_sums_cap = 0;
};
}

struct maiter_graph {
  int device = 0;
  int64_t n = 0, m = 0;
  int* rp = nullptr;           // n + 1 int32 offsets
  int* col = nullptr;          // m targets
  uint32_t* w = nullptr;       // m weights or null
  uint2* cw = nullptr;         // weighted graphs: (target, weight) per edge, one 8-byte load
  uint2* lstat = nullptr;      // graph-static scorer features (computed on first use)
  int wf32 = 0;                // w read as float: 0 unchecked, 1 finite and >= 0, 2 not
  int64_t* rp64 = nullptr;     // staging of the int64 offsets (kept after the first update)
  unsigned* flag = nullptr;    // validation flags (kept after the first update)
  bool invalid = false;        // the last update failed validation: no runs
  int num_sms = 0;
  maiter::BinLayout* bins = nullptr;   // binned engine layout (built on first use)
  maiter::PullLayout* pull = nullptr;  // receive-side layout of the scalar round (built on first use)
  maiter::PullLayout* pullv = nullptr; // receive-side layout of the 64-query vector round
};

struct maiter_result {
  const maiter_graph* g = nullptr;   // identity check only: a result may outlive its graph
  int device = 0;
  int op = -1;
  int64_t n = 0;
  void* v = nullptr;           // n x V
  void* delta = nullptr;       // n x D
  void* delta_wide = nullptr;  // n x double: FP64 deltas of the mixed run's warm-up phase
  void* coef = nullptr;        // n x C (allocated on first use)
  double* ecoef = nullptr;     // m per-edge coefficients (SCALE_BY_EDGE, on first use)
  int* list[2] = {nullptr, nullptr};   // small / medium frontier (n entries each)
  int2* large = nullptr;               // large-vertex chunk entries
  void* large_d = nullptr;             // their taken deltas (8 bytes per entry)
  unsigned large_cap = 0;              // n + m / kChunk + 1 entries
  maiter::DevCtl* ctl = nullptr;
  maiter::TopqCtl* topq = nullptr;     // top-fraction selection (allocated on first use)
  unsigned* last_act = nullptr;        // learned scheduling / traces: last update round
  maiter::DevCtl* h_ctl = nullptr;   // pinned mirror
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // cached executable graph of the round loop
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t exec_key = 0;
  // asynchronous engine (allocated on its first use)
  maiter::AsyncCtl* actl = nullptr;
  maiter::AsyncCtl* h_actl = nullptr;  // pinned mirror
  cudaGraph_t agraph = nullptr;
  cudaGraphExec_t aexec = nullptr;
  uint64_t aexec_key = 0;
  // binned engine (allocated on its first use)
  void* bin_msg_v = nullptr;           // n messages c_j Delta_j (8 bytes each)
  void* bin_cmsg = nullptr;            // n coefficients c_j (8 bytes each)
  void* bin_msg_e = nullptr;           // one message per padded edge slot (8 bytes each)
  size_t bin_msg_e_cap = 0;
  void* pull_msg = nullptr;            // receive-side engine: the second message buffer (n x 8 bytes)
  maiter_stats stats{};
};

namespace maiter {
// A result with its state, frontier lists and control block for op on g.
maiter_status alloc_result(const maiter_graph* g, int op, maiter_result** out);
// The learned scorer's BF16 weights on the device, and its device (mlp.cu).
const MlpWeights* mlp_device_weights(const maiter_mlp* m);
int mlp_device(const maiter_mlp* m);
// Persistent asynchronous engine (async_engine.cu); v and Delta are initialised.
maiter_status run_async(const maiter_graph* g, const maiter_run_params* p, maiter_result* r,
                        cudaStream_t st);
void free_async(maiter_result* r);
// Binned engine (binned_engine.cu): dense rounds of + with messages summed per
// receiver bin in shared memory; v and Delta are initialised.
maiter_status run_binned(const maiter_graph* g, const maiter_run_params* p, maiter_result* r,
                         cudaStream_t st);
void free_bins(maiter_graph* g);
void invalidate_bins(maiter_graph* g);
// Receive-side engine (pull_engine.cu): dense rounds of + summed at the
// receivers over the transpose; v and Delta are initialised.
maiter_status run_pull(const maiter_graph* g, const maiter_run_params* p, maiter_result* r,
                       cudaStream_t st);
void free_pull(maiter_graph* g);
void invalidate_pull(maiter_graph* g);
// Builds (or rebuilds after an update) the transpose of g on stream st: the
// scalar round's layout (g->pull), or the vector round's (g->pullv, vec).
maiter_status ensure_pull(const maiter_graph* g, cudaStream_t st, bool vec = false);
}  // namespace maiter
