// maiter_sssp_noalloc: SSSP in DAIC form for callers that cannot allocate
// device memory.
//
// Who needs it: code that runs inside a host process whose device memory is
// owned by someone else - a plugin handed pre-allocated buffers by a framework
// with its own caching allocator (a cudaMalloc behind that allocator's back
// can fail or fragment its pool), or an embedded caller with a fixed memory
// budget.  Such callers can pass their graph and output buffers, but they
// cannot let the library call cudaMalloc for its working memory.
//
// How: the same round kernels as maiter_run (k_scan / k_push for the min
// operator), with their working memory - the two frontier lists and the
// control block - carved out of one file-scope device array of fixed size.
// Every GPU that loads this library holds that array until the process exits.
// The round loop is driven from the host, one short device-to-host read of the
// control word per round (no CUDA graph, no event, no pinned buffer).
#include <cstring>
#include <mutex>

#include "internal.h"

namespace maiter {
namespace {

constexpr int64_t kNoallocMaxN = int64_t(1) << 20;   // vertices
constexpr size_t kCtlBytes = 512;
constexpr int kNoallocLists = 2;   // small and medium lists (no chunked large-vertex list)
constexpr size_t kScratchBytes = kCtlBytes + sizeof(int) * kNoallocLists * size_t(kNoallocMaxN);
// slot layout: [DevCtl | ... | validation flag (last 4 bytes)]
static_assert(sizeof(DevCtl) + sizeof(unsigned) <= kCtlBytes, "control block must fit its slot");

// The working memory: control block, then the two frontier lists.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set up once per
// device).  In host code the symbol is only a host-side stand-in; the device
// address must come from cudaGetSymbolAddress.
maiter_status scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress(g_noalloc_scratch) failed on device %d: %s", device,
                cudaGetErrorString(e));
      return MAITER_ERR_CUDA;
    }
    g_scratch_ptr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[device]);
  return MAITER_OK;
}

// The device a caller buffer lives on: -1 when it is not device (or managed)
// memory.
int pointer_device(const void* p) {
  if (!p) return -1;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return -1;
  return at.device;
}

// Checks the CSR before any push reads through it.  flag bit 0: row offsets
// not starting at 0, decreasing, or not ending at m; bit 1: a target outside
// [0, n).  The flag word is cleared by the host before this kernel runs.
__global__ void k_noalloc_check(const int* __restrict__ rp, const int* __restrict__ col,
                                int64_t m, int64_t n, unsigned* flag) {
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = tid; i <= n; i += stride) {
    const int x = rp[i];
    bool bad = x < 0 || static_cast<int64_t>(x) > m;
    if (i == 0) bad |= (x != 0);
    if (i == n) bad |= (static_cast<int64_t>(x) != m);
    if (i < n) bad |= (rp[i + 1] < x);
    if (bad) atomicOr(flag, 1u);
  }
  for (int64_t e = tid; e < m; e += stride) {
    const int k = col[e];
    if (k < 0 || k >= n) atomicOr(flag, 2u);
  }
}

// Resets the control block (the array keeps the previous call's contents) and
// sets v = inf, Delta = inf except Delta[source] = 0 (Table 1, SSSP row).
__global__ void k_noalloc_init(DevCtl* ctl, DevCtl init, int64_t n, int64_t source,
                               uint32_t* __restrict__ v, uint32_t* __restrict__ delta) {
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  if (tid == 0) *ctl = init;
  for (int64_t i = tid; i < n; i += stride) {
    v[i] = kInfU32;
    delta[i] = (i == source) ? 0u : kInfU32;
  }
}

}  // namespace
}  // namespace maiter

using namespace maiter;

extern "C" maiter_status maiter_sssp_noalloc(int64_t n, int64_t m, const int32_t* row_ptr,
                                             const int32_t* col, const uint32_t* w,
                                             int64_t source, uint32_t* v_out,
                                             uint32_t* delta_out, int64_t max_rounds,
                                             int device, void* stream, int64_t* rounds_out) {
  set_error("%s", "");
  cudaGetLastError();
  MAITER_REQUIRE(n >= 1 && n <= kNoallocMaxN,
                 "maiter_sssp_noalloc: n = %lld outside [1, %lld] (the fixed working "
                 "memory holds at most %lld vertices)",
                 (long long)n, (long long)kNoallocMaxN, (long long)kNoallocMaxN);
  MAITER_REQUIRE(m >= 0 && m < (int64_t(1) << 31), "m = %lld out of range [0, 2^31)",
                 (long long)m);
  MAITER_REQUIRE(source >= 0 && source < n, "source %lld outside [0, n)", (long long)source);
  MAITER_REQUIRE(row_ptr && v_out && delta_out && (m == 0 || (col && w)),
                 "NULL buffer");
  MAITER_REQUIRE(device >= 0 && device < kMaxDevices, "device %d out of range", device);
  {
    // Every buffer must be device memory of `device`: a buffer of another GPU
    // would be read (and atomically written) across the interconnect, or fault.
    const void* bufs[5] = {row_ptr, v_out, delta_out, col, w};
    const char* names[5] = {"row_ptr", "v_out", "delta_out", "col", "w"};
    for (int i = 0; i < (m == 0 ? 3 : 5); ++i) {
      const int d = pointer_device(bufs[i]);
      MAITER_REQUIRE(d >= 0, "maiter_sssp_noalloc takes device pointers only (%s is not)",
                     names[i]);
      MAITER_REQUIRE(d == device, "maiter_sssp_noalloc: %s lives on device %d, not on device %d",
                     names[i], d, device);
    }
  }
  DeviceGuard guard(device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    // The round loop waits on the host after every round, which a capturing
    // stream cannot do (and the attempt would invalidate the caller's capture).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) cudaGetLastError();
    MAITER_REQUIRE(e == cudaSuccess && cs == cudaStreamCaptureStatusNone,
                   "maiter_sssp_noalloc: the stream is capturing (or the default stream "
                   "while another stream captures); the call synchronises with the host "
                   "every round, so it needs a stream that is not capturing");
  }

  unsigned char* scratch = nullptr;
  maiter_status s = scratch_address(device, &scratch);
  if (s != MAITER_OK) return s;
  DevCtl* ctl = reinterpret_cast<DevCtl*>(scratch);
  unsigned* flag = reinterpret_cast<unsigned*>(scratch + kCtlBytes - sizeof(unsigned));
  int* lists = reinterpret_cast<int*>(scratch + kCtlBytes);

  int num_sms = 0;
  MAITER_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
  constexpr int kBlock = 256;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, reinterpret_cast<const void*>(&k_push<OpMinU32, kBlock>), kBlock, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int push_grid = num_sms * per_sm;
  int scan_grid = num_sms * 4;
  const int need = static_cast<int>((n + kBlock - 1) / kBlock);
  if (need < scan_grid) scan_grid = need;

  MAITER_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
  k_noalloc_check<<<num_sms * 4, 256, 0, st>>>(row_ptr, col, m, n, flag);
  MAITER_CUDA(cudaGetLastError());
  unsigned h_flag = 0;
  MAITER_CUDA(cudaMemcpyAsync(&h_flag, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  MAITER_CUDA(cudaStreamSynchronize(st));
  if (h_flag & 1u) {
    set_error("row_ptr must start at 0, be non-decreasing and end at m = %lld", (long long)m);
    return MAITER_ERR_INVALID_ARG;
  }
  if (h_flag & 2u) {
    set_error("col holds a target outside [0, n = %lld)", (long long)n);
    return MAITER_ERR_INVALID_ARG;
  }

  DevCtl init{};
  init.max_rounds = max_rounds > 0 ? max_rounds : 1000000;
  k_noalloc_init<<<num_sms * 4, 256, 0, st>>>(ctl, init, n, source, v_out, delta_out);
  MAITER_CUDA(cudaGetLastError());

  KArgs<OpMinU32> a{};
  a.n = static_cast<int>(n);
  a.rp = row_ptr;
  a.edges.col = col;
  a.edges.w = w;
  a.coef = nullptr;
  a.damping = 0.0;
  a.v = v_out;
  a.delta = delta_out;
  for (int b = 0; b < 2; ++b) a.list[b] = lists + size_t(b) * kNoallocMaxN;
  // No chunked large-vertex path here: its entry count grows with m, which a
  // fixed array cannot bound, so every vertex of degree >= 32 takes the warp path.
  a.large = nullptr;
  a.large_d = nullptr;
  a.large_cap = 0;
  a.ctl = ctl;
  a.cut_warp = 32;
  a.cut_cta = 1 << 30;

  DevCtl h{};
  for (;;) {
    k_scan<OpMinU32, kBlock><<<scan_grid, kBlock, 0, st>>>(a);
    k_push<OpMinU32, kBlock><<<push_grid, kBlock, 0, st>>>(a, cudaGraphConditionalHandle{}, 0);
    MAITER_CUDA(cudaGetLastError());
    MAITER_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
    MAITER_CUDA(cudaStreamSynchronize(st));
    if (h.status != 0) break;
  }
  if (rounds_out) *rounds_out = static_cast<int64_t>(h.rounds);
  if (h.status != 1) {
    set_error("round cap of %lld reached before every distance was final",
              (long long)init.max_rounds);
    return MAITER_ERR_NOT_CONVERGED;
  }
  return MAITER_OK;
}
