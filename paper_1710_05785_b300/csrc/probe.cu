// Random-access ceilings of the device: how many 4- or 8-byte operations per
// second the memory system sustains at addresses with no locality.  The push
// kernels issue exactly such operations (one filter read and/or one atomic
// on Delta_k per edge, k a random vertex id), so these rates, measured on
// the array size of a workload's Delta, bound the push more tightly than the
// DRAM copy bandwidth does.  Diagnostic only: nothing in a run calls it.
#include "internal.h"

namespace maiter {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbeIters = 256;   // operations per thread per launch

// A 32-bit integer hash (xor-shift-multiply, constants of the "lowbias32"
// finaliser) spreads consecutive (thread, iteration) pairs over the array.
__device__ __forceinline__ unsigned probe_hash(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Every address is hash & mask with mask = words - 1 (words a power of two),
// so all accesses stay inside the array.
template <int KIND>
__global__ void __launch_bounds__(kProbeBlock) k_probe(void* buf, float* sink, unsigned mask,
                                                       unsigned seed) {
  const unsigned tid = blockIdx.x * kProbeBlock + threadIdx.x;
  float acc = 0.f;
  for (int i = 0; i < kProbeIters; ++i) {
    const unsigned h =
        probe_hash(tid * 0x9E3779B9u + static_cast<unsigned>(i) * 0x85EBCA6Bu + seed) & mask;
    if constexpr (KIND == MAITER_PROBE_RED_F32) atomicAdd(static_cast<float*>(buf) + h, 1.0f);
    else if constexpr (KIND == MAITER_PROBE_RED_F64) atomicAdd(static_cast<double*>(buf) + h, 1.0);
    else if constexpr (KIND == MAITER_PROBE_MIN_U32) atomicMin(static_cast<unsigned*>(buf) + h, tid);
    else acc += __ldcg(static_cast<const float*>(buf) + h);
  }
  if constexpr (KIND == MAITER_PROBE_LOAD_32) sink[tid] = acc;   // keeps the loads
}

template <int KIND>
void launch_probe(int grid, cudaStream_t st, void* buf, float* sink, unsigned mask, unsigned seed) {
  k_probe<KIND><<<grid, kProbeBlock, 0, st>>>(buf, sink, mask, seed);
}

}  // namespace
}  // namespace maiter

using namespace maiter;

extern "C" maiter_status maiter_probe_random_rate(int device, int kind, int log2_words,
                                                  double* gops) {
  set_error("%s", "");
  cudaGetLastError();   // a stale non-sticky error must not fail this call's checks
  MAITER_REQUIRE(gops, "NULL argument");
  MAITER_REQUIRE(kind >= MAITER_PROBE_RED_F32 && kind <= MAITER_PROBE_LOAD_32,
                 "unknown probe kind %d", kind);
  MAITER_REQUIRE(log2_words >= 10 && log2_words <= 28, "log2_words %d outside [10, 28]",
                 log2_words);
  int ndev = 0;
  MAITER_CUDA(cudaGetDeviceCount(&ndev));
  MAITER_REQUIRE(device >= 0 && device < ndev, "device %d out of range", device);
  DeviceGuard guard(device);
  cudaDeviceProp prop{};
  MAITER_CUDA(cudaGetDeviceProperties(&prop, device));
  void (*launch)(int, cudaStream_t, void*, float*, unsigned, unsigned) = nullptr;
  const void* fn = nullptr;
  switch (kind) {
    case MAITER_PROBE_RED_F32:
      launch = &launch_probe<MAITER_PROBE_RED_F32>;
      fn = reinterpret_cast<const void*>(&k_probe<MAITER_PROBE_RED_F32>);
      break;
    case MAITER_PROBE_RED_F64:
      launch = &launch_probe<MAITER_PROBE_RED_F64>;
      fn = reinterpret_cast<const void*>(&k_probe<MAITER_PROBE_RED_F64>);
      break;
    case MAITER_PROBE_MIN_U32:
      launch = &launch_probe<MAITER_PROBE_MIN_U32>;
      fn = reinterpret_cast<const void*>(&k_probe<MAITER_PROBE_MIN_U32>);
      break;
    default:
      launch = &launch_probe<MAITER_PROBE_LOAD_32>;
      fn = reinterpret_cast<const void*>(&k_probe<MAITER_PROBE_LOAD_32>);
      break;
  }
  int per_sm = 0;
  MAITER_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProbeBlock, 0));
  const int grid = prop.multiProcessorCount * (per_sm > 0 ? per_sm : 1);
  const size_t words = size_t(1) << log2_words;
  const size_t elem = kind == MAITER_PROBE_RED_F64 ? 8 : 4;
  void* buf = nullptr;
  float* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  maiter_status rc = MAITER_OK;
  auto check = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == MAITER_OK) {
      set_error("%s failed: %s", what, cudaGetErrorString(e));
      rc = e == cudaErrorMemoryAllocation ? MAITER_ERR_OOM : MAITER_ERR_CUDA;
    }
    return rc == MAITER_OK;
  };
  float best = 0.f;
  if (check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate") &&
      check(cudaEventCreate(&e0), "cudaEventCreate") &&
      check(cudaEventCreate(&e1), "cudaEventCreate") &&
      check(cudaMalloc(&buf, words * elem), "cudaMalloc") &&
      check(cudaMalloc(&sink, sizeof(float) * size_t(grid) * kProbeBlock), "cudaMalloc") &&
      check(cudaMemsetAsync(buf, kind == MAITER_PROBE_MIN_U32 ? 0xff : 0, words * elem, st),
            "cudaMemsetAsync")) {
    const unsigned mask = static_cast<unsigned>(words - 1);
    // one warm-up launch, then the best of three
    for (int rep = 0; rep < 4 && rc == MAITER_OK; ++rep) {
      check(cudaEventRecord(e0, st), "cudaEventRecord");
      launch(grid, st, buf, sink, mask, static_cast<unsigned>(rep));
      check(cudaGetLastError(), "probe launch");
      check(cudaEventRecord(e1, st), "cudaEventRecord");
      if (check(cudaEventSynchronize(e1), "cudaEventSynchronize") && rep > 0) {
        float ms = 0.f;
        if (check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime") && ms > 0.f &&
            (best == 0.f || ms < best))
          best = ms;
      }
    }
  }
  if (st) cudaStreamSynchronize(st);
  cudaFree(sink);
  cudaFree(buf);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (rc != MAITER_OK) return rc;
  const double ops = double(grid) * kProbeBlock * kProbeIters;
  *gops = best > 0.f ? ops / (double(best) * 1e-3) / 1e9 : 0.0;
  return MAITER_OK;
}
