// Accumulation operators of delta-based accumulative iterative computation
// (DAIC) and the per-vertex update of the asynchronous DAIC (Eq. 5).
//
// An operator type bundles:
//   V      - type of the state v_j,
//   D      - type of the delta Delta_j (what the scatter atomics act on),
//   C      - type of the per-source coefficient of g_{j,k}(x) = c_j * x,
//   Msg    - what one activated vertex hands to each of its out-edges,
//   fold() - v_j <- v_j (+) Delta_j; Delta_j <- 0 (the identity), returning
//            the message basis,
//   scatter() - Delta_k <- Delta_k (+) g_{j,k}(Delta_j) for one edge.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace maiter {

constexpr uint32_t kInfU32 = 0xFFFFFFFFu;

// Vertex-update context shared by all operators.
struct EdgeCtx {
  const int* __restrict__ col;
  const uint32_t* __restrict__ w;
};

// ------------------------------------------------------------------ + FP64
struct OpSumF64 {
  using V = double;
  using D = double;
  using C = double;
  using Msg = double;
  static constexpr bool kIsSum = true;

  // Pending-priority |v_j (+) Delta_j - v_j| = |Delta_j| (Section 3.5).
  __device__ static __forceinline__ double priority(D d, V) { return fabs(d); }
  __device__ static __forceinline__ bool pending(D d, V) { return d != 0.0; }

  // Read-and-reset Delta_j atomically so a message that lands between the
  // read and the reset cannot be lost; fold it into v_j.  The update of a
  // vertex is owned by one thread per round, so v_j needs no atomic.
  __device__ static __forceinline__ Msg fold(int j, int deg, D* delta, V* v, const C* coef,
                                             double damping) {
    unsigned long long bits =
        atomicExch(reinterpret_cast<unsigned long long*>(delta + j), 0ull);
    double d = __longlong_as_double(static_cast<long long>(bits));
    if (d == 0.0) return 0.0;
    v[j] += d;
    if (deg == 0) return 0.0;
    double c = coef ? coef[j] : damping / static_cast<double>(deg);
    return c * d;
  }
  __device__ static __forceinline__ bool live(Msg m) { return m != 0.0; }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    int k = __ldcs(g.col + e);
    atomicAdd(delta + k, m);
  }
};

// ------------------------------------------ + with FP32 deltas, FP64 state
struct OpSumMixed {
  using V = double;
  using D = float;
  using C = float;
  using Msg = float;
  static constexpr bool kIsSum = true;

  __device__ static __forceinline__ double priority(D d, V) { return fabs(static_cast<double>(d)); }
  __device__ static __forceinline__ bool pending(D d, V) { return d != 0.0f; }

  __device__ static __forceinline__ Msg fold(int j, int deg, D* delta, V* v, const C* coef,
                                             double damping) {
    float d = atomicExch(delta + j, 0.0f);
    if (d == 0.0f) return 0.0f;
    v[j] += static_cast<double>(d);
    if (deg == 0) return 0.0f;
    double c = coef ? static_cast<double>(coef[j]) : damping / static_cast<double>(deg);
    return static_cast<float>(c * static_cast<double>(d));
  }
  __device__ static __forceinline__ bool live(Msg m) { return m != 0.0f; }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    int k = __ldcs(g.col + e);
    atomicAdd(delta + k, m);
  }
};

// ------------------------------------------------ min over uint32 (SSSP)
// g_{j,k}(x) = x + w_jk, saturating at infinity (Table 1, SSSP row).
//
// min is idempotent (x min x = x), so folding the same delta twice changes
// nothing.  The update therefore keeps Delta_j instead of resetting it to
// infinity: Delta then only ever decreases, the pending test stays
// Delta_j < v_j (priority v_j - min(v_j, Delta_j) > 0 of the SSSP subsection),
// and the read of Delta_j needs no atomic exchange.
struct OpMinU32 {
  using V = uint32_t;
  using D = uint32_t;
  using C = float;  // unused
  using Msg = uint32_t;
  static constexpr bool kIsSum = false;

  __device__ static __forceinline__ double priority(D d, V v) {
    return d < v ? static_cast<double>(v - d) : 0.0;
  }
  __device__ static __forceinline__ bool pending(D d, V v) { return d < v; }

  __device__ static __forceinline__ Msg fold(int j, int, D* delta, V* v, const C*, double) {
    uint32_t d = __ldcg(delta + j);
    uint32_t cur = v[j];
    if (d >= cur) return kInfU32;
    v[j] = d;
    return d;
  }
  __device__ static __forceinline__ bool live(Msg m) { return m != kInfU32; }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    int k = __ldcs(g.col + e);
    uint32_t wk = __ldcs(g.w + e);
    uint32_t s = m + wk;
    uint32_t nd = (s < m) ? kInfU32 : s;  // saturate: an overflowing message is infinity
    if (nd < __ldcg(delta + k)) atomicMin(delta + k, nd);
  }
};

}  // namespace maiter
