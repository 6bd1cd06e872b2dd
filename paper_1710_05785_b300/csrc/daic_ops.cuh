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

// u32 -> f32 without an I2F (B300 issues conversions on its narrow FP64
// pipe), rounded to nearest like the conversion: each 16-bit half is exact
// as (2^23 + half) - 2^23, and one fma joins them with a single rounding.
__device__ __forceinline__ float u32_to_f32(unsigned x) {
  const float hi = __uint_as_float(0x4B000000u | (x >> 16)) - 8388608.0f;
  const float lo = __uint_as_float(0x4B000000u | (x & 0xFFFFu)) - 8388608.0f;
  return fmaf(hi, 65536.0f, lo);
}

constexpr uint32_t kInfU32 = 0xFFFFFFFFu;

// Vertex-update context shared by all operators.
struct EdgeCtx {
  const int* __restrict__ col;
  const uint32_t* __restrict__ w;
  const double* __restrict__ ecoef;   // per-edge coefficients (g = c_e x), or null
  const uint2* __restrict__ cw;       // weighted graphs: (target, weight) pairs
};

__device__ __forceinline__ double atomic_take(double* p) {
  unsigned long long bits = atomicExch(reinterpret_cast<unsigned long long*>(p), 0ull);
  return __longlong_as_double(static_cast<long long>(bits));
}
__device__ __forceinline__ float atomic_take(float* p) { return atomicExch(p, 0.0f); }

// ------------------------------------------------------------------ + (sum)
// State v in FP64; delta in DT (double or float); coefficients in CT.  The
// message c_j * Delta_j is an FP32 product when both are FP32, else formed in
// FP64 and rounded once to DT.
template <class DT, class CT>
struct OpSum {
  using V = double;
  using D = DT;
  using C = CT;
  using Msg = DT;
  static constexpr bool kIsSum = true;
  static constexpr DT kNone = DT(0);   // "nothing pending"

  // Pending-priority |v_j (+) Delta_j - v_j| = |Delta_j| (Section 3.5).
  __device__ static __forceinline__ double priority(D d, V) { return fabs(static_cast<double>(d)); }
  __device__ static __forceinline__ bool pending(D d, V) { return d != D(0); }

  // Read-and-reset Delta_j atomically so a message that lands between the
  // read and the reset cannot be lost; fold it into v_j.  The update of a
  // vertex is owned by one thread per round, so v_j needs no atomic.
  __device__ static __forceinline__ Msg fold(int j, int deg, D* delta, V* v, const C* coef,
                                             double damping) {
    const D d = atomic_take(delta + j);
    if (d == D(0)) return D(0);
    // v is read and written once a round: streamed (evict-first), so it does
    // not push the Delta lines the pushes' atomics need out of L2
    __stcs(v + j, __ldcs(v + j) + static_cast<double>(d));
    if (deg == 0) return D(0);
    return message(j, deg, d, coef, damping);
  }
  // c_j Delta_j: in FP32 when delta and coefficient are FP32, else formed in
  // FP64 and rounded once to D.
  __device__ static __forceinline__ Msg message(int j, int deg, D d, const C* coef,
                                                double damping) {
    if constexpr (sizeof(D) == 4 && sizeof(C) == 4) {
      if (coef) return coef[j] * d;
    }
    const double c = coef ? static_cast<double>(coef[j]) : damping / static_cast<double>(deg);
    return static_cast<D>(c * static_cast<double>(d));
  }
  // Large vertices are split into chunks processed by different CTAs, so
  // their delta is taken in the frontier scan (atomic exchange, exact) and
  // the state update happens once, by the CTA of chunk 0.
  __device__ static __forceinline__ D take(int j, D* delta, const V*) {
    return atomic_take(delta + j);
  }
  __device__ static __forceinline__ void untake(int j, D d, D* delta) {
    if (d != D(0)) atomicAdd(delta + j, d);
  }
  __device__ static __forceinline__ Msg finish(int j, int deg, D d, V* v, const C* coef,
                                               double damping, bool first_chunk) {
    if (d == D(0)) return D(0);
    if (first_chunk) __stcs(v + j, __ldcs(v + j) + static_cast<double>(d));
    if (deg == 0) return D(0);
    return message(j, deg, d, coef, damping);
  }

  __device__ static __forceinline__ bool live(Msg m) { return m != Msg(0); }
  struct Edge { int k; };
  __device__ static __forceinline__ Edge load(const EdgeCtx& g, int64_t e) {
    return Edge{__ldcs(g.col + e)};
  }
  __device__ static __forceinline__ void apply(Edge ed, Msg m, D* delta) {
    atomicAdd(delta + ed.k, m);
  }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    apply(load(g, e), m, delta);
  }
};

// + with a coefficient per edge, g_{j,k}(x) = c_{jk} x, all FP64: the Jacobi
// method's -A_kj / A_kk (Section 4.3) and any other linear update whose weights
// depend on the receiver.  A vertex's message is Delta_j itself; each edge
// scales it.  Coefficients may be negative, so Delta is signed and the
// priority and the residual use |Delta|.
struct OpSumEdge {
  using V = double;
  using D = double;
  using C = double;
  using Msg = double;
  static constexpr bool kIsSum = true;
  static constexpr double kNone = 0.0;

  __device__ static __forceinline__ double priority(D d, V) { return fabs(d); }
  __device__ static __forceinline__ bool pending(D d, V) { return d != 0.0; }
  __device__ static __forceinline__ Msg fold(int j, int deg, D* delta, V* v, const C*, double) {
    const double d = atomic_take(delta + j);
    if (d == 0.0) return 0.0;
    v[j] += d;
    return deg == 0 ? 0.0 : d;
  }
  __device__ static __forceinline__ D take(int j, D* delta, const V*) { return atomic_take(delta + j); }
  __device__ static __forceinline__ void untake(int j, D d, D* delta) {
    if (d != 0.0) atomicAdd(delta + j, d);
  }
  __device__ static __forceinline__ Msg finish(int j, int deg, D d, V* v, const C*, double,
                                               bool first_chunk) {
    if (d == 0.0) return 0.0;
    if (first_chunk) v[j] += d;
    return deg == 0 ? 0.0 : d;
  }
  __device__ static __forceinline__ bool live(Msg m) { return m != 0.0; }
  struct Edge { int k; double c; };
  __device__ static __forceinline__ Edge load(const EdgeCtx& g, int64_t e) {
    return Edge{__ldg(g.col + e), __ldg(g.ecoef + e)};
  }
  __device__ static __forceinline__ void apply(Edge ed, Msg m, D* delta) {
    const double x = ed.c * m;
    if (x != 0.0) atomicAdd(delta + ed.k, x);
  }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    apply(load(g, e), m, delta);
  }
};

using OpSumF64 = OpSum<double, double>;     // all FP64
using OpSumWarm = OpSum<double, float>;     // mixed precision, FP64-delta phase
using OpSumMixed = OpSum<float, float>;     // mixed precision, FP32-delta phase

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
  static constexpr bool kIsMax = false;
  static constexpr uint32_t kNone = kInfU32;   // infinity: identity of min, nothing pending
  __device__ static __forceinline__ double value(uint32_t x) { return static_cast<double>(x); }
  __device__ static __forceinline__ float fvalue(uint32_t x) { return u32_to_f32(x); }

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
  // Large vertices: the scan only records Delta_j (nothing to undo); chunk
  // 0's CTA folds it into v_j.
  __device__ static __forceinline__ D take(int j, D* delta, const V*) { return __ldcg(delta + j); }
  __device__ static __forceinline__ void untake(int, D, D*) {}
  __device__ static __forceinline__ Msg finish(int j, int, D d, V* v, const C*, double,
                                               bool first_chunk) {
    if (first_chunk && d < v[j]) v[j] = d;
    return d;
  }

  __device__ static __forceinline__ bool live(Msg m) { return m != kInfU32; }
  struct Edge { int k; uint32_t w; };
  __device__ static __forceinline__ Edge load(const EdgeCtx& g, int64_t e) {
    if (g.cw) {
      const uint2 x = __ldcs(g.cw + e);   // streamed: leave L1 to the filter reads
      return Edge{static_cast<int>(x.x), x.y};
    }
    return Edge{__ldg(g.col + e), __ldg(g.w + e)};   // caller-owned arrays (no pairs)
  }
  __device__ static __forceinline__ void apply(Edge ed, Msg m, D* delta) {
    const uint32_t s = m + ed.w;
    const uint32_t nd = (s < m) ? kInfU32 : s;  // saturate: an overflowing message is infinity
    // The filter read may come from L1: Delta only decreases, so a stale
    // value is larger and the test can only let an extra atomic through.
    if (nd < __ldca(delta + ed.k)) atomicMin(delta + ed.k, nd);
  }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    apply(load(g, e), m, delta);
  }
};

// ------------------------------------------- min over float32 (SSSP, FP32)
// The same operator on non-negative IEEE single distances and weights (the
// float weights of the paper's synthetic SSSP graphs, Section 6.1).  v and
// Delta hold the bit patterns: for non-negative floats the unsigned order of
// the bits is the order of the values, so the unsigned atomicMin is the float
// min and every pending test is a bit comparison.  Infinity is +inf
// (0x7F800000); a message is fl(Delta_j + w_jk) with IEEE round-to-nearest,
// and an overflowing sum is +inf, i.e. no message.  Rounded addition is
// monotone, so the fixed point is, for every vertex, the least over paths of
// the path's sum accumulated from the source in this rounding.
struct OpMinF32 {
  using V = uint32_t;
  using D = uint32_t;
  using C = float;  // unused
  using Msg = uint32_t;
  static constexpr bool kIsSum = false;
  static constexpr bool kIsMax = false;
  static constexpr uint32_t kNone = 0x7F800000u;   // +inf
  __device__ static __forceinline__ double value(uint32_t x) {
    return static_cast<double>(__uint_as_float(x));
  }
  __device__ static __forceinline__ float fvalue(uint32_t x) { return __uint_as_float(x); }

  __device__ static __forceinline__ double priority(D d, V v) {
    return d < v ? value(v) - value(d) : 0.0;
  }
  __device__ static __forceinline__ bool pending(D d, V v) { return d < v; }

  __device__ static __forceinline__ Msg fold(int j, int, D* delta, V* v, const C*, double) {
    const uint32_t d = __ldcg(delta + j);
    const uint32_t cur = v[j];
    if (d >= cur) return kNone;
    v[j] = d;
    return d;
  }
  __device__ static __forceinline__ D take(int j, D* delta, const V*) { return __ldcg(delta + j); }
  __device__ static __forceinline__ void untake(int, D, D*) {}
  __device__ static __forceinline__ Msg finish(int j, int, D d, V* v, const C*, double,
                                               bool first_chunk) {
    if (first_chunk && d < v[j]) v[j] = d;
    return d;
  }

  __device__ static __forceinline__ bool live(Msg m) { return m != kNone; }
  struct Edge { int k; uint32_t w; };
  __device__ static __forceinline__ Edge load(const EdgeCtx& g, int64_t e) {
    if (g.cw) {
      const uint2 x = __ldcs(g.cw + e);   // streamed: leave L1 to the filter reads
      return Edge{static_cast<int>(x.x), x.y};
    }
    return Edge{__ldg(g.col + e), __ldg(g.w + e)};   // caller-owned arrays (no pairs)
  }
  __device__ static __forceinline__ void apply(Edge ed, Msg m, D* delta) {
    const uint32_t nd = __float_as_uint(__fadd_rn(__uint_as_float(m), __uint_as_float(ed.w)));
    // The filter read may come from L1: Delta only decreases, so a stale
    // value is larger and the test can only let an extra atomic through.
    if (nd < __ldca(delta + ed.k)) atomicMin(delta + ed.k, nd);
  }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    apply(load(g, e), m, delta);
  }
};

// ------------------------------------------- max over int32 (components)
// Connected components (Table 1): (+) = max, g_{i,j}(x) = x, v^0 = -1,
// Delta^1_j = j; every vertex ends with the largest id among the vertices
// that reach it (on a symmetric graph, the largest id of its component).
// Idempotent like min: Delta is kept, only ever grows, and j is pending iff
// Delta_j > v_j.
struct OpMaxI32 {
  using V = int32_t;
  using D = int32_t;
  using C = float;  // unused
  using Msg = int32_t;
  static constexpr bool kIsSum = false;
  static constexpr bool kIsMax = true;
  static constexpr int32_t kNone = -1;   // identity of max over labels >= 0
  __device__ static __forceinline__ double value(int32_t x) { return static_cast<double>(x); }
  __device__ static __forceinline__ float fvalue(int32_t x) { return static_cast<float>(x); }

  __device__ static __forceinline__ double priority(D d, V v) {
    return d > v ? static_cast<double>(d) - static_cast<double>(v) : 0.0;
  }
  __device__ static __forceinline__ bool pending(D d, V v) { return d > v; }

  __device__ static __forceinline__ Msg fold(int j, int, D* delta, V* v, const C*, double) {
    const int32_t d = __ldcg(delta + j);
    const int32_t cur = v[j];
    if (d <= cur) return kNone;
    v[j] = d;
    return d;
  }
  __device__ static __forceinline__ D take(int j, D* delta, const V*) { return __ldcg(delta + j); }
  __device__ static __forceinline__ void untake(int, D, D*) {}
  __device__ static __forceinline__ Msg finish(int j, int, D d, V* v, const C*, double,
                                               bool first_chunk) {
    if (first_chunk && d > v[j]) v[j] = d;
    return d;
  }

  __device__ static __forceinline__ bool live(Msg m) { return m != kNone; }
  struct Edge { int k; };
  __device__ static __forceinline__ Edge load(const EdgeCtx& g, int64_t e) {
    return Edge{__ldg(g.col + e)};
  }
  __device__ static __forceinline__ void apply(Edge ed, Msg m, D* delta) {
    if (m > __ldcg(delta + ed.k)) atomicMax(delta + ed.k, m);
  }
  __device__ static __forceinline__ void scatter(const EdgeCtx& g, int64_t e, Msg m, D* delta) {
    apply(load(g, e), m, delta);
  }
};

}  // namespace maiter
