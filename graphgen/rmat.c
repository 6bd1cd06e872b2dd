/*
 * Seeded synthetic graph inputs, shared by the CPU oracle and the CUDA path.
 *
 * This file holds no arithmetic of the delta-propagation method: it only draws
 * random edges and lays them out as a CSR.  Every random number is a pure
 * function of (seed, stream, counter), so the output does not depend on the
 * thread count or on the order in which edges are generated.
 *
 * Counter-based generator: the SplitMix64 output function (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
 * applied to  key(seed, stream) + counter * golden_gamma.
 *
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each edge picks one of the
 * four quadrants of the adjacency matrix per level with probabilities
 * (a, b, c, d), Graph500 style, without noise.  Vertex ids are then relabelled
 * by a seeded Fisher-Yates permutation, and each row's targets are sorted so
 * the CSR is canonical.  Multi-edges and self-loops are kept.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Key of one independent stream. */
uint64_t gg_stream_key(uint64_t seed, uint64_t stream) {
  return sm64_mix(sm64_mix(seed + GOLDEN) + (stream + 1) * GOLDEN);
}

/* counter-th 64-bit draw of a stream. */
uint64_t gg_draw(uint64_t key, uint64_t counter) {
  return sm64_mix(key + (counter + 1) * GOLDEN);
}

/* uniform integer in [0, bound) by Lemire's multiply-high reduction */
static inline uint64_t bounded(uint64_t r, uint64_t bound) {
  return (uint64_t)(((__uint128_t)r * (__uint128_t)bound) >> 64);
}

enum { STREAM_EDGES = 0, STREAM_PERM = 1, STREAM_WEIGHTS = 2, STREAM_SOURCES = 3,
       STREAM_LOGNORMAL = 4, STREAM_LN_DEGREE = 5, STREAM_LN_SOURCE = 6, STREAM_LN_WEIGHT = 7 };

/* Fill perm[0..n) with a seeded uniform permutation (Fisher-Yates, Durstenfeld). */
void gg_permutation(int64_t n, uint64_t seed, int32_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  uint64_t key = gg_stream_key(seed, STREAM_PERM);
  for (int64_t i = n - 1; i > 0; --i) {
    int64_t j = (int64_t)bounded(gg_draw(key, (uint64_t)i), (uint64_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
}

/*
 * R-MAT edge list: src[e], dst[e] for e in [0, m), before relabelling.
 * Probabilities are given as 32-bit thresholds: a draw u (32 bits) picks
 * quadrant 0 if u < ta, 1 if u < tab, 2 if u < tabc, else 3.
 */
void gg_rmat_edges(int scale, int64_t m, uint64_t seed, double a, double b, double c,
                   int32_t* src, int32_t* dst) {
  const double two32 = 4294967296.0;
  const uint64_t ta = (uint64_t)(a * two32);
  const uint64_t tab = (uint64_t)((a + b) * two32);
  const uint64_t tabc = (uint64_t)((a + b + c) * two32);
  const uint64_t key = gg_stream_key(seed, STREAM_EDGES);
  const int draws = (scale + 1) / 2;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    uint32_t s = 0, t = 0;
    for (int k = 0; k < draws; ++k) {
      uint64_t r = gg_draw(key, (uint64_t)e * 32u + (uint64_t)k);
      for (int h = 0; h < 2; ++h) {
        int level = 2 * k + h;
        if (level >= scale) break;
        uint64_t u = h ? (r & 0xFFFFFFFFULL) : (r >> 32);
        uint32_t q = u < ta ? 0u : (u < tab ? 1u : (u < tabc ? 2u : 3u));
        s = (s << 1) | (q >> 1);
        t = (t << 1) | (q & 1u);
      }
    }
    src[e] = (int32_t)s;
    dst[e] = (int32_t)t;
  }
}

/* Edge weights, uniform integers in [wlo, whi], one per edge index. */
void gg_uniform_weights(int64_t m, uint64_t seed, uint32_t wlo, uint32_t whi, uint32_t* w) {
  const uint64_t key = gg_stream_key(seed, STREAM_WEIGHTS);
  const uint64_t span = (uint64_t)whi - (uint64_t)wlo + 1u;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) w[e] = wlo + (uint32_t)bounded(gg_draw(key, (uint64_t)e), span);
}

static int cmp_u64(const void* x, const void* y) {
  uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
  return (a > b) - (a < b);
}

/*
 * Build a CSR from an edge list: row_ptr[n+1] (int64), col[m] (int32) and, if
 * w_in is not NULL, w_out[m].  Within a row, (target, weight) pairs are sorted
 * ascending, so the result depends only on the multiset of edges.
 * If perm is not NULL, endpoints are relabelled through it first.
 * Returns 0 on success, -1 on allocation failure.
 */
int gg_build_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                 const uint32_t* w_in, const int32_t* perm,
                 int64_t* row_ptr, int32_t* col, uint32_t* w_out) {
  int64_t* cursor = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  uint64_t* packed = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
  if (!cursor || !packed) { free(cursor); free(packed); return -1; }
  for (int64_t e = 0; e < m; ++e) {
    int32_t s = perm ? perm[src[e]] : src[e];
    cursor[s + 1]++;
  }
  for (int64_t i = 0; i < n; ++i) cursor[i + 1] += cursor[i];
  memcpy(row_ptr, cursor, (size_t)(n + 1) * sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e) {
    int32_t s = perm ? perm[src[e]] : src[e];
    int32_t t = perm ? perm[dst[e]] : dst[e];
    uint32_t wt = w_in ? w_in[e] : 0u;
    packed[cursor[s]++] = ((uint64_t)(uint32_t)t << 32) | wt;
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
    if (hi - lo > 1) qsort(packed + lo, (size_t)(hi - lo), sizeof(uint64_t), cmp_u64);
  }
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    col[e] = (int32_t)(packed[e] >> 32);
    if (w_out) w_out[e] = (uint32_t)(packed[e] & 0xFFFFFFFFULL);
  }
  free(cursor);
  free(packed);
  return 0;
}

/* k distinct draws from candidates[0..nc) (seeded, without replacement). */
int gg_pick(int64_t nc, const int32_t* candidates, int64_t k, uint64_t seed, uint64_t stream,
            int32_t* out) {
  if (k > nc) return -1;
  int32_t* tmp = (int32_t*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
  if (!tmp) return -1;
  memcpy(tmp, candidates, (size_t)nc * sizeof(int32_t));
  uint64_t key = gg_stream_key(seed, STREAM_SOURCES + 16 * stream);
  for (int64_t i = 0; i < k; ++i) {   /* partial Fisher-Yates from the front */
    int64_t j = i + (int64_t)bounded(gg_draw(key, (uint64_t)i), (uint64_t)(nc - i));
    int32_t t = tmp[i]; tmp[i] = tmp[j]; tmp[j] = t;
    out[i] = tmp[i];
  }
  free(tmp);
  return 0;
}

/* uniform doubles in [0,1) with 53 random bits */
void gg_uniform01(int64_t count, uint64_t seed, uint64_t stream, double* out) {
  uint64_t key = gg_stream_key(seed, STREAM_SOURCES + 16 * stream + 1);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i)
    out[i] = (double)(gg_draw(key, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
}

/*
 * Log-normal synthetic graphs of the paper's evaluation (Section 6.1): the
 * in-degree of every vertex is drawn from a log-normal distribution
 * LN(mu, sigma) and rounded to the nearest integer (capped at cap), and each
 * in-edge's source is a uniform vertex id (with replacement).  Edge weights,
 * when asked for, are LN(wmu, wsigma) rounded to IEEE single.
 *
 * Standard normal deviates by the Box-Muller transform (Box and Muller, Ann.
 * Math. Stat. 1958) from two 53-bit uniforms of the same counter; u1 lies in
 * (0, 1] so its logarithm is finite.
 */
static inline double normal01(uint64_t key, uint64_t counter) {
  const double u1 = (double)((gg_draw(key, 2 * counter) >> 11) + 1) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(gg_draw(key, 2 * counter + 1) >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* In-degrees deg[0..n); returns their sum m. */
int64_t gg_lognormal_indegrees(int64_t n, uint64_t seed, double mu, double sigma, int64_t cap,
                               int64_t* deg) {
  const uint64_t key = gg_stream_key(seed, STREAM_LN_DEGREE);
  int64_t m = 0;
#pragma omp parallel for schedule(static) reduction(+ : m)
  for (int64_t k = 0; k < n; ++k) {
    double d = floor(exp(mu + sigma * normal01(key, (uint64_t)k)) + 0.5);
    if (d > (double)cap) d = (double)cap;
    deg[k] = (int64_t)d;
    m += deg[k];
  }
  return m;
}

/* Edges of target k at [offs[k], offs[k+1]): dst = k, src uniform in [0, n). */
void gg_lognormal_edges(int64_t n, uint64_t seed, const int64_t* offs, int32_t* src,
                        int32_t* dst) {
  const uint64_t key = gg_stream_key(seed, STREAM_LN_SOURCE);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t k = 0; k < n; ++k)
    for (int64_t e = offs[k]; e < offs[k + 1]; ++e) {
      src[e] = (int32_t)bounded(gg_draw(key, (uint64_t)e), (uint64_t)n);
      dst[e] = (int32_t)k;
    }
}

/* Float weights LN(mu, sigma), one per edge index, as IEEE single bit patterns. */
void gg_lognormal_weights(int64_t m, uint64_t seed, double mu, double sigma, uint32_t* w) {
  const uint64_t key = gg_stream_key(seed, STREAM_LN_WEIGHT);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    float f = (float)exp(mu + sigma * normal01(key, (uint64_t)e));
    uint32_t bits;
    memcpy(&bits, &f, sizeof(bits));
    w[e] = bits;
  }
}
