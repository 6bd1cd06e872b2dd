/*
 * CPU oracle for delta-based accumulative iterative computation (DAIC).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load this library.  It shares no code with the
 * CUDA path and is written for obviousness, not speed: plain loops, FP64
 * accumulation, one thread.
 *
 * What it computes (each function cites the passage it follows):
 *   or_linear_power    - the plain definition of a linear fixed point
 *                        v = c + P^T v (Eq. 1 with f affine, the PageRank update
 *                        of Eq. 2), by synchronous pull iteration (Section 2).
 *   or_linear_residual - one application of that update, r = c + P^T v - v.
 *   or_linear_power_edges - the same fixed point with one coefficient per
 *                        edge (the Jacobi row of Table 1, Section 4.3).
 *   or_daic_sum        - asynchronous DAIC with + (Eq. 5, receive/update), in
 *                        round-robin or priority order (Section 3.5).
 *   or_daic_min        - asynchronous DAIC with min (SSSP row of Table 1).
 *   or_dijkstra        - textbook single-source shortest paths (binary heap).
 *   or_bellman_ford    - brute-force relaxation to a fixed point (tiny inputs).
 *   or_max_reach       - connected components by labels (Table 1, max): for
 *                        every vertex the largest id among the vertices that
 *                        reach it (itself included).
 *   or_union_find_max  - components of the undirected version of the graph
 *                        by union-find, labelled with their largest id.
 *   or_dijkstra_f32 / or_bellman_ford_f32 - the same with IEEE single
 *                        weights and distances (the paper's float-weighted
 *                        synthetic SSSP graphs, Section 6.1): every tentative
 *                        distance is fl(d_j + w_jk), rounded to nearest.
 *
 * Conventions: CSR of out-edges, row_ptr[n+1] int64, col[m] int32,
 * per-source coefficient coef[j] (so g_{j,k}(x) = coef[j] * x), integer
 * weights w[m] (uint32).  Infinity for distances is UINT32_MAX.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_INF32 0xFFFFFFFFu

/* ---------------------------------------------------------------- linear */

/* In-edge lists (transpose), so each new v_j is a sum over j's in-neighbours. */
static int transpose(int64_t n, const int64_t* row_ptr, const int32_t* col,
                     int64_t** t_ptr, int32_t** t_src) {
  int64_t m = row_ptr[n];
  int64_t* tp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* ts = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int64_t* fill = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!tp || !ts || !fill) { free(tp); free(ts); free(fill); return -1; }
  for (int64_t e = 0; e < m; ++e) tp[col[e] + 1]++;
  for (int64_t j = 0; j < n; ++j) tp[j + 1] += tp[j];
  for (int64_t j = 0; j < n; ++j) fill[j] = tp[j];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) ts[fill[col[e]]++] = (int32_t)i;
  free(fill);
  *t_ptr = tp;
  *t_src = ts;
  return 0;
}

/*
 * Synchronous iteration of v_j <- c_j + sum_{i -> j} coef_i * v_i from v = 0
 * (Section 2: every vertex updates from the previous iteration's states).  With
 * coef_i = d/|N(i)| and c_j = 1-d this is PageRank (Eq. 2).  Stops when the L1
 * change between two iterations is below tol, or after max_iter iterations.
 * Returns the number of iterations, or -1 on allocation failure.
 */
int64_t or_linear_power(int64_t n, const int64_t* row_ptr, const int32_t* col,
                        const double* coef, const double* c, double tol, int64_t max_iter,
                        double* v_out) {
  int64_t *tp = NULL;
  int32_t *ts = NULL;
  if (transpose(n, row_ptr, col, &tp, &ts) != 0) return -1;
  double* cur = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* nxt = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!cur || !nxt) { free(tp); free(ts); free(cur); free(nxt); return -1; }
  int64_t it = 0;
  for (; it < max_iter; ++it) {
    double change = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      double s = c[j];
      for (int64_t e = tp[j]; e < tp[j + 1]; ++e) s += coef[ts[e]] * cur[ts[e]];
      nxt[j] = s;
      change += fabs(s - cur[j]);
    }
    double* t = cur; cur = nxt; nxt = t;
    if (change < tol) { ++it; break; }
  }
  memcpy(v_out, cur, (size_t)n * sizeof(double));
  free(tp); free(ts); free(cur); free(nxt);
  return it;
}

/*
 * r = c + P^T v - v, computed with a push over out-edges (one application of
 * the update function of Eq. 1).  Since (I - P^T)(v* - v) = r, this bounds the
 * distance to the fixed point of any candidate v without solving for v*.
 */
void or_linear_residual(int64_t n, const int64_t* row_ptr, const int32_t* col,
                        const double* coef, const double* c, const double* v, double* r) {
  for (int64_t j = 0; j < n; ++j) r[j] = c[j] - v[j];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) r[col[e]] += coef[i] * v[i];
}

/* ------------------------------------------------- indexed binary max-heap */

typedef struct {
  int64_t size;
  int32_t* heap;     /* heap[k] = vertex */
  int64_t* pos;      /* pos[vertex] = index in heap, or -1 */
  double* key;       /* key[vertex] */
} maxheap;

static int heap_init(maxheap* h, int64_t n) {
  h->size = 0;
  h->heap = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  h->pos = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  h->key = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!h->heap || !h->pos || !h->key) return -1;
  for (int64_t j = 0; j < n; ++j) h->pos[j] = -1;
  return 0;
}
static void heap_free(maxheap* h) { free(h->heap); free(h->pos); free(h->key); }
static void heap_swap(maxheap* h, int64_t a, int64_t b) {
  int32_t x = h->heap[a], y = h->heap[b];
  h->heap[a] = y; h->heap[b] = x;
  h->pos[y] = a; h->pos[x] = b;
}
/* larger key first; equal keys: smaller vertex id first */
static int heap_above(const maxheap* h, int64_t a, int64_t b) {
  double ka = h->key[h->heap[a]], kb = h->key[h->heap[b]];
  return ka > kb || (ka == kb && h->heap[a] < h->heap[b]);
}
static void heap_up(maxheap* h, int64_t k) {
  while (k > 0) {
    int64_t p = (k - 1) / 2;
    if (!heap_above(h, k, p)) break;
    heap_swap(h, k, p);
    k = p;
  }
}
static void heap_down(maxheap* h, int64_t k) {
  for (;;) {
    int64_t l = 2 * k + 1, r = l + 1, b = k;
    if (l < h->size && heap_above(h, l, b)) b = l;
    if (r < h->size && heap_above(h, r, b)) b = r;
    if (b == k) break;
    heap_swap(h, k, b);
    k = b;
  }
}
/* insert, or move to its new key */
static void heap_set(maxheap* h, int32_t v, double key) {
  h->key[v] = key;
  if (h->pos[v] < 0) {
    h->heap[h->size] = v;
    h->pos[v] = h->size++;
    heap_up(h, h->pos[v]);
  } else {
    heap_up(h, h->pos[v]);
    heap_down(h, h->pos[v]);
  }
}
static int32_t heap_pop(maxheap* h) {
  int32_t top = h->heap[0];
  heap_swap(h, 0, h->size - 1);
  h->size--;
  h->pos[top] = -1;
  if (h->size > 0) heap_down(h, 0);
  return top;
}

/* ------------------------------------------------------ asynchronous DAIC */

/*
 * One update of vertex j with + (Eq. 5, update): fold the pending delta into
 * the state, send g_{j,k}(delta) = coef_j * delta to every out-neighbour k
 * (each message is received at once: Delta_k += message), reset Delta_j to 0.
 * The delta folded at a vertex without out-edges is added to *leak.
 */
static void update_sum(int32_t j, const int64_t* row_ptr, const int32_t* col,
                       const double* coef, double* v, double* delta, double* leak,
                       maxheap* pq) {
  double dj = delta[j];
  v[j] += dj;
  delta[j] = 0.0;
  if (pq && pq->pos[j] >= 0) heap_set(pq, j, 0.0);
  if (row_ptr[j + 1] == row_ptr[j]) { *leak += dj; return; }
  double msg = coef[j] * dj;
  if (msg == 0.0) return;   /* the paper sends only messages different from 0 */
  for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
    int32_t k = col[e];
    delta[k] += msg;
    if (pq) heap_set(pq, k, fabs(delta[k]));
  }
}

static double l1(const double* x, int64_t n) {
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j) s += fabs(x[j]);
  return s;
}

/*
 * Asynchronous DAIC with + (Eq. 5) from state (v, delta) in place.
 * sched = 0: round-robin, sweeping the state table in vertex order and
 *            updating every vertex whose delta is not 0 (Section 3.5);
 * sched = 1: priority, always updating argmax_j |Delta_j| next, which is the
 *            priority |v_j + Delta_j - v_j| of Section 3.5 (ties: lower id).
 * Stops when sum_j |Delta_j| < eps (checked after every sweep, and every n
 * updates under priority) or after max_updates updates.
 * Outputs: *leak accumulates the delta folded at vertices without out-edges,
 * *updates counts updates, *pushes counts messages sent.
 * Returns 0 when converged, 1 when max_updates was hit, -1 on allocation failure.
 */
int or_daic_sum(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* coef,
                double* v, double* delta, int sched, double eps, int64_t max_updates,
                double* leak, int64_t* updates, int64_t* pushes) {
  int64_t upd = 0, msgs = 0;
  if (sched == 0) {
    while (l1(delta, n) >= eps) {
      for (int64_t j = 0; j < n; ++j) {
        if (delta[j] == 0.0) continue;
        if (upd >= max_updates) { *updates = upd; *pushes = msgs; return 1; }
        msgs += row_ptr[j + 1] - row_ptr[j];
        update_sum((int32_t)j, row_ptr, col, coef, v, delta, leak, NULL);
        ++upd;
      }
    }
    *updates = upd;
    *pushes = msgs;
    return 0;
  }
  maxheap pq;
  if (heap_init(&pq, n) != 0) { heap_free(&pq); return -1; }
  for (int64_t j = 0; j < n; ++j)
    if (delta[j] != 0.0) heap_set(&pq, (int32_t)j, fabs(delta[j]));
  int rc = 0;
  for (;;) {
    if (upd % (n > 0 ? n : 1) == 0 && l1(delta, n) < eps) break;
    if (pq.size == 0 || pq.key[pq.heap[0]] == 0.0) break;
    if (upd >= max_updates) { rc = 1; break; }
    int32_t j = heap_pop(&pq);
    msgs += row_ptr[j + 1] - row_ptr[j];
    update_sum(j, row_ptr, col, coef, v, delta, leak, &pq);
    ++upd;
  }
  if (rc == 0 && l1(delta, n) >= eps) rc = 1;
  heap_free(&pq);
  *updates = upd;
  *pushes = msgs;
  return rc;
}

/*
 * Asynchronous DAIC with min and g_{j,k}(x) = x + w_jk (SSSP row of Table 1),
 * from (v, delta) in place; infinity is UINT32_MAX and x + w saturates there.
 * Update of j (Eq. 5): v_j <- min(v_j, Delta_j); send Delta_j + w_jk to every
 * out-neighbour k (Delta_k <- min(Delta_k, message)); reset Delta_j to the
 * identity of min, infinity.  A vertex is worth updating only when
 * min(v_j, Delta_j) differs from v_j, i.e. Delta_j < v_j.
 * sched = 0: round-robin sweeps; sched = 1: priority v_j - min(v_j, Delta_j)
 * of the SSSP subsection, with v_j = infinity read as the largest priority and
 * ties broken towards the smaller delta, then the lower id.
 * Stops when no vertex has Delta_j < v_j.  Returns 0, or 1 if max_updates hit.
 */
int or_daic_min(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                uint32_t* v, uint32_t* delta, int sched, int64_t max_updates,
                int64_t* updates, int64_t* pushes) {
  int64_t upd = 0, msgs = 0;
  int rc = 0;
  if (sched == 0) {
    int changed = 1;
    while (changed) {
      changed = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (!(delta[j] < v[j])) continue;
        if (upd >= max_updates) { rc = 1; goto done; }
        uint32_t dj = delta[j];
        v[j] = dj;
        delta[j] = OR_INF32;
        for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
          uint64_t s = (uint64_t)dj + w[e];
          uint32_t msg = s >= OR_INF32 ? OR_INF32 : (uint32_t)s;
          if (msg < delta[col[e]]) delta[col[e]] = msg;
          ++msgs;
        }
        ++upd;
        changed = 1;
      }
    }
  } else {
    /* priority key: larger first; v = inf -> 2^40 + (2^32 - delta), else v - delta */
    maxheap pq;
    if (heap_init(&pq, n) != 0) { heap_free(&pq); return -1; }
#define MINKEY(j) (v[j] == OR_INF32 ? 1099511627776.0 + (4294967296.0 - (double)delta[j]) \
                                    : (double)(v[j] - delta[j]))
    for (int64_t j = 0; j < n; ++j)
      if (delta[j] < v[j]) heap_set(&pq, (int32_t)j, MINKEY(j));
    while (pq.size > 0) {
      if (upd >= max_updates) { rc = 1; break; }
      int32_t j = heap_pop(&pq);
      uint32_t dj = delta[j];
      v[j] = dj;
      delta[j] = OR_INF32;
      for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
        int32_t k = col[e];
        uint64_t s = (uint64_t)dj + w[e];
        uint32_t msg = s >= OR_INF32 ? OR_INF32 : (uint32_t)s;
        if (msg < delta[k]) {
          delta[k] = msg;
          if (delta[k] < v[k]) heap_set(&pq, k, MINKEY(k));
        }
        ++msgs;
      }
      ++upd;
    }
#undef MINKEY
    heap_free(&pq);
  }
done:
  *updates = upd;
  *pushes = msgs;
  return rc;
}

/* ------------------------------------------------------- shortest paths */

typedef struct { uint64_t d; int32_t v; } hitem;

static void hpush(hitem* h, int64_t* sz, hitem x) {
  int64_t k = (*sz)++;
  h[k] = x;
  while (k > 0) {
    int64_t p = (k - 1) / 2;
    if (h[p].d <= h[k].d) break;
    hitem t = h[p]; h[p] = h[k]; h[k] = t;
    k = p;
  }
}
static hitem hpop(hitem* h, int64_t* sz) {
  hitem top = h[0];
  h[0] = h[--(*sz)];
  int64_t k = 0;
  for (;;) {
    int64_t l = 2 * k + 1, r = l + 1, b = k;
    if (l < *sz && h[l].d < h[b].d) b = l;
    if (r < *sz && h[r].d < h[b].d) b = r;
    if (b == k) break;
    hitem t = h[b]; h[b] = h[k]; h[k] = t;
    k = b;
  }
  return top;
}

/*
 * Dijkstra's algorithm with a binary heap and lazy deletion, 64-bit distances.
 * dist_out[j] = shortest distance from src, UINT32_MAX if unreachable.
 * Returns 0, -1 on allocation failure, -2 if a distance does not fit below
 * UINT32_MAX (the 32-bit encoding would be ambiguous).
 */
int or_dijkstra(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                int32_t src, uint32_t* dist_out) {
  int64_t m = row_ptr[n];
  uint64_t* dist = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
  char* done = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  hitem* h = (hitem*)malloc((size_t)(m + 2) * sizeof(hitem));
  if (!dist || !done || !h) { free(dist); free(done); free(h); return -1; }
  for (int64_t j = 0; j < n; ++j) dist[j] = UINT64_MAX;
  int64_t sz = 0;
  dist[src] = 0;
  hitem s0 = {0, src};
  hpush(h, &sz, s0);
  while (sz > 0) {
    hitem t = hpop(h, &sz);
    if (done[t.v]) continue;
    done[t.v] = 1;
    for (int64_t e = row_ptr[t.v]; e < row_ptr[t.v + 1]; ++e) {
      uint64_t nd = t.d + w[e];
      int32_t k = col[e];
      if (nd < dist[k]) {
        dist[k] = nd;
        hitem x = {nd, k};
        hpush(h, &sz, x);
      }
    }
  }
  int rc = 0;
  for (int64_t j = 0; j < n; ++j) {
    if (dist[j] == UINT64_MAX) dist_out[j] = OR_INF32;
    else if (dist[j] >= OR_INF32) { dist_out[j] = OR_INF32; rc = -2; }
    else dist_out[j] = (uint32_t)dist[j];
  }
  free(dist); free(done); free(h);
  return rc;
}

/* Bellman-Ford: relax every edge until nothing changes (n-1 passes suffice). */
void or_bellman_ford(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                     int32_t src, uint32_t* dist) {
  for (int64_t j = 0; j < n; ++j) dist[j] = OR_INF32;
  dist[src] = 0;
  for (int64_t pass = 0; pass < n; ++pass) {
    int changed = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (dist[i] == OR_INF32) continue;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        uint64_t nd = (uint64_t)dist[i] + w[e];
        if (nd < dist[col[e]]) { dist[col[e]] = (uint32_t)nd; changed = 1; }
      }
    }
    if (!changed) break;
  }
}

/* ------------------------------------------------- float shortest paths */

/*
 * Dijkstra's algorithm on float weights w (IEEE single, finite, >= 0), every
 * distance formed in single precision as fl(dist[j] + w[e]) (C float
 * addition, round to nearest).  With w >= 0, fl(d + w) >= d, so a vertex's
 * distance is final when it leaves the heap, exactly as with exact
 * arithmetic; the result is the least, over paths from src, of the path's
 * sum accumulated from the source in single precision.  Unreachable: +inf.
 * Heap keys are the distances' bit patterns (ordered like the values for
 * non-negative floats).  Returns 0, or -1 on allocation failure.
 */
static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

int or_dijkstra_f32(int64_t n, const int64_t* row_ptr, const int32_t* col, const float* w,
                    int32_t src, float* dist) {
  int64_t m = row_ptr[n];
  char* done = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  hitem* h = (hitem*)malloc((size_t)(m + 2) * sizeof(hitem));
  if (!done || !h) { free(done); free(h); return -1; }
  for (int64_t j = 0; j < n; ++j) dist[j] = INFINITY;
  int64_t sz = 0;
  dist[src] = 0.0f;
  hitem s0 = {0, src};
  hpush(h, &sz, s0);
  while (sz > 0) {
    hitem t = hpop(h, &sz);
    if (done[t.v]) continue;
    done[t.v] = 1;
    for (int64_t e = row_ptr[t.v]; e < row_ptr[t.v + 1]; ++e) {
      float nd = dist[t.v] + w[e];
      int32_t k = col[e];
      if (nd < dist[k]) {
        dist[k] = nd;
        hitem x = {f2u(nd), k};
        hpush(h, &sz, x);
      }
    }
  }
  free(done); free(h);
  return 0;
}

/* Float Bellman-Ford: relax every edge in single precision until nothing changes. */
void or_bellman_ford_f32(int64_t n, const int64_t* row_ptr, const int32_t* col, const float* w,
                         int32_t src, float* dist) {
  for (int64_t j = 0; j < n; ++j) dist[j] = INFINITY;
  dist[src] = 0.0f;
  for (int64_t pass = 0; pass < n; ++pass) {
    int changed = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (isinf(dist[i])) continue;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        float nd = dist[i] + w[e];
        if (nd < dist[col[e]]) { dist[col[e]] = nd; changed = 1; }
      }
    }
    if (!changed) break;
  }
}

/* ------------------------------------------------------- component labels */

/*
 * label[j] = max { i : there is a path i ->* j } (j reaches itself).  Sources
 * in decreasing id order: a breadth-first search from i labels every vertex
 * it reaches that is still unlabelled, and stops at labelled ones (whatever a
 * labelled vertex reaches was already labelled from a larger id).  O(n + m).
 * Returns 0, or -1 on allocation failure.
 */
int or_max_reach(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t* label) {
  int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!queue) return -1;
  for (int64_t j = 0; j < n; ++j) label[j] = -1;
  for (int64_t i = n - 1; i >= 0; --i) {
    if (label[i] >= 0) continue;
    int64_t head = 0, tail = 0;
    label[i] = (int32_t)i;
    queue[tail++] = (int32_t)i;
    while (head < tail) {
      int32_t u = queue[head++];
      for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        int32_t k = col[e];
        if (label[k] < 0) { label[k] = (int32_t)i; queue[tail++] = k; }
      }
    }
  }
  free(queue);
  return 0;
}

static int32_t uf_find(int32_t* parent, int32_t x) {
  while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
  return x;
}

/* Union-find over every edge as undirected; label = largest id of the set. */
int or_union_find_max(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t* label) {
  int32_t* parent = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!parent) return -1;
  for (int64_t j = 0; j < n; ++j) parent[j] = (int32_t)j;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
      int32_t a = uf_find(parent, (int32_t)j), b = uf_find(parent, col[e]);
      if (a != b) { if (a < b) parent[a] = b; else parent[b] = a; }   /* larger id is the root */
    }
  for (int64_t j = 0; j < n; ++j) label[j] = uf_find(parent, (int32_t)j);
  free(parent);
  return 0;
}

/* ----------------------------------------------- per-edge linear update */

/*
 * Synchronous iteration of v_k <- c_k + sum_{e = (j -> k)} ecoef_e * v_j from
 * v = 0, edges taken in CSR order (the Jacobi method of Section 4.3 when
 * ecoef_e = -A_kj / A_kk and c_k = b_k / A_kk).  Stops when the L1 change
 * between two iterations is below tol, or after max_iter iterations.
 * Returns the number of iterations, or -1 on allocation failure.
 */
int64_t or_linear_power_edges(int64_t n, const int64_t* row_ptr, const int32_t* col,
                              const double* ecoef, const double* c, double tol,
                              int64_t max_iter, double* v_out) {
  double* cur = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* nxt = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!cur || !nxt) { free(cur); free(nxt); return -1; }
  int64_t it = 0;
  for (; it < max_iter; ++it) {
    memcpy(nxt, c, (size_t)n * sizeof(double));
    for (int64_t j = 0; j < n; ++j)
      for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) nxt[col[e]] += ecoef[e] * cur[j];
    double change = 0.0;
    for (int64_t j = 0; j < n; ++j) change += fabs(nxt[j] - cur[j]);
    double* t = cur; cur = nxt; nxt = t;
    if (change < tol) { ++it; break; }
  }
  memcpy(v_out, cur, (size_t)n * sizeof(double));
  free(cur); free(nxt);
  return it;
}
