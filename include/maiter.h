/*
 * maiter.h - C ABI of a single-GPU (B300, sm_103a) engine for delta-based
 * accumulative iterative computation (DAIC), after "Maiter: An Asynchronous
 * Graph Processing Framework for Delta-based Accumulative Iterative
 * Computation" (Zhang, Gao, Gao, Wang).
 *
 * What the engine computes.  A DAIC is the tuple (g_{j,k}, (+), v0, Delta1)
 * (Section 4.1, Table 1).  Each activated vertex j performs the update of the
 * asynchronous DAIC (Eq. 5):
 *     v_j <- v_j (+) Delta_j;
 *     for every out-edge (j, k): Delta_k <- Delta_k (+) g_{j,k}(Delta_j),
 *         skipped when the message equals the identity 0 of (+);
 *     Delta_j <- 0.
 * Vertices are activated by a scheduling policy (Section 3.5): all pending
 * vertices (round-robin), those above a threshold, or a top fraction by
 * priority |v_j (+) Delta_j - v_j|.  The run stops when the termination test
 * of Section 5.1 holds: sum_j |Delta_j| < eps for (+) = +, no pending vertex
 * for (+) = min.  By Theorems 1 and 3 the result is the fixed point of the
 * plain iteration v = f(v) (Eq. 1) whatever the schedule.
 *
 * Only (+, g) pairs that satisfy the four DAIC conditions of Section 3.1 are
 * offered: + with a linear g, and min with g(x) = x + w.  No user callbacks
 * cross this boundary.
 *
 * Conventions for every call:
 *  - Every call returns a maiter_status (0 = success) and never aborts; on
 *    failure maiter_last_error() returns a message (thread-local).
 *  - Array arguments may be host or device pointers; the kind is detected
 *    with cudaPointerGetAttributes.  Inputs are copied; the caller keeps
 *    ownership of everything it passes.
 *  - Graph layout: CSR of OUT-edges.  row_ptr[n+1] (int64, row_ptr[0] = 0,
 *    non-decreasing, row_ptr[n] = m), col[m] (int32, 0 <= col < n), optional
 *    w[m] (uint32 edge weights).  Multi-edges and self-loops are allowed.
 *    Limits: n < 2^31, m < 2^31.
 *  - The engine runs on the device given at maiter_graph_create and on the
 *    stream given in the run parameters; calls are synchronous w.r.t. the
 *    host (they return after the device work they issued has finished),
 *    except where stated.
 */
#ifndef MAITER_H
#define MAITER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct maiter_graph maiter_graph;    /* opaque: device copy of the CSR */
typedef struct maiter_result maiter_result;  /* opaque: device v, Delta, workspace, stats */

typedef enum {
  MAITER_OK = 0,
  MAITER_ERR_INVALID_ARG = -1,   /* bad pointer, size, enum, CSR or value */
  MAITER_ERR_OOM = -2,           /* device or pinned allocation failed */
  MAITER_ERR_CUDA = -3,          /* a CUDA call failed; message has details */
  MAITER_ERR_NOT_CONVERGED = -4, /* max_rounds reached; state is readable */
  MAITER_ERR_TIMEOUT = -5,       /* a bounded device wait ran out; state readable */
  MAITER_ERR_UNSUPPORTED = -6    /* valid request this build does not serve */
} maiter_status;

/* The accumulation operator (+) and the precision of each field. */
typedef enum {
  MAITER_OP_SUM_F64 = 0,   /* (+) = +; v, Delta, coefficients, residual FP64 */
  MAITER_OP_SUM_MIXED = 1, /* (+) = +; Delta and coefficients FP32, v and the
                              residual reduction FP64 (after an FP64-delta
                              warm-up phase, see mixed_switch) */
  MAITER_OP_MIN_U32 = 2,   /* (+) = min over uint32, identity UINT32_MAX (inf) */
  MAITER_OP_MIN_F32 = 3,   /* (+) = min over IEEE float32 distances >= 0, identity
                              +inf; the graph's 32-bit weights are read as floats
                              (finite, >= 0: checked once per graph), messages are
                              fl(Delta_j + w) rounded to nearest.  v and Delta are
                              returned as float32.  Round engine, schedules ALL,
                              THRESHOLD (as ALL), TOPFRAC and BUCKET. */
  MAITER_OP_MAX_I32 = 4    /* (+) = max over int32 labels, identity -1 (connected
                              components, Table 1): with g = IDENTITY, v0 = -1 and
                              Delta^1_j = j by default, every vertex ends with the
                              largest id among the vertices that reach it (its
                              component's largest id on a symmetric graph).
                              Round engine, schedules ALL, THRESHOLD (as ALL) and
                              TOPFRAC (priority Delta_j - v_j). */
} maiter_op;

/* The message function g_{j,k}. */
typedef enum {
  MAITER_G_SCALE_BY_SRC = 0, /* g_{j,k}(x) = coef[j] * x.  With coef == NULL,
                                coef[j] = damping / outdeg(j) (PageRank,
                                Section 4.2, sender's out-degree). */
  MAITER_G_ADD_EDGE = 1,     /* g_{j,k}(x) = x + w[e] (SSSP, Table 1), saturating
                                at UINT32_MAX; needs edge weights */
  MAITER_G_SCALE_BY_EDGE = 2, /* g_{j,k}(x) = coef[e] * x with one FP64 coefficient
                                per edge e = (j, k), in CSR order (SUM_F64 only):
                                the Jacobi method's -A_kj / A_kk (Table 1); signed */
  MAITER_G_IDENTITY = 3      /* g_{j,k}(x) = x (connected components, MAX_I32) */
} maiter_g;

/* Which vertices an iteration activates (Section 3.5, Section 5.1). */
typedef enum {
  MAITER_SCHED_ALL = 0,       /* every vertex with a pending delta
                                 (Delta_j != 0 for +, Delta_j < v_j for min) */
  MAITER_SCHED_THRESHOLD = 1, /* +: |Delta_j| > threshold; min: as ALL */
  MAITER_SCHED_TOPFRAC = 2,   /* the top_frac fraction of pending vertices by
                                 priority, ties included (priority queue of
                                 Section 5.1) */
  MAITER_SCHED_LEARNED = 3,   /* about the top_frac fraction of pending vertices
                                 by the score of a learned network (params.scorer,
                                 a maiter_mlp): the threshold is the score ranked
                                 top_frac among 4096 vertices drawn by a hash of
                                 the round (extraction by sampling, Section 5.1);
                                 every 8th round activates every pending vertex,
                                 so none can starve (Theorem 3 needs every vertex
                                 updated again eventually) */
  MAITER_SCHED_BUCKET = 4     /* min only, distance-ordered (delta-stepping): the
                                 pending vertices with Delta_j < tau, where tau starts
                                 at the bucket width `threshold` and, whenever no
                                 pending vertex lies below it, moves to the smallest
                                 pending Delta plus the width (priority by distance,
                                 the ordered variant of the SSSP priority of
                                 Section 4.1); same fixed point */
} maiter_sched;

typedef struct maiter_mlp maiter_mlp;       /* opaque: learned priority scorer */

typedef enum {
  MAITER_ENGINE_SYNC = 0,     /* round loop: frontier, then push; the loop and its
                                 termination test run on the device (CUDA graph
                                 with a conditional node), no host round trip */
  MAITER_ENGINE_ASYNC = 1,    /* persistent kernel of round-robin workers: every
                                 CTA owns an interleaved share of the vertices and
                                 sweeps it again and again, updating each pending
                                 vertex it finds and scattering its messages with
                                 atomics, with no barrier between CTAs (Eq. 5,
                                 Section 3.2).  A launch ends when no CTA finds
                                 work; between launches an exact device reduction
                                 tests termination (the periodic check of Section
                                 5.1).  Sums update a vertex whose |delta| exceeds
                                 half the mean |delta| of the check before (ALL:
                                 never less than eps / (2n)).  SUM_F64 and MIN_U32;
                                 schedules ALL and THRESHOLD. */
  MAITER_ENGINE_BINNED = 2,   /* rounds in which every vertex with a pending delta
                                 sends (the synchronous DAIC of Section 3.2, schedule
                                 ALL), for SUM_F64 / SUM_MIXED with g = SCALE_BY_SRC.
                                 The messages of a round are written to bins of
                                 16384 receivers (one slot per edge, in a layout the
                                 library builds from the CSR on first use and after
                                 maiter_graph_update) and each bin is summed in
                                 shared memory in FP64, then folded: no atomic in
                                 global memory per edge.  Needs n <= 2^28; memory
                                 about 4 bytes per edge for the layout plus 8 per
                                 edge for the messages of a result.  The loop and its
                                 termination test run on the device as for SYNC. */
  MAITER_ENGINE_PULL = 3      /* the same dense rounds (schedule ALL, SUM_F64 /
                                 SUM_MIXED, g = SCALE_BY_SRC) with the receive step
                                 of Eq. 5 computed at the receivers: every vertex
                                 sums the messages c_j Delta_j of its in-neighbours
                                 over the transpose of the graph (built by the
                                 library on first use and after maiter_graph_update:
                                 about 5 bytes per edge + 12 per vertex; messages
                                 are stored by sender rank), then folds.  No atomic
                                 per edge; one per 4096 in-edges of a vertex with
                                 more than 2048.  Memory per result: two n x 8 byte
                                 message buffers.  The loop and its termination
                                 test run on the device as for SYNC. */
} maiter_engine;

/* Run flags (bit set). */
typedef enum {
  MAITER_FLAG_PROFILE_KERNELS = 1, /* drive the round loop from the host, one
                                      launch per kernel with CUDA events around
                                      each, and report per-kernel device time in
                                      maiter_stats (same kernels and launch
                                      shapes; one host sync per round) */
  MAITER_FLAG_INJECT_STALL = 2     /* ASYNC, for testing the bounded waits: the
                                      first queue launch gets a phantom pending
                                      item that nothing completes, so its idle
                                      warps wait timeout_ms and the run returns
                                      MAITER_ERR_TIMEOUT (no fault, no hang) */
} maiter_flags;

typedef struct maiter_run_params {
  int32_t op;          /* maiter_op */
  int32_t g;           /* maiter_g; must be SCALE_BY_SRC for sums, ADD_EDGE for min */
  int32_t sched;       /* maiter_sched */
  int32_t engine;      /* maiter_engine */
  int32_t flags;       /* maiter_flags */
  int32_t reserved0;   /* must be 0 */
  const void* coef;    /* n per-source coefficients (double for SUM_F64, float for
                          SUM_MIXED), host or device, or NULL (see damping);
                          with g = SCALE_BY_EDGE: m per-edge doubles (required) */
  double damping;      /* d in coef[j] = d / outdeg(j) when coef == NULL */
  const void* v0;      /* n initial states (double for sums, uint32 / float for min,
                          int32 for max), or NULL: the identity (0 for +,
                          infinity for min, -1 for max) */
  const void* delta0;  /* n initial deltas (double for both sums, uint32 / float for
                          min, int32 for max), or NULL: 1 - damping everywhere for
                          sums (PageRank, Table 1), 0 at `source` and infinity
                          elsewhere for min, Delta_j = j for max */
  int64_t source;      /* min with delta0 == NULL: the source vertex */
  double threshold;    /* THRESHOLD: activate |Delta_j| > threshold.  When a
                          round selects nothing while the residual is still
                          >= eps, the threshold is divided by 10 (down to 0) so
                          every run terminates.  BUCKET: the bucket width (> 0,
                          at least 1 is meaningful for integer distances). */
  double top_frac;     /* TOPFRAC: fraction q in (0, 1] */
  double eps;          /* sums: stop when sum_j |Delta_j| < eps (FP64 reduction) */
  double mixed_switch; /* SUM_MIXED: deltas are FP64 until the residual has
                          fallen to mixed_switch x its initial value, then
                          rounded once to FP32 for the rest of the run (default
                          0.01; 1 = FP32 deltas from the first round, 0 = FP64
                          deltas throughout).  FP32 accumulation of many
                          messages into one delta loses ~sqrt(k) ulps at a
                          vertex of in-degree k, which is why the large early
                          deltas are accumulated in FP64.  Under TOPFRAC and
                          LEARNED a held-back vertex's delta grows over several
                          rounds, so its messages round at a coarser step:
                          1e-3 keeps PageRank at R-MAT scale 24 within 1e-6
                          (measured 1.6e-7 at LEARNED q = 0.5, against 8.3e-7
                          at 0.01). */
  int64_t max_rounds;  /* round cap; <= 0 means 1,000,000 */
  int64_t timeout_ms;  /* ASYNC: budget of every bounded device wait per launch
                          (0 = 10,000 ms); when it runs out the run returns
                          MAITER_ERR_TIMEOUT with a valid, resumable state */
  void* stream;        /* cudaStream_t to run on; NULL = the default stream */
  /* Tuning (0 = built-in default), e.g. from the autotuner: */
  int32_t cut_warp;    /* out-degree below which a vertex takes the warp-gathered
                          path (default 32) */
  int32_t cut_cta;     /* out-degree from which a vertex is split into 1024-edge
                          chunks, one CTA each (default 512) */
  int32_t push_blocks_per_sm;  /* cap on resident push CTAs per SM (default: occupancy) */
  int32_t reserved1;   /* must be 0 */
  const maiter_mlp* scorer;    /* LEARNED: the network (same device as the graph) */
} maiter_run_params;

typedef struct maiter_stats {
  int64_t rounds;        /* frontier/push rounds executed */
  int64_t activations;   /* vertex updates performed */
  int64_t edge_pushes;   /* messages sent (sum of out-degrees of updated vertices) */
  double residual;       /* final sum_j |Delta_j| (sums) or pending count (min) */
  double elapsed_ms;     /* device time of the run (CUDA events) */
  int32_t status;        /* maiter_status of the run */
  int32_t converged;     /* 1 if the termination test held */
  int64_t kernel_launches; /* kernels this run launched */
  /* Filled only under MAITER_FLAG_PROFILE_KERNELS (else 0): */
  double push_ms;        /* summed device time of the push (update+scatter) kernel */
  double scan_ms;        /* summed device time of the frontier/termination kernel */
  int64_t push_launches;
  int64_t scan_launches;
  /* SUM_MIXED: the part of rounds / activations / edge_pushes spent in the
     FP64-delta warm-up phase (0 for other ops) */
  int64_t warm_rounds;
  int64_t warm_activations;
  int64_t warm_edge_pushes;
  /* ENGINE_BINNED: padded edge slots of the layout (every round moves one
     message per slot), and under MAITER_FLAG_PROFILE_KERNELS the summed
     device time of its two round kernels (push_ms is their sum) */
  int64_t slots;
  double bin_scatter_ms;
  double bin_gather_ms;
} maiter_stats;

/* Fills *p with defaults: PageRank-style sum in FP64, d = 0.8, sched ALL,
 * eps = 1e-8, threshold = 0, top_frac = 0.01, source = -1, max_rounds 1e6.
 * Paper: the PageRank IterateKernel of Section 5.2 (v = 0, Delta = 1 - d,
 * + as accumulate, d / outdeg as send) and the 1 % queue of Section 5.1. */
void maiter_params_default(maiter_run_params* p);

/* Paper: the Partitioner of Section 5.2, which fills each state-table
 * entry's data field (Section 5.1) with the vertex's adjacency list.  Here
 * the caller's CSR is the single partition and row j's targets are entry j's
 * data field.
 * Uploads and validates a CSR of out-edges (layout above) on `device`.
 * w may be NULL (no weights; min runs then fail with INVALID_ARG).
 * On success *out owns device copies; free with maiter_graph_destroy.
 * Errors: INVALID_ARG (sizes, ordering, col range), OOM, CUDA. */
maiter_status maiter_graph_create(int64_t n, int64_t m, const int64_t* row_ptr,
                                  const int32_t* col, const uint32_t* w, int device,
                                  maiter_graph** out);

/* Paper: the Partitioner of Section 5.2 again (the data field of every
 * state-table entry, Section 5.1), for a new input of the same shape.
 * Replaces the contents of g with another CSR of the same n and m (and
 * weights iff g has them), from host or device arrays, stream-ordered on
 * `stream` (NULL = default stream; pinned host arrays copy asynchronously),
 * then validates it like maiter_graph_create and returns after validation.
 * Device buffers keep their addresses, so results created for g and their
 * cached launch graphs stay valid: a stream of same-shaped inputs reuses
 * them.  Quantities derived from the contents (in-degrees, the float-weight
 * check) are recomputed on their next use.  The caller orders the update
 * against runs of g on other streams.  Errors: INVALID_ARG (after which g
 * refuses runs until a valid update), CUDA. */
maiter_status maiter_graph_update(maiter_graph* g, const int64_t* row_ptr, const int32_t* col,
                                  const uint32_t* w, void* stream);

/* Frees the device copy of the CSR (the state table's data fields,
 * Section 5.1); NULL is ignored.  Every run on g must have returned. */
void maiter_graph_destroy(maiter_graph* g);

/* Paper: the IterateKernel (init = v0 / delta0, accumulate = op, send = g)
 * and TermChecker (eps) of Section 5.2, executed as the asynchronous DAIC of
 * Section 3.2 (Eq. 5) under the scheduling of Section 3.5 / Section 5.1.
 * Runs a DAIC to termination (Eq. 5 updates, Section 3.5 schedules).
 * If *out is NULL a new result is allocated; otherwise *out must be a result
 * earlier returned for this graph and is reused without allocation (its
 * previous state is overwritten).  On OK, NOT_CONVERGED and TIMEOUT, *out
 * holds a readable result whose (v, Delta) is a valid DAIC state (it can be
 * passed back as v0/delta0 to resume); on other errors a freshly allocated
 * result is freed and *out is left as it was.  A result may be destroyed
 * before or after its graph; a graph must outlive every run on it.
 * Errors: INVALID_ARG, OOM, CUDA, NOT_CONVERGED, TIMEOUT, UNSUPPORTED. */
maiter_status maiter_run(const maiter_graph* g, const maiter_run_params* p,
                         maiter_result** out);

/* Paper: the dump of the state table's v fields when the terminator stops
 * the run (Section 5.1, Iteration Termination).
 * Copies the n states v into `out` (host or device): double for sums, uint32
 * for min, float for MIN_F32, int32 for max.  count must equal n.
 * Errors: INVALID_ARG (NULL, count), CUDA. */
maiter_status maiter_get_state(const maiter_result* r, void* out, int64_t count);

/* Paper: the state table's Delta fields (Section 5.1); with the states they
 * form the complete DAIC state (v, Delta) that a checkpoint saves (Section
 * 5.1, Fault Tolerance) and that resumes a run as v0 / delta0.
 * Copies the n pending deltas Delta into `out`: double (SUM_F64), float
 * (SUM_MIXED) or uint32 (min).  count must equal n.
 * Errors: INVALID_ARG (NULL, count), CUDA. */
maiter_status maiter_get_delta(const maiter_result* r, void* out, int64_t count);

/* Paper: the progress estimator / terminator of Section 5.1 (TermChecker,
 * Section 5.2): the last residual sum_j |Delta_j| the device measured, the
 * rounds, updates and messages of the run, and its device time.
 * Errors: INVALID_ARG (NULL). */
maiter_status maiter_get_stats(const maiter_result* r, maiter_stats* out);

/* Frees a result's device state table (v, Delta: Section 5.1) and workspace;
 * NULL is ignored.  May come before or after maiter_graph_destroy. */
void maiter_result_destroy(maiter_result* r);

/* SSSP (min, g(x) = x + w, all pending vertices per round) that allocates no
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that hold device buffers but may not call cudaMalloc - for example a plugin
 * whose device memory belongs to a host framework's caching allocator (an
 * allocation behind that allocator's back can fail or fragment its pool), or
 * a caller with a fixed memory budget.
 *
 * Inputs (device pointers on `device` only): row_ptr[n+1] as INT32 offsets
 * (row_ptr[0] = 0, non-decreasing, row_ptr[n] = m), col[m], w[m]; source in
 * [0, n).  Outputs (device, caller-owned): v_out[n] receives the distances
 * (UINT32_MAX if unreachable), delta_out[n] the final deltas.  *rounds_out
 * (host, may be NULL) receives the number of rounds.  A buffer that is not
 * device memory of `device` (host memory, or another GPU's) is rejected with
 * INVALID_ARG before anything is launched.
 *
 * Working memory: the frontier lists and the control block live in one
 * fixed device array inside the library, 8 MiB + 512 B, which every GPU that
 * loads the library holds until the process exits.  Hence n is limited to
 * 1,048,576 (2^20) vertices; larger n returns MAITER_ERR_INVALID_ARG with a
 * message.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current).  All calls share the one
 * array and it keeps the previous call's contents (each call resets what must
 * start at zero), so calls that overlap on the GPU - on two streams, or from
 * two threads - race and must be serialised by the caller.
 *
 * The round loop runs from the host: per round two kernel launches on
 * `stream` and a small device-to-host read of the control block (into a host
 * stack variable) that the host waits for, so the call returns when the
 * distances are final.  `stream` (NULL = the default stream) must therefore
 * not be capturing; a capturing stream, or the default stream while another
 * stream captures, is rejected with INVALID_ARG before anything is launched.
 * Errors: INVALID_ARG (sizes, pointers, stream, bad CSR), NOT_CONVERGED
 * (max_rounds, <= 0 means 1,000,000; the state is readable), CUDA. */
maiter_status maiter_sssp_noalloc(int64_t n, int64_t m, const int32_t* row_ptr,
                                  const int32_t* col, const uint32_t* w, int64_t source,
                                  uint32_t* v_out, uint32_t* delta_out, int64_t max_rounds,
                                  int device, void* stream, int64_t* rounds_out);

/* -------------------------------------------------------- learned scorer
 * Paper: the priority field of the state table and the priority queue that
 * extracts the highest-priority entries each round (Section 5.1), motivated
 * by Section 3.5 (priority |v (+) Delta - v|, Theorem 4).  The network that
 * predicts a priority is this library's own; the paper has none.
 * A 2-layer network 8 -> 64 (ReLU) -> 1 scores pending vertices for
 * MAITER_SCHED_LEARNED.  Weights are BF16 on the device (an FP32 master copy
 * is kept for training); inputs are rounded to BF16; every product is
 * accumulated in FP32.  Parameters, FP32, in this order: W1[64][8] (row-major),
 * b1[64], w2[64], b2 (641 values).  Features of vertex j (8 values, the
 * library computes them itself when scheduling; maiter_trace records them):
 *   sum ops: log1p(|Delta_j| n), log1p(v_j), log1p(indeg_j), log1p(outdeg_j),
 *            log1p(rounds since j's last update), 1,
 *            log1p(|Delta_j| n / (outdeg_j + 1)), 0
 *   min:     log1p(Delta_j) or 0 if infinite, log1p(v_j) or 0 if infinite,
 *            log1p(indeg_j), log1p(outdeg_j), log1p(rounds since last update),
 *            [Delta_j finite], [v_j finite], 0 */
#define MAITER_MLP_INPUTS 8
#define MAITER_MLP_HIDDEN 64
#define MAITER_MLP_PARAMS 641

/* Creates a network on `device` with seeded He-style random weights.
 * Errors: INVALID_ARG, OOM, CUDA (all mlp calls). */
maiter_status maiter_mlp_create(int device, uint64_t seed, maiter_mlp** out);
maiter_status maiter_mlp_set_params(maiter_mlp* m, const float* params);   /* 641 FP32 */
maiter_status maiter_mlp_get_params(const maiter_mlp* m, float* params);
/* out[i] = network(x[i*8 .. i*8+8)) for i < n (x, out: host or device FP32). */
maiter_status maiter_mlp_forward(const maiter_mlp* m, const float* x, int64_t n, float* out);
/* Gradient of the mean squared error (1/n) sum_i (net(x_i) - y_i)^2 with
 * respect to the 641 parameters (evaluated at the BF16 weights), and the loss. */
maiter_status maiter_mlp_gradients(const maiter_mlp* m, const float* x, const float* y, int64_t n,
                                   float* grad, float* loss);
/* Adam on the GPU: `epochs` passes over (x, y) in seeded random minibatches
 * of `batch` rows; *final_loss = mean squared error of the last minibatch. */
maiter_status maiter_mlp_train(maiter_mlp* m, const float* x, const float* y, int64_t n,
                               int32_t epochs, int32_t batch, float lr, uint64_t seed,
                               float* final_loss);
void maiter_mlp_destroy(maiter_mlp* m);   /* NULL is ignored */

/* Paper: a run as maiter_run (Section 5.2) whose priority fields (Section
 * 5.1) are sampled after every round - the training data of the scorer.
 * Activation trace of a round-engine run (SUM_F64 or MIN_U32; any schedule
 * but LEARNED): after every push of the first max_records rounds, records for
 * each of the num_sample vertices in `sample` its 8 features, Delta, v and the
 * round of its last update (1-based, 0 = never), into host arrays of
 * max_records x num_sample rows.  The run continues to termination; *out
 * receives its result (as maiter_run).  *records = rows written. */
maiter_status maiter_trace(const maiter_graph* g, const maiter_run_params* p,
                           const int32_t* sample, int32_t num_sample, int32_t max_records,
                           float* features, double* delta, double* v, uint32_t* last_update,
                           int32_t* records, maiter_result** out);

/* ------------------------------------------------------------------ batch
 * Many queries - personalised PageRank (+, g = d x / outdeg) and SSSP (min,
 * g = x + w) - over several graphs of uneven size, advanced together round by
 * round in ONE CUDA-graph launch (a WHILE node; no host round trip between
 * rounds).  Each query has its own v and Delta (query-major layout); a round
 * updates every (query, vertex) item of a sparse frontier and appends the
 * receivers whose delta crosses the query's threshold eps_q / n (sum) or whose
 * distance improves (min).  A sum query ends when its frontier is empty, which
 * proves sum |Delta| <= eps_q (every vertex is at or below eps_q / n); a min
 * query ends when no distance can improve (exact).  Personalised PageRank is
 * PageRank (Section 4.2) with Delta1 = (1 - d) / |S| on the seed set S and 0
 * elsewhere (the Rooted PageRank row of Table 1 with damping). */
typedef struct maiter_batch maiter_batch;   /* opaque: query-major state + frontiers */

typedef struct maiter_query {
  int32_t graph;        /* index into the graphs array */
  int32_t op;           /* MAITER_OP_SUM_F64 (PPR) or MAITER_OP_MIN_U32 (SSSP) */
  const int32_t* seeds; /* host array of num_seeds distinct vertex ids */
  int32_t num_seeds;
  int32_t reserved;     /* must be 0 */
  double damping;       /* PPR: d in [0, 1) */
  double eps;           /* PPR: bound on sum_j |Delta_j| at termination (> 0) */
} maiter_query;

typedef struct maiter_batch_params {
  int64_t max_rounds;      /* <= 0 means 1,000,000 */
  void* stream;            /* cudaStream_t; NULL = default stream */
  int32_t cut_large;       /* out-degree from which an item is split into chunks
                              processed by separate CTAs (0 = 1024) */
  int32_t chunk;           /* edges per chunk (0 = 1024, else >= 32) */
  int32_t push_blocks_per_sm;  /* cap on resident push CTAs per SM (0 = occupancy) */
  int32_t flags;           /* MAITER_FLAG_PROFILE_KERNELS or 0 */
  int32_t mode;            /* 0 = dense (default): every query is a round-engine
                              run of its own - all pending vertices per round,
                              exact termination sum |Delta| < eps_q - and one
                              independent branch of the graph, so queries run
                              side by side; 1 = sparse frontiers of (query,
                              vertex) items as described above; 2 = dense with
                              the branches chained: the queries run one after
                              another, in order, inside one graph launch (no
                              host round trip between them); 3 = the
                              personalised-PageRank queries of each graph in
                              groups of up to 64, each group one receive-side
                              run (the receive step of Eq. 5 at the receivers,
                              as MAITER_ENGINE_PULL) over query vectors: a
                              vertex's deltas, states and messages for the
                              group's queries are contiguous, so an in-edge
                              costs one 256-byte read for all of them; FP32
                              deltas and messages, FP64 states and per-query
                              FP64 residuals, each query stopping its count at
                              sum |Delta| < eps_q / 2 (the other half of its
                              bound is left to the FP32 rounding; the group
                              runs until all have); SSSP queries as in mode 0 */
  int32_t reserved;        /* must be 0 */
} maiter_batch_params;

void maiter_batch_params_default(maiter_batch_params* p);

/* Paper: many IterateKernel runs (Section 5.2) of the Rooted PageRank and
 * SSSP rows of Table 1, each with its own state table (Section 5.1).
 * Runs every query to termination.  All graphs must live on one device.  If
 * *out is non-NULL and was returned for the same graphs, query graphs/ops and
 * tuning, it is reused without allocation; otherwise it is (re)built.
 * Errors: INVALID_ARG, OOM (also when a frontier outgrows its bounded
 * capacity), CUDA, NOT_CONVERGED (state readable). */
maiter_status maiter_run_batch(const maiter_graph* const* graphs, int32_t num_graphs,
                               const maiter_query* queries, int32_t num_queries,
                               const maiter_batch_params* p, maiter_batch** out);

/* Paper: the dump of one query's state table v fields (Section 5.1).
 * Copies query `query`'s states (double for PPR, uint32 for SSSP; count = n
 * of its graph) into `out` (host or device).  Errors: INVALID_ARG, CUDA. */
maiter_status maiter_batch_get_state(const maiter_batch* b, int32_t query, void* out,
                                     int64_t count);

/* Paper: the progress estimator of Section 5.1, summed over the queries.
 * Aggregate statistics of the last run (rounds, updates, pushes, time). */
maiter_status maiter_batch_get_stats(const maiter_batch* b, maiter_stats* out);

/* Per query (Section 5.1's per-run termination): the last round in which it
 * still had frontier items.  count must equal the number of queries. */
maiter_status maiter_batch_query_rounds(const maiter_batch* b, int32_t* out, int32_t count);

void maiter_batch_destroy(maiter_batch* b);   /* NULL is ignored */

/* Message of the last failed call on this thread ("" if none).  No paper
 * counterpart (error reporting of this boundary). */
const char* maiter_last_error(void);

/* Library version string (no paper counterpart). */
const char* maiter_version(void);

/* Name (NUL-terminated, truncated to len) and SM count of a device; used to
 * key tuning caches (no paper counterpart).  Errors: INVALID_ARG, CUDA. */
maiter_status maiter_device_info(int device, char* name, int32_t len, int32_t* num_sms);

/* Diagnostic with no paper counterpart (a hardware measurement).
 * The rate at which `device` serves 4- or 8-byte operations at
 * random addresses of a device array of 2^log2_words elements (an integer
 * hash of (thread, iteration) picks each address; a grid of one wave of
 * 256-thread CTAs, 256 operations per thread).  The push kernels issue such
 * operations on Delta_k (k a random vertex id), so this rate at the size of
 * a workload's Delta array is the ceiling their edge loop is held to while
 * the array fits in L2.  The array is allocated, zeroed (all ones for MIN)
 * and freed by the call, on a stream of its own.  *gops receives operations
 * per second / 1e9, best of three launches after one warm-up.
 * Errors: INVALID_ARG (NULL gops, unknown kind, log2_words outside
 * [10, 28], bad device), OOM, CUDA. */
typedef enum {
  MAITER_PROBE_RED_F32 = 0,  /* atomicAdd of a float, result unused (RED) */
  MAITER_PROBE_RED_F64 = 1,  /* atomicAdd of a double, result unused */
  MAITER_PROBE_MIN_U32 = 2,  /* atomicMin of a uint32, result unused */
  MAITER_PROBE_LOAD_32 = 3   /* 4-byte load cached in L2 only */
} maiter_probe_kind;

maiter_status maiter_probe_random_rate(int device, int kind, int log2_words, double* gops);

#ifdef __cplusplus
}
#endif

#endif /* MAITER_H */
