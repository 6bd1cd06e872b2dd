"""Python binding of libmaiter, the B300 (sm_103a) engine for delta-based
accumulative iterative computation (DAIC).

Argument marshalling only: every step of a run executes in the CUDA kernels of
``libmaiter.so`` behind the C ABI declared in ``include/maiter.h``.  There is
no CPU fallback; if the library is missing or no GPU is present, calls raise.

Arrays may be numpy arrays (host memory) or CUDA tensors (device memory, any
object with ``data_ptr()``); the library detects the pointer kind itself.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmaiter.so")

# maiter_status
OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_NOT_CONVERGED = -4
ERR_TIMEOUT = -5
ERR_UNSUPPORTED = -6
_STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED",
                 -5: "TIMEOUT", -6: "UNSUPPORTED"}

# maiter_op / maiter_g / maiter_sched / maiter_engine
OP_SUM_F64, OP_SUM_MIXED, OP_MIN_U32, OP_MIN_F32, OP_MAX_I32 = 0, 1, 2, 3, 4
G_SCALE_BY_SRC, G_ADD_EDGE, G_SCALE_BY_EDGE, G_IDENTITY = 0, 1, 2, 3
SCHED_ALL, SCHED_THRESHOLD, SCHED_TOPFRAC, SCHED_LEARNED, SCHED_BUCKET = 0, 1, 2, 3, 4
MLP_INPUTS, MLP_HIDDEN, MLP_PARAMS = 8, 64, 641
ENGINE_SYNC, ENGINE_ASYNC, ENGINE_BINNED, ENGINE_PULL = 0, 1, 2, 3
FLAG_PROFILE_KERNELS, FLAG_INJECT_STALL = 1, 2
# maiter_batch_params.mode
BATCH_DENSE, BATCH_SPARSE, BATCH_DENSE_CHAINED, BATCH_PULL_GROUPS = 0, 1, 2, 3
# maiter_probe_kind
PROBE_RED_F32, PROBE_RED_F64, PROBE_MIN_U32, PROBE_LOAD_32 = 0, 1, 2, 3

INF32 = 0xFFFFFFFF

_STATE_DTYPE = {OP_SUM_F64: np.float64, OP_SUM_MIXED: np.float64, OP_MIN_U32: np.uint32,
                OP_MIN_F32: np.float32, OP_MAX_I32: np.int32}
_DELTA_DTYPE = {OP_SUM_F64: np.float64, OP_SUM_MIXED: np.float32, OP_MIN_U32: np.uint32,
                OP_MIN_F32: np.float32, OP_MAX_I32: np.int32}
_DELTA0_DTYPE = {OP_SUM_F64: np.float64, OP_SUM_MIXED: np.float64, OP_MIN_U32: np.uint32,
                 OP_MIN_F32: np.float32, OP_MAX_I32: np.int32}
_COEF_DTYPE = {OP_SUM_F64: np.float64, OP_SUM_MIXED: np.float32}


class RunParams(ctypes.Structure):
    """Mirror of ``maiter_run_params``."""
    _fields_ = [
        ("op", ctypes.c_int32), ("g", ctypes.c_int32), ("sched", ctypes.c_int32),
        ("engine", ctypes.c_int32), ("flags", ctypes.c_int32), ("reserved0", ctypes.c_int32),
        ("coef", ctypes.c_void_p), ("damping", ctypes.c_double),
        ("v0", ctypes.c_void_p), ("delta0", ctypes.c_void_p),
        ("source", ctypes.c_int64),
        ("threshold", ctypes.c_double), ("top_frac", ctypes.c_double), ("eps", ctypes.c_double),
        ("mixed_switch", ctypes.c_double),
        ("max_rounds", ctypes.c_int64), ("timeout_ms", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("cut_warp", ctypes.c_int32), ("cut_cta", ctypes.c_int32),
        ("push_blocks_per_sm", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("scorer", ctypes.c_void_p),
    ]


class Stats(ctypes.Structure):
    """Mirror of ``maiter_stats``."""
    _fields_ = [
        ("rounds", ctypes.c_int64), ("activations", ctypes.c_int64),
        ("edge_pushes", ctypes.c_int64), ("residual", ctypes.c_double),
        ("elapsed_ms", ctypes.c_double), ("status", ctypes.c_int32),
        ("converged", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
        ("push_ms", ctypes.c_double), ("scan_ms", ctypes.c_double),
        ("push_launches", ctypes.c_int64), ("scan_launches", ctypes.c_int64),
        ("warm_rounds", ctypes.c_int64), ("warm_activations", ctypes.c_int64),
        ("warm_edge_pushes", ctypes.c_int64),
        ("slots", ctypes.c_int64), ("bin_scatter_ms", ctypes.c_double),
        ("bin_gather_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MaiterError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"maiter {_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib():
    """The loaded libmaiter.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmaiter.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.maiter_graph_create.argtypes = [i64, i64, P, P, P, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p)]
        L.maiter_graph_create.restype = i32
        L.maiter_graph_destroy.argtypes = [P]
        L.maiter_graph_update.argtypes = [P, P, P, P, P]
        L.maiter_graph_update.restype = i32
        L.maiter_run.argtypes = [P, ctypes.POINTER(RunParams), ctypes.POINTER(ctypes.c_void_p)]
        L.maiter_run.restype = i32
        L.maiter_get_state.argtypes = [P, P, i64]
        L.maiter_get_state.restype = i32
        L.maiter_get_delta.argtypes = [P, P, i64]
        L.maiter_get_delta.restype = i32
        L.maiter_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
        L.maiter_get_stats.restype = i32
        L.maiter_result_destroy.argtypes = [P]
        L.maiter_params_default.argtypes = [ctypes.POINTER(RunParams)]
        L.maiter_last_error.restype = ctypes.c_char_p
        L.maiter_version.restype = ctypes.c_char_p
        L.maiter_batch_params_default.argtypes = [ctypes.POINTER(BatchParams)]
        L.maiter_run_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32,
                                       ctypes.POINTER(QuerySpec), i32,
                                       ctypes.POINTER(BatchParams), ctypes.POINTER(ctypes.c_void_p)]
        L.maiter_run_batch.restype = i32
        L.maiter_batch_get_state.argtypes = [P, i32, P, i64]
        L.maiter_batch_get_state.restype = i32
        L.maiter_batch_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
        L.maiter_batch_get_stats.restype = i32
        L.maiter_batch_query_rounds.argtypes = [P, P, i32]
        L.maiter_batch_query_rounds.restype = i32
        L.maiter_batch_destroy.argtypes = [P]
        L.maiter_device_info.argtypes = [ctypes.c_int, ctypes.c_char_p, i32, ctypes.POINTER(i32)]
        L.maiter_device_info.restype = i32
        L.maiter_probe_random_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_double)]
        L.maiter_probe_random_rate.restype = i32
        L.maiter_mlp_create.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]
        L.maiter_mlp_create.restype = i32
        L.maiter_mlp_set_params.argtypes = [P, P]
        L.maiter_mlp_set_params.restype = i32
        L.maiter_mlp_get_params.argtypes = [P, P]
        L.maiter_mlp_get_params.restype = i32
        L.maiter_mlp_forward.argtypes = [P, P, i64, P]
        L.maiter_mlp_forward.restype = i32
        L.maiter_mlp_gradients.argtypes = [P, P, P, i64, P, ctypes.POINTER(ctypes.c_float)]
        L.maiter_mlp_gradients.restype = i32
        L.maiter_mlp_train.argtypes = [P, P, P, i64, i32, i32, ctypes.c_float, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_float)]
        L.maiter_mlp_train.restype = i32
        L.maiter_mlp_destroy.argtypes = [P]
        L.maiter_trace.argtypes = [P, ctypes.POINTER(RunParams), P, i32, i32, P, P, P, P,
                                   ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_void_p)]
        L.maiter_trace.restype = i32
        _lib = L
    return _lib


def last_error() -> str:
    return lib().maiter_last_error().decode()


def _check(status: int, allow=(OK,)):
    if status not in allow:
        raise MaiterError(status, last_error())
    return status


def _addr(x):
    """Raw address of a host numpy array or a device tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported array type {type(x)}")


def _as(x, dtype, n, name):
    """Host arrays are converted to the exact dtype; device tensors are checked."""
    if x is None:
        return None
    if isinstance(x, np.ndarray) or isinstance(x, (list, tuple)):
        a = np.ascontiguousarray(x, dtype=dtype)
        if a.shape != (n,):
            raise ValueError(f"{name} must have shape ({n},)")
        return a
    if hasattr(x, "element_size"):
        if x.numel() != n or x.element_size() != np.dtype(dtype).itemsize:
            raise ValueError(f"{name}: need {n} elements of {np.dtype(dtype).name}")
    return x


def params_default() -> RunParams:
    p = RunParams()
    lib().maiter_params_default(ctypes.byref(p))
    return p


class Graph:
    """``maiter_graph``: a device copy of a CSR of out-edges."""

    def __init__(self, row_ptr, col, w=None, device: int = 0):
        n = int(len(row_ptr)) - 1
        if isinstance(row_ptr, np.ndarray) or isinstance(row_ptr, (list, tuple)):
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        if isinstance(col, np.ndarray) or isinstance(col, (list, tuple)):
            col = np.ascontiguousarray(col, dtype=np.int32)
        if isinstance(w, np.ndarray) and w.dtype == np.float32:
            w = np.ascontiguousarray(w).view(np.uint32)   # float weights travel as their bits
        elif w is not None and (isinstance(w, np.ndarray) or isinstance(w, (list, tuple))):
            w = np.ascontiguousarray(w, dtype=np.uint32)
        m = int(len(col))
        h = ctypes.c_void_p()
        _check(lib().maiter_graph_create(n, m, _addr(row_ptr), _addr(col), _addr(w), device,
                                         ctypes.byref(h)))
        self.handle = h
        self.n, self.m, self.device = n, m, device
        self.weighted = w is not None

    def update(self, row_ptr, col, w=None, stream=None):
        """``maiter_graph_update``: new contents of the same n and m (and
        weights iff the graph has them), copied in place on ``stream``; results
        of this graph stay valid."""
        if isinstance(row_ptr, (np.ndarray, list, tuple)):
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        if isinstance(col, (np.ndarray, list, tuple)):
            col = np.ascontiguousarray(col, dtype=np.int32)
        if isinstance(w, np.ndarray) and w.dtype == np.float32:
            w = np.ascontiguousarray(w).view(np.uint32)
        elif w is not None and isinstance(w, (np.ndarray, list, tuple)):
            w = np.ascontiguousarray(w, dtype=np.uint32)
        if int(len(row_ptr)) - 1 != self.n or int(len(col)) != self.m:
            raise ValueError(f"update needs n = {self.n} and m = {self.m}")
        _check(lib().maiter_graph_update(self.handle, _addr(row_ptr), _addr(col), _addr(w), stream))

    @classmethod
    def from_csr(cls, g, device: int = 0):
        """From any object with row_ptr, col and (optional) w attributes."""
        return cls(g.row_ptr, g.col, getattr(g, "w", None), device)

    def close(self):
        if self.handle:
            lib().maiter_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result:
    """``maiter_result``: device v and Delta of a run, plus its statistics."""

    def __init__(self, handle, graph: Graph, op: int):
        self.handle = handle
        self.graph = graph
        self.op = op

    def state(self, out=None):
        """v (float64 for sums, uint32 for min); into ``out`` if given."""
        if out is None:
            out = np.empty(self.graph.n, dtype=_STATE_DTYPE[self.op])
        _check(lib().maiter_get_state(self.handle, _addr(out), self.graph.n))
        return out

    def delta(self, out=None):
        """Delta (float64 / float32 / uint32 by op); into ``out`` if given."""
        if out is None:
            out = np.empty(self.graph.n, dtype=_DELTA_DTYPE[self.op])
        _check(lib().maiter_get_delta(self.handle, _addr(out), self.graph.n))
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(lib().maiter_get_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self.handle:
            lib().maiter_result_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(graph: Graph, op: int = OP_SUM_F64, *, coef=None, damping: float = 0.8, v0=None,
        delta0=None, source: int = -1, sched: int = SCHED_ALL, threshold: float = 0.0,
        top_frac: float = 0.01, eps: float = 1e-8, mixed_switch: float = 0.01,
        max_rounds: int = 1000000,
        timeout_ms: int = 0, stream=None, engine: int = ENGINE_SYNC, flags: int = 0,
        cut_warp: int = 0, cut_cta: int = 0, push_blocks_per_sm: int = 0, scorer=None,
        edge_coef=None, result: Result | None = None,
        allow_not_converged: bool = False) -> Result:
    """``maiter_run``: one DAIC run to termination.  ``stream`` is a raw
    cudaStream_t handle (e.g. ``torch.cuda.current_stream().cuda_stream``).
    ``edge_coef`` (m float64, CSR order) selects g_{j,k}(x) = c_e x
    (MAITER_G_SCALE_BY_EDGE, e.g. the Jacobi method's -A_kj / A_kk)."""
    n = graph.n
    p = params_default()
    p.op = op
    p.g = {OP_MIN_U32: G_ADD_EDGE, OP_MIN_F32: G_ADD_EDGE, OP_MAX_I32: G_IDENTITY}.get(
        op, G_SCALE_BY_SRC)
    p.sched, p.engine, p.flags = sched, engine, flags
    keep = []
    if edge_coef is not None:
        if coef is not None:
            raise ValueError("give coef (per source) or edge_coef (per edge), not both")
        edge_coef = _as(edge_coef, np.float64, graph.m, "edge_coef")
        keep.append(edge_coef)
        p.g = G_SCALE_BY_EDGE
        p.coef = _addr(edge_coef)
    if coef is not None:
        coef = _as(coef, _COEF_DTYPE[op], n, "coef")
        keep.append(coef)
        p.coef = _addr(coef)
    p.damping = damping
    if v0 is not None:
        v0 = _as(v0, _STATE_DTYPE[op], n, "v0")
        keep.append(v0)
        p.v0 = _addr(v0)
    if delta0 is not None:
        delta0 = _as(delta0, _DELTA0_DTYPE[op], n, "delta0")
        keep.append(delta0)
        p.delta0 = _addr(delta0)
    p.source = source
    p.threshold, p.top_frac, p.eps = threshold, top_frac, eps
    p.mixed_switch = mixed_switch
    p.cut_warp, p.cut_cta, p.push_blocks_per_sm = cut_warp, cut_cta, push_blocks_per_sm
    p.scorer = scorer.handle.value if scorer is not None else None
    p.max_rounds, p.timeout_ms = max_rounds, timeout_ms
    p.stream = stream
    h = ctypes.c_void_p(result.handle.value if result is not None else None)
    # both leave a readable, resumable state
    allow = (OK, ERR_NOT_CONVERGED, ERR_TIMEOUT) if allow_not_converged else (OK,)
    st = lib().maiter_run(graph.handle, ctypes.byref(p), ctypes.byref(h))
    if result is None and h.value:
        result = Result(h, graph, op)
    _check(st, allow)
    return result


class QuerySpec(ctypes.Structure):
    """Mirror of ``maiter_query``."""
    _fields_ = [("graph", ctypes.c_int32), ("op", ctypes.c_int32), ("seeds", ctypes.c_void_p),
                ("num_seeds", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("damping", ctypes.c_double), ("eps", ctypes.c_double)]


class BatchParams(ctypes.Structure):
    """Mirror of ``maiter_batch_params``."""
    _fields_ = [("max_rounds", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("cut_large", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("push_blocks_per_sm", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Batch:
    """``maiter_batch``: the query-major states of a batched run."""

    def __init__(self, handle, graphs, queries):
        self.handle = handle
        self.graphs = graphs
        self.queries = queries

    def state(self, q: int, out=None):
        op, g = self.queries[q][0], self.graphs[self.queries[q][1]]
        if out is None:
            out = np.empty(g.n, dtype=np.uint32 if op == OP_MIN_U32 else np.float64)
        _check(lib().maiter_batch_get_state(self.handle, q, _addr(out), g.n))
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(lib().maiter_batch_get_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def query_rounds(self) -> np.ndarray:
        out = np.empty(len(self.queries), dtype=np.int32)
        _check(lib().maiter_batch_query_rounds(self.handle, _addr(out), len(self.queries)))
        return out

    def close(self):
        if self.handle:
            lib().maiter_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_batch(graphs, queries, *, max_rounds: int = 1000000, stream=None, cut_large: int = 0,
              chunk: int = 0, push_blocks_per_sm: int = 0, flags: int = 0, mode: int = 0,
              batch: Batch | None = None) -> Batch:
    """``maiter_run_batch``.  ``queries`` is a list of dicts with keys op
    (OP_SUM_F64 or OP_MIN_U32), graph (index), seeds (ids), and for PageRank
    damping and eps.  ``mode``: BATCH_DENSE (each query a round-engine run,
    all side by side in one graph launch), BATCH_SPARSE ((query, vertex)
    frontiers), BATCH_DENSE_CHAINED (the dense runs one after another, in
    order, in one graph launch) or BATCH_PULL_GROUPS (the PageRank queries of
    a graph 64 at a time as one receive-side run over query vectors, FP32
    deltas and FP64 state; SSSP queries as in BATCH_DENSE)."""
    G = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    Q = (QuerySpec * len(queries))()
    keep = []
    for i, q in enumerate(queries):
        seeds = np.ascontiguousarray(q["seeds"], dtype=np.int32)
        keep.append(seeds)
        Q[i].graph, Q[i].op = int(q["graph"]), int(q["op"])
        Q[i].seeds, Q[i].num_seeds = seeds.ctypes.data, int(seeds.shape[0])
        Q[i].damping = float(q.get("damping", 0.8))
        Q[i].eps = float(q.get("eps", 1e-6))
    p = BatchParams()
    lib().maiter_batch_params_default(ctypes.byref(p))
    p.max_rounds, p.stream = max_rounds, stream
    p.cut_large, p.chunk, p.push_blocks_per_sm, p.flags = cut_large, chunk, push_blocks_per_sm, flags
    p.mode = mode
    h = ctypes.c_void_p(batch.handle.value if batch is not None else None)
    st = lib().maiter_run_batch(G, len(graphs), Q, len(queries), ctypes.byref(p), ctypes.byref(h))
    if batch is None and h.value:
        batch = Batch(h, list(graphs), [(int(q["op"]), int(q["graph"])) for q in queries])
    elif batch is not None:
        batch.queries = [(int(q["op"]), int(q["graph"])) for q in queries]
    _check(st)
    return batch


class MLP:
    """``maiter_mlp``: the learned priority scorer (8 -> 64 -> 1, BF16 weights)."""

    def __init__(self, device: int = 0, seed: int = 0, params=None):
        h = ctypes.c_void_p()
        _check(lib().maiter_mlp_create(device, seed, ctypes.byref(h)))
        self.handle = h
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (MLP_PARAMS,):
            raise ValueError(f"need {MLP_PARAMS} parameters")
        _check(lib().maiter_mlp_set_params(self.handle, _addr(p)))

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(lib().maiter_mlp_get_params(self.handle, _addr(out)))
        return out

    def forward(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, MLP_INPUTS)
        out = np.empty(x.shape[0], dtype=np.float32)
        _check(lib().maiter_mlp_forward(self.handle, _addr(x), x.shape[0], _addr(out)))
        return out

    def gradients(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, MLP_INPUTS)
        y = np.ascontiguousarray(y, dtype=np.float32)
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        _check(lib().maiter_mlp_gradients(self.handle, _addr(x), _addr(y), x.shape[0], _addr(g),
                                          ctypes.byref(loss)))
        return g, loss.value

    def train(self, x, y, epochs: int = 10, batch: int = 1024, lr: float = 1e-3, seed: int = 0):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, MLP_INPUTS)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        _check(lib().maiter_mlp_train(self.handle, _addr(x), _addr(y), x.shape[0], epochs, batch,
                                      lr, seed, ctypes.byref(loss)))
        return loss.value

    def close(self):
        if self.handle:
            lib().maiter_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace(graph: Graph, op: int, sample, max_records: int, **run_kwargs):
    """``maiter_trace``: features, deltas, states and last-update rounds of the
    sampled vertices after every push of the first ``max_records`` rounds of a
    round-engine run.  Returns (dict of arrays shaped [records, samples, ...],
    the run's Result)."""
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    ns = sample.shape[0]
    feat = np.empty((max_records, ns, MLP_INPUTS), dtype=np.float32)
    dl = np.empty((max_records, ns), dtype=np.float64)
    vs = np.empty((max_records, ns), dtype=np.float64)
    la = np.empty((max_records, ns), dtype=np.uint32)
    p = params_default()
    p.op = op
    p.g = G_ADD_EDGE if op in (OP_MIN_U32, OP_MIN_F32) else G_SCALE_BY_SRC
    for k, v in run_kwargs.items():
        setattr(p, k, v)
    rec = ctypes.c_int32(0)
    h = ctypes.c_void_p()
    st = lib().maiter_trace(graph.handle, ctypes.byref(p), _addr(sample), ns, max_records,
                            _addr(feat), _addr(dl), _addr(vs), _addr(la), ctypes.byref(rec),
                            ctypes.byref(h))
    res = Result(h, graph, op) if h.value else None
    _check(st, (OK, ERR_NOT_CONVERGED))
    r = rec.value
    return dict(features=feat[:r], delta=dl[:r], v=vs[:r], last_update=la[:r]), res


def device_info(device: int = 0) -> tuple[str, int]:
    """(name, SM count) of a CUDA device, from ``maiter_device_info``."""
    buf = ctypes.create_string_buffer(256)
    sms = ctypes.c_int32(0)
    _check(lib().maiter_device_info(device, buf, 256, ctypes.byref(sms)))
    return buf.value.decode(), sms.value


def probe_random_rate(kind: int, log2_words: int, device: int = 0) -> float:
    """Random-address operations per second / 1e9 that the device sustains
    into an array of 2**log2_words elements (``maiter_probe_random_rate``)."""
    out = ctypes.c_double(0.0)
    _check(lib().maiter_probe_random_rate(device, kind, log2_words, ctypes.byref(out)))
    return out.value


def version() -> str:
    return lib().maiter_version().decode()
