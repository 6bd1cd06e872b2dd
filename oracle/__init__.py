"""CPU oracle for delta-based accumulative iterative computation (DAIC).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the bench's
CPU-baseline leg are the only callers.  The product path (the CUDA library and
its binding) never imports this package, and this package never imports the
product.  Floating point is FP64 throughout.

Layout: ``oracle.c`` (plain C, built into ``liboracle.so``) holds the loops;
this module wraps them and adds the few steps that are a library primitive
(a dense solve, a sort).  What each function follows is cited in its
docstring.  The paper is "Maiter: An Asynchronous Graph Processing Framework
for Delta-based Accumulative Iterative Computation" (Zhang, Gao, Gao, Wang).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

INF32 = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P, i64, d, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.or_linear_power.argtypes = [i64, P, P, P, P, d, i64, P]
        lib.or_linear_power.restype = i64
        lib.or_linear_residual.argtypes = [i64, P, P, P, P, P, P]
        lib.or_daic_sum.argtypes = [i64, P, P, P, P, P, i32, d, i64, P, P, P]
        lib.or_daic_sum.restype = i32
        lib.or_daic_min.argtypes = [i64, P, P, P, P, P, i32, i64, P, P]
        lib.or_daic_min.restype = i32
        lib.or_dijkstra.argtypes = [i64, P, P, P, ctypes.c_int32, P]
        lib.or_dijkstra.restype = i32
        lib.or_bellman_ford.argtypes = [i64, P, P, P, ctypes.c_int32, P]
        lib.or_linear_power_edges.argtypes = [i64, P, P, P, P, d, i64, P]
        lib.or_linear_power_edges.restype = i64
        lib.or_max_reach.argtypes = [i64, P, P, P]
        lib.or_max_reach.restype = i32
        lib.or_union_find_max.argtypes = [i64, P, P, P]
        lib.or_union_find_max.restype = i32
        lib.or_dijkstra_f32.argtypes = [i64, P, P, P, ctypes.c_int32, P]
        lib.or_dijkstra_f32.restype = i32
        lib.or_bellman_ford_f32.argtypes = [i64, P, P, P, ctypes.c_int32, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    return (np.ascontiguousarray(g.row_ptr, dtype=np.int64),
            np.ascontiguousarray(g.col, dtype=np.int32))


# ------------------------------------------------------------ PageRank family

def pagerank_coef(g, d: float) -> np.ndarray:
    """g_{i,j}(x) = d * x / |N(i)| with |N(i)| the SENDER's out-degree
    (PageRank subsection of Section 4.2 and the derivation in Section 3.1;
    Table 1 prints |N(j)|, read as a typo).  Multi-edges count with
    multiplicity.  Vertices without out-edges get coefficient 0 (they send
    nothing)."""
    deg = np.diff(np.asarray(g.row_ptr, dtype=np.int64)).astype(np.float64)
    coef = np.zeros(g.n, dtype=np.float64)
    nz = deg > 0
    coef[nz] = d / deg[nz]
    return coef


def pagerank_c(n: int, d: float, seeds=None) -> np.ndarray:
    """Constant term c_j of Eq. 3: 1-d for PageRank (Eq. 2); for personalised
    PageRank, (1-d)/|S| on the seed set S and 0 elsewhere."""
    if seeds is None:
        return np.full(n, 1.0 - d)
    c = np.zeros(n)
    seeds = np.asarray(seeds, dtype=np.int64)
    c[seeds] += (1.0 - d) / len(seeds)
    return c


def linear_power(g, coef, c, tol: float = None, max_iter: int = 100000):
    """Fixed point of v = c + P^T v by synchronous iteration from v = 0
    (Section 2, Eq. 1; Eq. 2 for PageRank).  P[i, k] = coef[i] per edge i->k.
    tol defaults to 1e-13 * ||c||_1 on the L1 change.  Returns (v, iterations)."""
    rp, col = _csr(g)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    if tol is None:
        tol = 1e-13 * max(float(np.abs(c).sum()), 1e-300)
    v = np.empty(g.n)
    it = _load().or_linear_power(g.n, _p(rp), _p(col), _p(coef), _p(c), tol, max_iter, _p(v))
    if it < 0:
        raise MemoryError("or_linear_power")
    return v, int(it)


def pagerank(g, d: float = 0.8, seeds=None, tol: float = None):
    """PageRank (Eq. 2) or personalised PageRank fixed point, FP64."""
    v, _ = linear_power(g, pagerank_coef(g, d), pagerank_c(g.n, d, seeds), tol)
    return v


def linear_residual(g, coef, c, v) -> np.ndarray:
    """r = c + P^T v - v: one application of the update of Eq. 1 minus v.
    As (I - P^T)(v* - v) = r and ||(I - P^T)^{-1}||_1 <= 1/(1 - max_i coef_i
    outdeg_i), ||v* - v||_1 <= ||r||_1 / (1 - d) for PageRank."""
    rp, col = _csr(g)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    r = np.empty(g.n)
    _load().or_linear_residual(g.n, _p(rp), _p(col), _p(coef), _p(c), _p(v), _p(r))
    return r


def dense_solve(g, coef, c) -> np.ndarray:
    """Direct solve of (I - P^T) v = c with LU and partial pivoting (library
    routine) on a dense matrix; for n <= 2000.  Same fixed point as Eq. 1."""
    n = g.n
    if n > 2000:
        raise ValueError("dense_solve is for n <= 2000")
    A = np.eye(n)
    rp = np.asarray(g.row_ptr)
    col = np.asarray(g.col)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            A[col[e], i] -= coef[i]
    return np.linalg.solve(A, np.asarray(c, dtype=np.float64))


def katz(g, beta: float, s: int) -> np.ndarray:
    """Katz metric from s (Table 1): x = sum_{k >= 0} (beta A^T)^k e_s, the fixed
    point of x = e_s + beta A^T x (A the 0/1 adjacency, multi-edges counted),
    by the synchronous iteration of Eq. 1."""
    c = np.zeros(g.n)
    c[s] = 1.0
    v, _ = linear_power(g, np.full(g.n, float(beta)), c)
    return v


def linear_power_edges(g, ecoef, c, tol: float = None, max_iter: int = 100000):
    """Fixed point of v = c + M v with M[k, j] = sum of ecoef over the edges
    j -> k, by synchronous iteration from v = 0 (the Jacobi row of Table 1).
    tol defaults to 1e-13 * ||c||_1 on the L1 change.  Returns (v, iterations)."""
    rp, col = _csr(g)
    ecoef = np.ascontiguousarray(ecoef, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    if tol is None:
        tol = 1e-13 * max(float(np.abs(c).sum()), 1e-300)
    v = np.empty(g.n)
    it = _load().or_linear_power_edges(g.n, _p(rp), _p(col), _p(ecoef), _p(c), tol, max_iter, _p(v))
    if it < 0:
        raise MemoryError("or_linear_power_edges")
    return v, int(it)


def solve_linear_system(A, b) -> np.ndarray:
    """x with A x = b (dense LU with partial pivoting, library routine): what
    the Jacobi method of Section 4.3 converges to."""
    return np.linalg.solve(np.asarray(A, dtype=np.float64), np.asarray(b, dtype=np.float64))


def daic_sum(g, coef, v0, delta0, sched: str = "roundrobin", eps: float = 1e-12,
             max_updates: int = 1 << 62):
    """Asynchronous DAIC with + (Eq. 5) from (v0, delta0), serial.
    sched: "roundrobin" (table order, Section 5.1) or "priority" (largest
    |Delta_j| first, Section 3.5).  Returns dict with v, delta, leak (delta
    folded at vertices without out-edges), updates, pushes, converged."""
    rp, col = _csr(g)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    v = np.array(v0, dtype=np.float64, copy=True)
    delta = np.array(delta0, dtype=np.float64, copy=True)
    leak = ctypes.c_double(0.0)
    upd = ctypes.c_int64(0)
    psh = ctypes.c_int64(0)
    s = {"roundrobin": 0, "priority": 1}[sched]
    rc = _load().or_daic_sum(g.n, _p(rp), _p(col), _p(coef), _p(v), _p(delta), s, eps,
                             max_updates, ctypes.byref(leak), ctypes.byref(upd),
                             ctypes.byref(psh))
    if rc < 0:
        raise MemoryError("or_daic_sum")
    return dict(v=v, delta=delta, leak=leak.value, updates=upd.value, pushes=psh.value,
                converged=(rc == 0))


def pagerank_mass_invariant(v, delta, leak, n, d) -> float:
    """Returns sum(v) + (sum(delta) + d*leak)/(1-d) - n, which is 0 at every
    moment of a PageRank DAIC run started from v0 = 0, Delta1 = 1-d: a fold of
    delta at a vertex with out-edges moves delta into v and d*delta back into
    the deltas; at a vertex without out-edges the delta stays in v (leak).
    With no such vertices this is the paper's statement that sum_j R_j rises
    from 0.2 N to N (Section 6.4, d = 0.8)."""
    return float(np.sum(v) + (np.sum(delta) + d * leak) / (1.0 - d) - n)


# ------------------------------------------------------------------- SSSP

def sssp_init(n: int, source: int):
    """SSSP row of Table 1: v0 = inf everywhere, Delta1 = 0 at the source and
    inf elsewhere."""
    v = np.full(n, INF32, dtype=np.uint32)
    delta = np.full(n, INF32, dtype=np.uint32)
    delta[source] = 0
    return v, delta


def dijkstra(g, source: int) -> np.ndarray:
    """Shortest distances from ``source`` (uint32, INF32 if unreachable)."""
    rp, col = _csr(g)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    out = np.empty(g.n, dtype=np.uint32)
    rc = _load().or_dijkstra(g.n, _p(rp), _p(col), _p(w), int(source), _p(out))
    if rc == -1:
        raise MemoryError("or_dijkstra")
    if rc == -2:
        raise OverflowError("a shortest distance does not fit in 32 bits")
    return out


def bellman_ford(g, source: int) -> np.ndarray:
    rp, col = _csr(g)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    out = np.empty(g.n, dtype=np.uint32)
    _load().or_bellman_ford(g.n, _p(rp), _p(col), _p(w), int(source), _p(out))
    return out


def max_reach_labels(g) -> np.ndarray:
    """Connected-components labels of Table 1 (max): for every vertex the
    largest id among the vertices that reach it, itself included (int32)."""
    rp, col = _csr(g)
    out = np.empty(g.n, dtype=np.int32)
    if _load().or_max_reach(g.n, _p(rp), _p(col), _p(out)) != 0:
        raise MemoryError("or_max_reach")
    return out


def component_labels(g) -> np.ndarray:
    """Components of the graph taken as undirected (union-find), each vertex
    labelled with its component's largest id (int32)."""
    rp, col = _csr(g)
    out = np.empty(g.n, dtype=np.int32)
    if _load().or_union_find_max(g.n, _p(rp), _p(col), _p(out)) != 0:
        raise MemoryError("or_union_find_max")
    return out


def _float_weights(g) -> np.ndarray:
    w = np.asarray(g.w)
    return np.ascontiguousarray(w.view(np.float32) if w.dtype == np.uint32 else w,
                                dtype=np.float32)


def dijkstra_f32(g, source: int) -> np.ndarray:
    """Shortest distances over float weights (float32, +inf if unreachable),
    every distance formed as fl(d + w) in single precision.  ``g.w`` holds the
    weights as float32 or as their uint32 bit patterns."""
    rp, col = _csr(g)
    w = _float_weights(g)
    out = np.empty(g.n, dtype=np.float32)
    if _load().or_dijkstra_f32(g.n, _p(rp), _p(col), _p(w), int(source), _p(out)) != 0:
        raise MemoryError("or_dijkstra_f32")
    return out


def bellman_ford_f32(g, source: int) -> np.ndarray:
    rp, col = _csr(g)
    w = _float_weights(g)
    out = np.empty(g.n, dtype=np.float32)
    _load().or_bellman_ford_f32(g.n, _p(rp), _p(col), _p(w), int(source), _p(out))
    return out


def daic_min(g, v0, delta0, sched: str = "roundrobin", max_updates: int = 1 << 62):
    """Asynchronous DAIC with min and g(x) = x + w (SSSP row of Table 1)."""
    rp, col = _csr(g)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    v = np.array(v0, dtype=np.uint32, copy=True)
    delta = np.array(delta0, dtype=np.uint32, copy=True)
    upd = ctypes.c_int64(0)
    psh = ctypes.c_int64(0)
    s = {"roundrobin": 0, "priority": 1}[sched]
    rc = _load().or_daic_min(g.n, _p(rp), _p(col), _p(w), _p(v), _p(delta), s, max_updates,
                             ctypes.byref(upd), ctypes.byref(psh))
    if rc < 0:
        raise MemoryError("or_daic_min")
    return dict(v=v, delta=delta, updates=upd.value, pushes=psh.value, converged=(rc == 0))


# ------------------------------------------------------------- scheduling

def priority_key_f32(delta) -> np.ndarray:
    """Scheduling priority |v_j + Delta_j - v_j| = |Delta_j| for + (Section 3.5),
    rounded to FP32 (the precision both sides take the selection decision in)."""
    return np.abs(np.asarray(delta, dtype=np.float64)).astype(np.float32)


def topfrac_select(delta, q: float) -> np.ndarray:
    """Priority-queue extraction of Section 5.1: among vertices with a non-zero
    priority, take the top fraction q.  Reading: k = ceil(q * nnz) (at least 1),
    threshold = the k-th largest FP32 key, and every vertex whose key is >= the
    threshold is taken, ties included.  Returns the sorted selected ids."""
    key = priority_key_f32(delta)
    nz = np.nonzero(key > 0)[0]
    if nz.size == 0:
        return nz.astype(np.int64)
    k = max(1, int(math.ceil(q * nz.size)))
    kth = np.sort(key[nz])[::-1][k - 1]
    return np.nonzero(key >= kth)[0].astype(np.int64)


def relative_error(v, vstar) -> float:
    """max_j |v_j - v*_j| / max_j |v*_j| (norm-wise relative error)."""
    v = np.asarray(v, dtype=np.float64)
    vstar = np.asarray(vstar, dtype=np.float64)
    return float(np.max(np.abs(v - vstar)) / max(np.max(np.abs(vstar)), 1e-300))
