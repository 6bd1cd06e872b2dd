"""Seeded synthetic graph inputs shared by the oracle, the tests and the bench.

Holds no arithmetic of the delta-propagation method: it draws R-MAT edges,
weights, permutations and query seeds from a counter-based SplitMix64 stream
(see ``rmat.c``) and lays edges out as a CSR of out-edges.  Both the CPU oracle
and the CUDA path consume the identical arrays, so input preparation can never
cause a parity mismatch.

Workload recipe (the paper's evaluation uses the Google web graph and
log-normal synthetic graphs, Section 6.1; seeded R-MAT stands in for them):

* R-MAT quadrant probabilities (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), no noise;
* n = 2**scale vertices, m = edge_factor * n directed edges, exactly;
* vertex ids relabelled by a seeded permutation; multi-edges, self-loops and
  dangling vertices kept;
* SSSP weights uniform integers in [1, 255];
* default graph seed = 171005785 + scale.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgraphgen.so")
_lib = None

DEFAULT_SEED_BASE = 171005785


def build(force: bool = False) -> str:
    """Compile ``rmat.c`` into ``libgraphgen.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "rmat.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64, u64, d = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gg_permutation.argtypes = [i64, u64, P]
        lib.gg_rmat_edges.argtypes = [ctypes.c_int, i64, u64, d, d, d, P, P]
        lib.gg_uniform_weights.argtypes = [i64, u64, ctypes.c_uint32, ctypes.c_uint32, P]
        lib.gg_build_csr.argtypes = [i64, i64, P, P, P, P, P, P, P]
        lib.gg_build_csr.restype = ctypes.c_int
        lib.gg_pick.argtypes = [i64, P, i64, u64, u64, P]
        lib.gg_pick.restype = ctypes.c_int
        lib.gg_uniform01.argtypes = [i64, u64, u64, P]
        lib.gg_draw.argtypes = [u64, u64]
        lib.gg_draw.restype = u64
        lib.gg_lognormal_indegrees.argtypes = [i64, u64, d, d, i64, P]
        lib.gg_lognormal_indegrees.restype = i64
        lib.gg_lognormal_edges.argtypes = [i64, u64, P, P, P]
        lib.gg_lognormal_weights.argtypes = [i64, u64, d, d, P]
        lib.gg_stream_key.argtypes = [u64, u64]
        lib.gg_stream_key.restype = u64
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class CSRGraph:
    """Out-edge CSR: targets of vertex j are col[row_ptr[j]:row_ptr[j+1]]."""
    n: int
    m: int
    row_ptr: np.ndarray            # int64[n+1]
    col: np.ndarray                # int32[m]
    w: np.ndarray | None = None    # uint32[m] or None
    name: str = ""

    @property
    def outdeg(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def csr_from_edges(n, src, dst, w=None, perm=None, name="") -> CSRGraph:
    """CSR (canonical: each row's (target, weight) pairs sorted) from an edge list."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    if dst.shape[0] != m:
        raise ValueError("src and dst lengths differ")
    if m and (src.min() < 0 or src.max() >= n or dst.min() < 0 or dst.max() >= n):
        raise ValueError("edge endpoint out of range")
    win = None if w is None else np.ascontiguousarray(w, dtype=np.uint32)
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(m, 0), dtype=np.int32)
    wout = None if win is None else np.empty(m, dtype=np.uint32)
    if lib.gg_build_csr(n, m, _ptr(src), _ptr(dst), _ptr(win), _ptr(pm), _ptr(row_ptr),
                        _ptr(col), _ptr(wout)) != 0:
        raise MemoryError("gg_build_csr: allocation failed")
    return CSRGraph(n, m, row_ptr, col, wout, name)


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _load().gg_permutation(n, seed, _ptr(out))
    return out


def rmat_edges(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19):
    """Raw R-MAT edge list (before relabelling): (src, dst) int32 arrays."""
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    _load().gg_rmat_edges(scale, m, seed, a, b, c, _ptr(src), _ptr(dst))
    return src, dst


def uniform_weights(m: int, seed: int, lo: int = 1, hi: int = 255) -> np.ndarray:
    w = np.empty(m, dtype=np.uint32)
    _load().gg_uniform_weights(m, seed, lo, hi, _ptr(w))
    return w


def rmat(scale: int, edge_factor: int, seed: int | None = None, weights: bool = False,
         permute: bool = True, a=0.57, b=0.19, c=0.19) -> CSRGraph:
    """Seeded R-MAT graph as a canonical CSR of out-edges."""
    if seed is None:
        seed = DEFAULT_SEED_BASE + scale
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, seed, a, b, c)
    w = uniform_weights(src.shape[0], seed) if weights else None
    perm = permutation(n, seed) if permute else None
    return csr_from_edges(n, src, dst, w, perm, name=f"rmat{scale}-ef{edge_factor}-s{seed}")


def lognormal(n: int, seed: int | None = None, mu: float = -0.5, sigma: float = 2.3,
              weights: bool = False, wmu: float = 0.0, wsigma: float = 1.0,
              cap: int | None = None) -> CSRGraph:
    """The paper's synthetic graphs (Section 6.1): each vertex's in-degree is
    round(exp(N(mu, sigma))) (capped at ``cap``, default n), its in-neighbours
    uniform vertex ids drawn with replacement.  With ``weights``, each edge
    gets an IEEE single weight exp(N(wmu, wsigma)) (the paper's SSSP graphs use
    (0, 1)), stored in ``w`` as its uint32 bit pattern (``float_weights(g)``
    reads it back).  Canonical CSR of out-edges, no relabelling."""
    lib = _load()
    if seed is None:
        seed = DEFAULT_SEED_BASE + 2000 + int(np.log2(max(n, 1)))
    deg = np.empty(n, dtype=np.int64)
    m = int(lib.gg_lognormal_indegrees(n, seed, mu, sigma, int(cap if cap is not None else n),
                                       _ptr(deg)))
    offs = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=offs[1:])
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.gg_lognormal_edges(n, seed, _ptr(offs), _ptr(src), _ptr(dst))
    w = None
    if weights:
        w = np.empty(m, dtype=np.uint32)
        lib.gg_lognormal_weights(m, seed, wmu, wsigma, _ptr(w))
    return csr_from_edges(n, src, dst, w, None, name=f"lognormal-n{n}-s{seed}")


def symmetrize(g: CSRGraph) -> CSRGraph:
    """The graph with every edge also reversed (an undirected graph as a
    directed one; weights, if any, copied to the reverse edge)."""
    src = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.row_ptr))
    w = None if g.w is None else np.concatenate([g.w, g.w])
    return csr_from_edges(g.n, np.concatenate([src, g.col]), np.concatenate([g.col, src]), w,
                          name=g.name + "-sym")


def float_weights(g: CSRGraph) -> np.ndarray:
    """The float32 view of a graph whose ``w`` holds IEEE single bit patterns."""
    return g.w.view(np.float32)


def pick(candidates: np.ndarray, k: int, seed: int, stream: int = 0) -> np.ndarray:
    """k distinct elements of ``candidates``, seeded (partial Fisher-Yates)."""
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    out = np.empty(k, dtype=np.int32)
    if _load().gg_pick(cand.shape[0], _ptr(cand), k, seed, stream, _ptr(out)) != 0:
        raise ValueError("cannot pick %d of %d candidates" % (k, cand.shape[0]))
    return out


def uniform01(count: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().gg_uniform01(count, seed, stream, _ptr(out))
    return out


def sssp_sources(g: CSRGraph, k: int, seed: int | None = None) -> np.ndarray:
    """k distinct SSSP sources among vertices whose out-degree is at least the
    mean degree m/n (such vertices sit in the giant out-component of an R-MAT
    graph with overwhelming probability)."""
    if seed is None:
        seed = DEFAULT_SEED_BASE + 1
    mean = max(1, g.m // max(g.n, 1))
    cand = np.nonzero(g.outdeg >= mean)[0].astype(np.int32)
    return pick(cand, k, seed, stream=1)


def ppr_seed_sets(n: int, count: int, seed: int, max_size: int = 64) -> list[np.ndarray]:
    """Seed sets for personalised PageRank queries: sizes round(exp(U(0, ln max_size)))
    (log-uniform on [1, max_size]), members distinct and uniform over [0, n)."""
    u = uniform01(count, seed, stream=2)
    sizes = np.clip(np.rint(np.exp(u * np.log(max_size))).astype(np.int64), 1, max_size)
    everyone = np.arange(n, dtype=np.int32)
    return [np.sort(pick(everyone, int(s), seed, stream=100 + q)) for q, s in enumerate(sizes)]


def small_graph(n: int, edges, weights=None, name="") -> CSRGraph:
    """CSR from an explicit edge list (tests and worked examples)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = None if weights is None else np.asarray(weights, dtype=np.uint32)
    return csr_from_edges(n, e[:, 0], e[:, 1], w, None, name=name)


def random_graph(n: int, m: int, seed: int, weights: bool = False, wlo=1, whi=255) -> CSRGraph:
    """Uniform random multigraph with m directed edges (tests)."""
    u = uniform01(2 * m, seed, stream=3)
    src = np.minimum((u[:m] * n).astype(np.int64), n - 1)
    dst = np.minimum((u[m:] * n).astype(np.int64), n - 1)
    w = uniform_weights(m, seed, wlo, whi) if weights else None
    return csr_from_edges(n, src, dst, w, None, name=f"uniform{n}x{m}-s{seed}")
