"""Autotuner for the engine's launch parameters.

Picks, per (GPU, graph signature, workload kind), the degree cut-offs, the
chunk size of high-degree vertices and the number of resident push CTAs per
SM by timing each candidate on the workload (or a sample of it) with the
engine's own event timing, and caches the winner in a JSON file so later runs
start tuned.  Every candidate runs the same kernels to the same termination
test, so tuning never changes a result beyond floating-point summation order.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "maiter_b300_autotune.json")

RUN_SPACE = {
    "cut_warp": [16, 32, 64],
    "cut_cta": [256, 512, 2048],
    "push_blocks_per_sm": [0, 4],
}
BATCH_SPACE = {
    "mode": [0, 1],                 # dense per-query loops / sparse frontiers
    "cut_large": [256, 1024, 4096],
    "chunk": [512, 1024, 2048],
    "push_blocks_per_sm": [0, 4],
}


def candidates(space: dict) -> list[dict]:
    """Cartesian product of a parameter space, in a fixed order."""
    keys = sorted(space)
    out = []
    for values in itertools.product(*(space[k] for k in keys)):
        c = dict(zip(keys, values))
        if "cut_warp" in c and c["cut_warp"] > c["cut_cta"]:
            continue
        # the dense batch mode ignores the sparse mode's chunking parameters
        if c.get("mode") == 0 and (c.get("cut_large") != 1024 or c.get("chunk") != 1024):
            continue
        out.append(c)
    return out


def graph_signature(*graphs) -> str:
    """Stable signature of graph shapes: n, m and the out-degree histogram in
    powers of two (what the cut-offs depend on), not the edges themselves."""
    import numpy as np
    h = hashlib.sha256()
    for g in graphs:
        deg = np.diff(np.asarray(g.row_ptr, dtype=np.int64))
        hist = np.bincount(np.floor(np.log2(np.maximum(deg, 1))).astype(np.int64), minlength=32)
        h.update(np.array([g.n, g.m], dtype=np.int64).tobytes())
        h.update(hist.astype(np.int64).tobytes())
    return h.hexdigest()[:16]


class Cache:
    """JSON cache of tuned configurations keyed by a string."""

    def __init__(self, path: str | None = DEFAULT_CACHE):
        self.path = path
        self.data = {}
        if path and os.path.exists(path):
            try:
                with open(path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key):
        return self.data.get(key)

    def put(self, key, value):
        self.data[key] = value
        if self.path:
            os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def search(space: dict, measure, repeats: int = 2) -> tuple[dict, list]:
    """Times every candidate with ``measure(config) -> ms`` (best of
    ``repeats`` after one warm call) and returns (best config, all timings)."""
    timings = []
    for c in candidates(space):
        measure(c)
        ms = min(measure(c) for _ in range(repeats))
        timings.append((ms, c))
    timings.sort(key=lambda t: t[0])
    return dict(timings[0][1]), [(round(t, 4), c) for t, c in timings]


def tune_run(mt, graph_csr, G, run_kwargs: dict, cache: Cache | None = None,
             space: dict | None = None, device: int = 0) -> dict:
    """Tuned cut_warp / cut_cta / push_blocks_per_sm for ``mt.run(G, **run_kwargs)``."""
    space = space or RUN_SPACE
    name, sms = mt.device_info(device)
    kind = json.dumps({k: v for k, v in sorted(run_kwargs.items()) if k in
                       ("op", "sched", "engine", "top_frac")})
    key = f"run|{name}|{sms}|{graph_signature(graph_csr)}|{kind}"
    if cache is not None and cache.get(key):
        return dict(cache.get(key)["config"])
    result = [None]

    def measure(c):
        result[0] = mt.run(G, result=result[0], **run_kwargs, **c)
        return result[0].stats()["elapsed_ms"]

    best, timings = search(space, measure)
    if cache is not None:
        cache.put(key, {"config": best, "timings": timings[:5]})
    return best


def tune_batch(mt, graph_csrs, G, queries, cache: Cache | None = None,
               space: dict | None = None, sample: int = 64, device: int = 0) -> dict:
    """Tuned cut_large / chunk / push_blocks_per_sm for ``mt.run_batch``, timed
    on an evenly spaced sample of at most ``sample`` queries."""
    space = space or BATCH_SPACE
    name, sms = mt.device_info(device)
    ops = sorted({int(q["op"]) for q in queries})
    key = f"batch|{name}|{sms}|{graph_signature(*graph_csrs)}|{ops}|{len(queries)}"
    if cache is not None and cache.get(key):
        return dict(cache.get(key)["config"])
    step = max(1, len(queries) // sample)
    qs = queries[::step][:sample]
    batches = {}

    def measure(c):
        k = (c.get("mode", 0), c["cut_large"], c["chunk"])
        batches[k] = mt.run_batch(G, qs, batch=batches.get(k), **c)
        return batches[k].stats()["elapsed_ms"]

    best, timings = search(space, measure)
    for b in batches.values():
        b.close()
    if cache is not None:
        cache.put(key, {"config": best, "timings": timings[:5]})
    return best
