"""Training the learned priority scorer on activation traces of the method's
own runs.

A trace (``maiter_trace``) records, after every push of a round-engine run
with top-fraction scheduling, the scorer's 8 input features of a sample of
vertices, their deltas and the round of their last update.  Labels are
hindsight facts of the same run:

* sum ops (PageRank-style): log of the mass an update of the vertex in the
  recorded round moves per message, (1 - d [outdeg > 0]) |Delta_j| n /
  (outdeg_j + 1): the residual sum_k |Delta_k| falls by (1 - d) |Delta_j| (all
  of it for a dangling vertex) and the update costs outdeg_j messages.  The
  paper's priority |Delta_j| (Section 3.5) weighed by that cost; a high score
  means "cheap for what it removes", so the scheduler updates those first and
  lets the other deltas accumulate.  (Labelling with the mass moved at the
  vertex's next update in the trace instead taught the network mostly its
  degrees and scheduled worse.)
* min (SSSP): 1 if the vertex's tentative distance Delta_j is already its
  final distance, else 0: updating a vertex whose distance will still drop
  sends messages that will be sent again.

Training runs on the GPU through ``MLP.train`` (the library's own forward,
backward and Adam kernels).  This module only turns traces into (x, y).
"""
from __future__ import annotations

import numpy as np

INF32 = 0xFFFFFFFF


def labels_sum(tr: dict, outdeg: np.ndarray, n: int, d: float):
    """(X, y) for a sum-op trace (see module docstring): every record of a
    sampled vertex with a non-zero delta."""
    feat, dl = tr["features"], tr["delta"]
    rr, ss = np.nonzero(dl != 0.0)
    deg = outdeg[ss].astype(np.float64)
    mass = np.abs(dl[rr, ss]) * np.where(deg > 0, 1.0 - d, 1.0) * n / (deg + 1.0)
    keep = mass > 0
    X = feat[rr[keep], ss[keep]].astype(np.float32)
    y = np.log10(mass[keep]).astype(np.float32)
    return X, y


def labels_min(tr: dict, final: np.ndarray):
    """(X, y) for an SSSP trace: 1 where the pending tentative distance is final."""
    feat, dl, v = tr["features"], tr["delta"], tr["v"]
    pend = dl < v
    rr, ss = np.nonzero(pend)
    y = (dl[rr, ss] == final[ss].astype(np.float64)).astype(np.float32)
    X = feat[rr, ss].astype(np.float32)
    return X, y


def collect(mt, G, row_ptr, op: int, *, samples: int = 4096, records: int = 96, seed: int = 0,
            top_frac: float = 0.1, eps: float = 1e-8, damping: float = 0.8, source: int = -1):
    """Trace one round-engine run with top-fraction scheduling and label it."""
    n = len(row_ptr) - 1
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(n, size=min(samples, n), replace=False)).astype(np.int32)
    kw = dict(sched=mt.SCHED_TOPFRAC, top_frac=top_frac, eps=eps, damping=damping)
    if op == mt.OP_MIN_U32:
        kw["source"] = source
    tr, res = mt.trace(G, op, sample, records, **kw)
    outdeg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    if op == mt.OP_MIN_U32:
        final = res.state()
        X, y = labels_min(tr, final[sample])
    else:
        X, y = labels_sum(tr, outdeg[sample], n, damping)
    res.close()
    return X, y


def train(mt, X, y, *, device: int = 0, seed: int = 0, epochs: int = 30, batch: int = 1024,
          lr: float = 3e-3):
    """A new network trained on (X, y) with the library's GPU kernels."""
    net = mt.MLP(device=device, seed=seed)
    loss = net.train(X, y, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return net, loss
