import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def rmat24():
    """The R-MAT scale-24 graph (edge factor 16) of the full-size PageRank
    runs, generated once per session (about half a minute on the host)."""
    import graphgen
    return graphgen.rmat(24, 16)


@pytest.fixture(scope="session")
def pagerank24(rmat24):
    """PageRank (d = 0.8) on the scale-24 graph by the FP64 round engine to
    sum |Delta| < 4e-8, with the oracle's bound on its error:
    ||v* - v||_1 <= ||c + P^T v - v||_1 / (1 - d) (r computed by the oracle).
    Also holds the uploaded graph for further runs."""
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_1710_05785_b300 as mt
    g = rmat24
    dev = torch.device("cuda", 0)
    G = mt.Graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev))
    r = mt.run(G, mt.OP_SUM_F64, damping=0.8, eps=4e-8)
    assert r.stats()["converged"] == 1
    v = r.state()
    r.close()
    coef = oracle.pagerank_coef(g, 0.8)
    c = oracle.pagerank_c(g.n, 0.8)
    bound = float(np.abs(oracle.linear_residual(g, coef, c, v)).sum() / (1 - 0.8))
    yield {"g": g, "G": G, "v": v, "bound": bound}
    G.close()
