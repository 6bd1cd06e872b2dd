"""Top-fraction priority scheduling (priority-queue extraction, Section 5.1) on
the GPU: the selected set of a round is compared exactly with the oracle's
reading (k = ceil(q * #pending), threshold = the k-th largest FP32 key, ties
included), and the fixed point with the oracle's."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.8


@pytest.fixture(scope="module")
def mt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_05785_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("q", [0.01, 0.1, 0.37, 1.0])
@pytest.mark.parametrize("seed", [1, 2])
def test_one_round_selects_exactly_the_oracle_set(mt, q, seed):
    g = graphgen.rmat(12, 8)
    G = mt.Graph.from_csr(g)
    rng = np.random.default_rng(seed)
    # many ties and zeros, plus spread-out values over several binades
    vals = np.concatenate([[1e-3, 2e-3, 5e-3, 0.1], rng.uniform(1e-6, 1.0, 64)])
    delta0 = np.where(rng.random(g.n) < 0.3, 0.0, rng.choice(vals, g.n))
    r = mt.run(G, mt.OP_SUM_F64, v0=np.zeros(g.n), delta0=delta0, sched=mt.SCHED_TOPFRAC,
               top_frac=q, eps=1e-12, max_rounds=1, allow_not_converged=True)
    selected = np.nonzero(r.state() != 0.0)[0]
    np.testing.assert_array_equal(selected, oracle.topfrac_select(delta0, q))


@pytest.mark.parametrize("q", [0.05, 0.3])
def test_topfrac_pagerank_fixed_point(mt, q):
    g = graphgen.rmat(13, 8)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, eps=1e-8, sched=mt.SCHED_TOPFRAC, top_frac=q)
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= 1e-6


def test_topfrac_mixed_precision(mt):
    g = graphgen.rmat(13, 8)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_MIXED, eps=1e-8, sched=mt.SCHED_TOPFRAC, top_frac=0.2)
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= 1e-6


def test_topfrac_sssp_bit_exact(mt):
    g = graphgen.rmat(14, 16, weights=True)
    G = mt.Graph.from_csr(g)
    for s in graphgen.sssp_sources(g, 2):
        r = mt.run(G, mt.OP_MIN_U32, source=int(s), sched=mt.SCHED_TOPFRAC, top_frac=0.05)
        np.testing.assert_array_equal(r.state(), oracle.dijkstra(g, int(s)))


def test_topfrac_round_sizes_respect_the_fraction(mt):
    # every round activates at least one and about q of the pending vertices
    # (more only through ties), so activations per round stay well below n
    g = graphgen.rmat(14, 16)
    G = mt.Graph.from_csr(g)
    b = mt.run(G, mt.OP_SUM_F64, eps=1e-6, sched=mt.SCHED_TOPFRAC, top_frac=0.1).stats()
    assert b["rounds"] >= 1
    assert b["activations"] <= 0.2 * g.n * b["rounds"]
    assert b["edge_pushes"] <= g.m * b["rounds"]


def test_topfrac_rejects_bad_fraction(mt):
    g = graphgen.rmat(6, 4)
    G = mt.Graph.from_csr(g)
    for q in [0.0, 1.5]:
        with pytest.raises(mt.MaiterError):
            mt.run(G, mt.OP_SUM_F64, sched=mt.SCHED_TOPFRAC, top_frac=q)
