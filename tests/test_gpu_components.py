"""Connected components by max-label propagation (MAITER_OP_MAX_I32, Table 1:
max, g(x) = x, v^0 = -1, Delta^1_j = j): integer-exact, so every label is
compared bit-exactly with the oracle (union-find on symmetric graphs, the
largest reaching id on directed ones)."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_05785_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("scale,ef", [(6, 2), (12, 4), (16, 8)])
def test_components_of_symmetric_rmat(mt, scale, ef):
    g = graphgen.symmetrize(graphgen.rmat(scale, ef))
    r = mt.run(mt.Graph.from_csr(g), mt.OP_MAX_I32)
    labels = r.state()
    assert labels.dtype == np.int32
    np.testing.assert_array_equal(labels, oracle.component_labels(g))
    assert r.stats()["converged"] == 1


def test_directed_labels_are_the_largest_reaching_id(mt):
    for g in (graphgen.rmat(14, 4), graphgen.lognormal(1 << 14)):
        r = mt.run(mt.Graph.from_csr(g), mt.OP_MAX_I32)
        np.testing.assert_array_equal(r.state(), oracle.max_reach_labels(g))


def test_components_full_size_and_schedules(mt):
    g = graphgen.symmetrize(graphgen.rmat(20, 4))
    G = mt.Graph.from_csr(g)
    expect = oracle.component_labels(g)
    for kw in ({}, dict(sched=mt.SCHED_TOPFRAC, top_frac=0.1), dict(sched=mt.SCHED_THRESHOLD)):
        np.testing.assert_array_equal(mt.run(G, mt.OP_MAX_I32, **kw).state(), expect)


def test_components_hub_isolated_and_explicit_inputs(mt):
    # a star around vertex 0 (chunked path), a separate path 9000..9099 and
    # isolated vertices; Delta given explicitly as the ids gives the same labels
    n = 12000
    star = np.arange(1, 8000)
    path = np.arange(9000, 9099)
    src = np.concatenate([np.zeros(star.size, np.int64), star, path, path + 1])
    dst = np.concatenate([star, np.zeros(star.size, np.int64), path + 1, path])
    g = graphgen.csr_from_edges(n, src, dst)
    G = mt.Graph.from_csr(g)
    expect = oracle.component_labels(g)
    np.testing.assert_array_equal(mt.run(G, mt.OP_MAX_I32).state(), expect)
    r = mt.run(G, mt.OP_MAX_I32, v0=np.full(n, -1, np.int32), delta0=np.arange(n, dtype=np.int32))
    np.testing.assert_array_equal(r.state(), expect)
    assert expect[0] == 7999 and expect[9050] == 9099 and expect[10000] == 10000


def test_components_rejections(mt):
    G = mt.Graph.from_csr(graphgen.rmat(8, 4))
    for kw in (dict(sched=mt.SCHED_BUCKET, threshold=1.0), dict(engine=mt.ENGINE_ASYNC)):
        with pytest.raises(mt.MaiterError) as ei:
            mt.run(G, mt.OP_MAX_I32, **kw)
        assert ei.value.status == mt.ERR_UNSUPPORTED
