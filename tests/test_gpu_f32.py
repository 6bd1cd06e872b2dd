"""Float-weight SSSP (MAITER_OP_MIN_F32) on the paper's log-normal synthetic
graphs (Section 6.1: in-degrees LN(-0.5, 2.3), weights LN(0, 1) in IEEE
single).  Both sides form every distance as fl(d + w) rounded to nearest and
take the least over paths, so the GPU distances must equal the oracle's bit
for bit under every schedule."""
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


def sources(g, k):
    # the highest out-degree vertices reach the most of a log-normal graph
    return np.argsort(-np.diff(g.row_ptr), kind="stable")[:k]


@pytest.mark.parametrize("logn", [10, 14, 17])
def test_f32_sssp_bit_exact_on_lognormal_graphs(mt, logn):
    g = graphgen.lognormal(1 << logn, weights=True)
    G = mt.Graph.from_csr(g)
    for s in sources(g, 3):
        r = mt.run(G, mt.OP_MIN_F32, source=int(s))
        v = r.state()
        assert v.dtype == np.float32
        np.testing.assert_array_equal(v.view(np.uint32), oracle.dijkstra_f32(g, int(s)).view(np.uint32))
        assert r.stats()["converged"] == 1


@pytest.mark.parametrize("kw", [dict(sched=2, top_frac=0.05), dict(sched=4, threshold=0.5),
                                dict(sched=4, threshold=8.0)])
def test_f32_sssp_priority_and_bucket_schedules(mt, kw):
    g = graphgen.lognormal(1 << 15, weights=True)
    G = mt.Graph.from_csr(g)
    s = int(sources(g, 1)[0])
    r = mt.run(G, mt.OP_MIN_F32, source=s, **kw)
    np.testing.assert_array_equal(r.state().view(np.uint32), oracle.dijkstra_f32(g, s).view(np.uint32))


def test_f32_full_size_lognormal(mt):
    # 2^20 vertices (about 8.5 M edges), the bench's float workload
    g = graphgen.lognormal(1 << 20, weights=True)
    G = mt.Graph.from_csr(g)
    r = None
    for s in sources(g, 2):
        r = mt.run(G, mt.OP_MIN_F32, source=int(s), result=r)
        np.testing.assert_array_equal(r.state(), oracle.dijkstra_f32(g, int(s)))


def test_f32_integer_valued_weights_match_integer_run(mt):
    # R-MAT with its integer weights as floats: the same distances as MIN_U32
    g = graphgen.rmat(12, 8, weights=True)
    G = mt.Graph.from_csr(g)
    Gf = mt.Graph(g.row_ptr, g.col, g.w.astype(np.float32))
    s = int(graphgen.sssp_sources(g, 1)[0])
    du = mt.run(G, mt.OP_MIN_U32, source=s).state()
    df = mt.run(Gf, mt.OP_MIN_F32, source=s).state()
    expect = np.where(du == mt.INF32, np.inf, du.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(df, expect)


def test_f32_hub_multi_source_and_rounding(mt):
    # a star hub (chunked path) with tiny weights whose sums round, and two
    # sources given through delta0
    n = 7000
    src = np.concatenate([np.zeros(n - 1, np.int64), np.arange(1, n - 1)])
    dst = np.concatenate([np.arange(1, n), np.arange(2, n)])
    w = np.concatenate([np.full(n - 1, 1.0, np.float32), np.full(n - 2, 2.0 ** -24, np.float32)])
    g = graphgen.csr_from_edges(n, src, dst, w.view(np.uint32))
    G = mt.Graph.from_csr(g)
    d0 = np.full(n, np.inf, dtype=np.float32)
    d0[[0, 5000]] = 0.0
    r = mt.run(G, mt.OP_MIN_F32, delta0=d0)
    expect = np.minimum(oracle.dijkstra_f32(g, 0), oracle.dijkstra_f32(g, 5000))
    np.testing.assert_array_equal(r.state(), expect)


def test_f32_rejects_bad_weights_and_engines(mt):
    g = graphgen.lognormal(256, weights=True)
    for bad in (-1.0, np.inf, np.nan):
        w = graphgen.float_weights(g).copy()
        w[7] = bad
        G = mt.Graph(g.row_ptr, g.col, w)
        with pytest.raises(mt.MaiterError) as ei:
            mt.run(G, mt.OP_MIN_F32, source=0)
        assert ei.value.status == mt.ERR_INVALID_ARG
    G = mt.Graph.from_csr(g)
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_MIN_F32, source=0, engine=mt.ENGINE_ASYNC)
    assert ei.value.status == mt.ERR_UNSUPPORTED
