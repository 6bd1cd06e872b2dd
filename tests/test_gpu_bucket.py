"""Distance-ordered (BUCKET, delta-stepping) scheduling of the min operator:
any bucket width reaches the same fixed point, so every distance is compared
bit-exactly with Dijkstra; the work statistics are checked against what every
schedule must do (each reachable vertex is updated and pushes all its edges
at least once)."""
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


def check_work(mt, g, r):
    st = r.stats()
    reach = r.state() != mt.INF32
    assert st["converged"] == 1
    assert st["activations"] >= reach.sum()
    assert st["edge_pushes"] >= np.diff(g.row_ptr)[reach].sum()


@pytest.mark.parametrize("scale,ef", [(6, 4), (11, 8), (14, 16)])
@pytest.mark.parametrize("width", [1.0, 16.0, 256.0, 1e12])
def test_bucket_sssp_bit_exact(mt, scale, ef, width):
    g = graphgen.rmat(scale, ef, weights=True)
    G = mt.Graph.from_csr(g)
    for s in graphgen.sssp_sources(g, 2):
        r = mt.run(G, mt.OP_MIN_U32, source=int(s), sched=mt.SCHED_BUCKET, threshold=width)
        np.testing.assert_array_equal(r.state(), oracle.dijkstra(g, int(s)))
        check_work(mt, g, r)


def test_bucket_full_size_and_fewer_pushes_than_all(mt):
    # R-MAT scale 20, edge factor 16 (the bench graph): exact, and a narrow
    # bucket pushes fewer edges than updating every pending vertex
    g = graphgen.rmat(20, 16, weights=True)
    G = mt.Graph.from_csr(g)
    s = int(graphgen.sssp_sources(g, 1)[0])
    expect = oracle.dijkstra(g, s)
    r = mt.run(G, mt.OP_MIN_U32, source=s, sched=mt.SCHED_BUCKET, threshold=64.0)
    np.testing.assert_array_equal(r.state(), expect)
    check_work(mt, g, r)
    a = mt.run(G, mt.OP_MIN_U32, source=s)
    assert r.stats()["edge_pushes"] < a.stats()["edge_pushes"]
    assert r.stats()["rounds"] > a.stats()["rounds"]


def test_bucket_hub_multi_source_and_unreachable(mt):
    # a star hub (chunked large-vertex path), a second source through delta0,
    # and vertices nobody reaches
    n = 6000
    src = np.concatenate([np.zeros(n - 100, np.int64), np.arange(1, n - 200)])
    dst = np.concatenate([np.arange(1, n - 99), np.arange(2, n - 199)])
    w = (np.arange(src.size) % 13 + 1).astype(np.uint32)
    g = graphgen.csr_from_edges(n, src, dst, w)
    G = mt.Graph.from_csr(g)
    d0 = np.full(n, mt.INF32, dtype=np.uint32)
    d0[[0, 4000]] = 0
    r = mt.run(G, mt.OP_MIN_U32, delta0=d0, sched=mt.SCHED_BUCKET, threshold=8.0)
    expect = np.minimum(oracle.dijkstra(g, 0), oracle.dijkstra(g, 4000))
    np.testing.assert_array_equal(r.state(), expect)
    assert (r.state()[n - 99:] == mt.INF32).all()


def test_bucket_rejections(mt):
    g = graphgen.rmat(8, 4, weights=True)
    G = mt.Graph.from_csr(g)
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_F64, sched=mt.SCHED_BUCKET, threshold=1.0)
    assert ei.value.status == mt.ERR_INVALID_ARG
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_MIN_U32, source=0, sched=mt.SCHED_BUCKET, threshold=0.0)
    assert ei.value.status == mt.ERR_INVALID_ARG
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_MIN_U32, source=0, sched=mt.SCHED_BUCKET, threshold=4.0,
               engine=mt.ENGINE_ASYNC)
    assert ei.value.status == mt.ERR_UNSUPPORTED
