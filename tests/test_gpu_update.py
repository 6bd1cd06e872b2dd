"""maiter_graph_update: new contents of the same shape copied into a graph's
buffers; results and their launch graphs stay valid and give the new graph's
fixed point; invalid contents are rejected and block runs until fixed."""
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


def test_update_then_reuse_results(mt):
    a = graphgen.rmat(12, 8, weights=True, seed=11)
    b = graphgen.rmat(12, 8, weights=True, seed=12)
    assert a.m == b.m
    G = mt.Graph.from_csr(a)
    s = int(graphgen.sssp_sources(a, 1)[0])
    r = mt.run(G, mt.OP_MIN_U32, source=s)
    np.testing.assert_array_equal(r.state(), oracle.dijkstra(a, s))
    p = mt.run(G, mt.OP_SUM_F64, eps=1e-9)
    stream = torch.cuda.current_stream().cuda_stream
    G.update(b.row_ptr, b.col, b.w, stream=stream)
    r2 = mt.run(G, mt.OP_MIN_U32, source=s, result=r)      # same result, same launch graph
    assert r2 is r
    np.testing.assert_array_equal(r.state(), oracle.dijkstra(b, s))
    mt.run(G, mt.OP_SUM_F64, eps=1e-9, result=p)
    assert oracle.relative_error(p.state(), oracle.pagerank(b, 0.8)) <= 1e-6
    # from device arrays too
    G.update(torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda(),
             torch.from_numpy(a.w.view(np.int32)).cuda())
    np.testing.assert_array_equal(mt.run(G, mt.OP_MIN_U32, source=s, result=r).state(),
                                  oracle.dijkstra(a, s))


def test_invalid_update_blocks_runs_until_fixed(mt):
    a = graphgen.rmat(10, 8, weights=True)
    G = mt.Graph.from_csr(a)
    bad = a.col.copy()
    bad[5] = a.n + 3
    with pytest.raises(mt.MaiterError) as ei:
        G.update(a.row_ptr, bad, a.w)
    assert ei.value.status == mt.ERR_INVALID_ARG
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_F64)
    assert ei.value.status == mt.ERR_INVALID_ARG
    with pytest.raises(mt.MaiterError) as ei:
        G.update(a.row_ptr, a.col)            # the graph has weights
    assert ei.value.status == mt.ERR_INVALID_ARG
    G.update(a.row_ptr, a.col, a.w)
    s = int(graphgen.sssp_sources(a, 1)[0])
    np.testing.assert_array_equal(mt.run(G, mt.OP_MIN_U32, source=s).state(), oracle.dijkstra(a, s))


def test_update_rechecks_float_weights(mt):
    g = graphgen.lognormal(2048, weights=True)
    G = mt.Graph.from_csr(g)
    s = int(np.argmax(np.diff(g.row_ptr)))
    mt.run(G, mt.OP_MIN_F32, source=s)                   # checked once: fine
    w = graphgen.float_weights(g).copy()
    w[3] = -1.0
    G.update(g.row_ptr, g.col, w)
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_MIN_F32, source=s)
    assert ei.value.status == mt.ERR_INVALID_ARG
