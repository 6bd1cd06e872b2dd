"""Vertex counts around the engine's tile sizes (the frontier scan takes
1024-vertex tiles of 256 threads; lists and pushes are cut in warps of 32)
and degenerate graphs, for every operator family, against the oracle:
uniform random multigraphs with 3n edges (self-loops and repeated edges
included), one vertex, and graphs without edges.  SSSP, float SSSP and
labels are exact; PageRank is within the relative tolerance 1e-6 that
sum |Delta| < 1e-10 guarantees with room to spare."""
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


SIZES = [1, 2, 31, 33, 255, 257, 1023, 1024, 1025, 2047, 3073, 4097]


@pytest.mark.parametrize("n", SIZES)
def test_every_operator_around_tile_sizes(mt, n):
    g = graphgen.random_graph(n, 3 * n, seed=100 + n, weights=True)
    G = mt.Graph.from_csr(g)
    for s in sorted({0, n // 2, n - 1}):
        np.testing.assert_array_equal(mt.run(G, mt.OP_MIN_U32, source=s).state(),
                                      oracle.dijkstra(g, s))
    gf = graphgen.CSRGraph(g.n, g.m, g.row_ptr, g.col,
                           (g.w.astype(np.float32) * np.float32(0.731)).view(np.uint32))
    np.testing.assert_array_equal(
        mt.run(mt.Graph.from_csr(gf), mt.OP_MIN_F32, source=n - 1).state().view(np.uint32),
        oracle.dijkstra_f32(gf, n - 1).view(np.uint32))
    r = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-10)
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= 1e-6
    np.testing.assert_array_equal(mt.run(G, mt.OP_MAX_I32).state(), oracle.max_reach_labels(g))


@pytest.mark.parametrize("n", [1, 1000, 1025])
def test_graphs_without_edges(mt, n):
    g = graphgen.random_graph(n, 0, seed=7)
    G = mt.Graph.from_csr(g)
    s = n // 3
    d = mt.run(G, mt.OP_MIN_U32, source=s)
    expect = np.full(n, mt.INF32, dtype=np.uint32)
    expect[s] = 0
    np.testing.assert_array_equal(d.state(), expect)
    assert d.stats()["converged"] == 1
    r = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-12)
    np.testing.assert_allclose(r.state(), np.full(n, 1 - D), rtol=1e-15)
    np.testing.assert_array_equal(mt.run(G, mt.OP_MAX_I32).state(), np.arange(n, dtype=np.int32))
