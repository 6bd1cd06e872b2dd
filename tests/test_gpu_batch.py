"""Batched engine: personalised PageRank and SSSP queries over graphs of uneven
size in one CUDA-graph launch, each query checked against the oracle.

PPR tolerance: the batch stops a query when no vertex has |Delta| > eps_q / n,
so sum |Delta| <= eps_q and ||v - v*||_1 <= eps_q / (1 - d).  With
eps_q = 1e-6 (1 - d)^2 / |S| and v* >= (1 - d) / |S| at the seeds, the
norm-wise relative error is at most 1e-6 (the bound asserted below)."""
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


def make_batch(scales, n_ppr, n_sssp, seed=7):
    graphs = [graphgen.rmat(s, 8, weights=True, seed=1000 + s + i) for i, s in enumerate(scales)]
    queries = []
    for gi, g in enumerate(graphs):
        for q, S in enumerate(graphgen.ppr_seed_sets(g.n, n_ppr, seed=seed + gi, max_size=16)):
            eps = 1e-6 * (1 - D) ** 2 / len(S)
            queries.append(dict(op=0, graph=gi, seeds=S, damping=D, eps=eps))
        for s in graphgen.sssp_sources(g, n_sssp, seed=seed + 100 + gi):
            queries.append(dict(op=2, graph=gi, seeds=[int(s)]))
    return graphs, queries


def check(mt, graphs, queries, b):
    for qi, q in enumerate(queries):
        g = graphs[q["graph"]]
        v = b.state(qi)
        if q["op"] == 2:
            expect = oracle.dijkstra(g, int(q["seeds"][0]))
            np.testing.assert_array_equal(v, expect, err_msg=f"query {qi}")
        else:
            vstar = oracle.pagerank(g, D, seeds=q["seeds"])
            assert oracle.relative_error(v, vstar) <= 1e-6, qi


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_batch_mixed_queries_uneven_graphs(mt, mode):
    graphs, queries = make_batch([8, 10, 11, 12], n_ppr=6, n_sssp=3)
    G = [mt.Graph.from_csr(g) for g in graphs]
    b = mt.run_batch(G, queries, mode=mode)
    check(mt, graphs, queries, b)
    st = b.stats()
    assert st["converged"] == 1 and st["rounds"] >= 1
    qr = b.query_rounds()
    # 0 for a query whose seeds send nothing (all of them dangling)
    assert (qr >= 0).all() and qr.max() <= st["rounds"] and (qr > 0).sum() > len(queries) // 2


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_batch_reuse_gives_the_same_answer(mt, mode):
    graphs, queries = make_batch([9, 11], n_ppr=4, n_sssp=2, seed=3)
    G = [mt.Graph.from_csr(g) for g in graphs]
    b = mt.run_batch(G, queries, mode=mode)
    first = [b.state(i).copy() for i in range(len(queries))]
    b2 = mt.run_batch(G, queries, batch=b, mode=mode)
    assert b2 is b
    for i, q in enumerate(queries):
        if q["op"] == 2:
            np.testing.assert_array_equal(first[i], b.state(i))
        else:
            assert oracle.relative_error(b.state(i), first[i]) <= 1e-6


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_batch_multi_source_sssp_and_hub_chunks(mt, mode):
    # a star hub (chunked path) plus an R-MAT graph; a two-seed SSSP query
    n = 6000
    src = np.concatenate([np.zeros(n - 1, np.int64), np.arange(1, n - 1)])
    dst = np.concatenate([np.arange(1, n), np.arange(2, n)])
    w = (np.arange(src.size) % 7 + 1).astype(np.uint32)
    star = graphgen.csr_from_edges(n, src, dst, w)
    r = graphgen.rmat(11, 8, weights=True)
    G = [mt.Graph.from_csr(star), mt.Graph.from_csr(r)]
    s2 = graphgen.sssp_sources(r, 2)
    queries = [dict(op=2, graph=0, seeds=[0]), dict(op=0, graph=0, seeds=[0, 5], damping=D,
                                                    eps=1e-6 * (1 - D) ** 2 / 2),
               dict(op=2, graph=1, seeds=[int(s2[0]), int(s2[1])])]
    b = mt.run_batch(G, queries, cut_large=256, chunk=512, mode=mode)
    np.testing.assert_array_equal(b.state(0), oracle.dijkstra(star, 0))
    assert oracle.relative_error(b.state(1), oracle.pagerank(star, D, seeds=[0, 5])) <= 1e-6
    expect = np.minimum(oracle.dijkstra(r, int(s2[0])), oracle.dijkstra(r, int(s2[1])))
    np.testing.assert_array_equal(b.state(2), expect)


def test_autotuned_configs_keep_results_exact(mt, tmp_path):
    from paper_1710_05785_b300 import autotune
    graphs, queries = make_batch([9, 11], n_ppr=3, n_sssp=2, seed=5)
    G = [mt.Graph.from_csr(g) for g in graphs]
    cache = autotune.Cache(str(tmp_path / "t.json"))
    best = autotune.tune_batch(mt, graphs, G, queries, cache=cache, sample=8)
    assert set(best) == {"mode", "cut_large", "chunk", "push_blocks_per_sm"}
    assert autotune.tune_batch(mt, graphs, G, queries, cache=cache, sample=8) == best  # cached
    b = mt.run_batch(G, queries, **best)
    check(mt, graphs, queries, b)
    # single-run tuning: SSSP on one graph, then an exact run with the tuned cut-offs
    g = graphs[1]
    Gs = G[1]
    s = int(queries[-1]["seeds"][0])
    cfg = autotune.tune_run(mt, g, Gs, dict(op=mt.OP_MIN_U32, source=s), cache=cache)
    r = mt.run(Gs, mt.OP_MIN_U32, source=s, **cfg)
    np.testing.assert_array_equal(r.state(), oracle.dijkstra(g, s))


def test_batch_rejects_bad_queries(mt):
    g = graphgen.rmat(6, 4, weights=True)
    G = [mt.Graph.from_csr(g)]
    with pytest.raises(mt.MaiterError):
        mt.run_batch(G, [dict(op=2, graph=0, seeds=[g.n])])
    with pytest.raises(mt.MaiterError):
        mt.run_batch(G, [dict(op=1, graph=0, seeds=[0])])
    with pytest.raises(mt.MaiterError):
        mt.run_batch(G, [dict(op=0, graph=1, seeds=[0], eps=1e-6)])


def test_chained_mode_runs_queries_one_after_another(mt):
    # mode 2: the same answers as separate maiter_run calls, query by query,
    # and a reused chained batch switches to mode 0 and back without mixing
    g = graphgen.rmat(12, 16, weights=True)
    G = mt.Graph.from_csr(g)
    src = [int(s) for s in graphgen.sssp_sources(g, 5)]
    queries = [dict(op=2, graph=0, seeds=[s]) for s in src]
    b = mt.run_batch([G], queries, mode=2)
    for i, s in enumerate(src):
        np.testing.assert_array_equal(b.state(i), mt.run(G, mt.OP_MIN_U32, source=s).state())
    b0 = mt.run_batch([G], queries, mode=0)
    b2 = mt.run_batch([G], queries, mode=2, batch=b)
    for i in range(len(src)):
        np.testing.assert_array_equal(b2.state(i), b0.state(i))
    assert b2.stats()["converged"] == 1


def test_pull_groups_of_64_queries(mt):
    # mode 3: 70 personalised-PageRank queries on one graph (a full group of
    # 64 and a group of 6) and 40 on another, with different damping factors
    # in one group, and SSSP queries on their own branches
    g1 = graphgen.rmat(10, 8, weights=True, seed=41)
    g2 = graphgen.rmat(9, 8, weights=True, seed=42)
    queries = []
    for gi, (g, count) in enumerate([(g1, 70), (g2, 40)]):
        for q, S in enumerate(graphgen.ppr_seed_sets(g.n, count, seed=50 + gi, max_size=8)):
            d = 0.85 if q % 3 == 0 else D
            queries.append(dict(op=0, graph=gi, seeds=S, damping=d, eps=1e-6 * (1 - d) ** 2 / len(S)))
        queries.append(dict(op=2, graph=gi, seeds=[int(graphgen.sssp_sources(g, 1)[0])]))
    G = [mt.Graph.from_csr(g1), mt.Graph.from_csr(g2)]
    b = mt.run_batch(G, queries, mode=3)
    graphs = [g1, g2]
    for qi, q in enumerate(queries):
        g = graphs[q["graph"]]
        if q["op"] == 2:
            np.testing.assert_array_equal(b.state(qi), oracle.dijkstra(g, int(q["seeds"][0])))
        else:
            vstar = oracle.pagerank(g, q["damping"], seeds=q["seeds"])
            assert oracle.relative_error(b.state(qi), vstar) <= 1e-6, qi
    st = b.stats()
    qr = b.query_rounds()
    assert st["converged"] == 1 and (qr >= 1).all() and qr.max() <= st["rounds"]
    # profiling mode: the same answers, host-driven
    bp = mt.run_batch(G, queries, mode=3, flags=mt.FLAG_PROFILE_KERNELS)
    assert bp.stats()["push_launches"] > 0
    for qi, q in enumerate(queries):
        if q["op"] == 0:
            assert oracle.relative_error(bp.state(qi), b.state(qi)) <= 1e-6
