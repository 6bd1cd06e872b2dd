"""The batch and learned workloads at their full configurations, every result
against the oracle.

Batch: 512 personalised-PageRank queries (seed sets of 1-64 vertices,
log-uniform sizes) and 128 SSSP sources over 8 R-MAT graphs of scales 16-22
(edge factor 16), exactly as the bench builds them, run in the dense mode
(the autotuner's pick on a B300), in the chained dense mode and with the
PageRank queries in receive-side groups (mode 3).  SSSP answers
are compared bit for bit with Dijkstra.  PPR answers are bounded by the
oracle's one-step residual r = c + P^T v - v: ||v* - v||_1 <= ||r||_1 / (1 - d),
divided by max v for the norm-wise relative error (<= 1e-6).

Learned: scorers trained on traces of R-MAT scale-20 runs, applied with
learned scheduling to PageRank at R-MAT scale 24 (FP64 and mixed precision;
bounded through the FP64 round-engine run and its oracle residual, as the
full-size tests do) and to SSSP at R-MAT scale 22 (4 sources, bit for bit
against Dijkstra)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.8
THREADS = max(2, min(16, os.cpu_count() or 2))


@pytest.fixture(scope="module")
def mt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_05785_b300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def c4(mt):
    import bench
    graphs, queries = bench.batch_workload()
    G = [mt.Graph.from_csr(g) for g in graphs]
    sssp = [i for i, q in enumerate(queries) if q["op"] == 2]
    # the oracle's C routines release the GIL: threads run them in parallel
    with ThreadPoolExecutor(THREADS) as ex:
        dist = list(ex.map(lambda i: oracle.dijkstra(graphs[queries[i]["graph"]],
                                                     int(queries[i]["seeds"][0])), sssp))
    coefs = [oracle.pagerank_coef(g, D) for g in graphs]
    yield graphs, queries, G, dict(zip(sssp, dist)), coefs
    for x in G:
        x.close()


def check_batch(graphs, queries, b, dijkstra, coefs, group=16):
    worst = 0.0
    for start in range(0, len(queries), group):
        idx = list(range(start, min(len(queries), start + group)))
        states = {i: b.state(i) for i in idx}

        def one(i):
            q = queries[i]
            if q["op"] == 2:
                return -1.0 if np.array_equal(states[i], dijkstra[i]) else np.inf
            g = graphs[q["graph"]]
            r = oracle.linear_residual(g, coefs[q["graph"]], oracle.pagerank_c(g.n, D, q["seeds"]),
                                       states[i])
            return float(np.abs(r).sum() / (1 - D) / states[i].max())

        with ThreadPoolExecutor(THREADS) as ex:
            res = list(ex.map(one, idx))
        for i, e in zip(idx, res):
            assert e != np.inf, f"SSSP query {i} differs from Dijkstra"
            assert e <= 1e-6, f"PPR query {i}: norm-wise error bound {e}"
            worst = max(worst, e)
    return worst


@pytest.mark.parametrize("mode", [0, 2])
def test_batch_full_config_against_the_oracle(mt, c4, mode):
    graphs, queries, G, dijkstra, coefs = c4
    assert len(queries) == 640 and len(graphs) == 8
    assert sum(q["op"] == 0 for q in queries) == 512
    b = mt.run_batch(G, queries, mode=mode)
    st = b.stats()
    assert st["converged"] == 1
    worst = check_batch(graphs, queries, b, dijkstra, coefs)
    print(f"mode {mode}: {st['elapsed_ms']:.1f} ms, worst PPR bound {worst:.2e}")
    b.close()


def test_batch_full_config_pull_groups(mt, c4):
    # mode 3 (FP32 deltas): SSSP bit for bit; each PPR state bounded through
    # an FP64 mode-0 state of the same query run to eps_q / 100 and that
    # state's own residual bound (the L1 residual of an FP32-delta state sums
    # the rounding of every vertex; a reference stopped at eps_q would spend
    # the whole 1e-6 on its own bound)
    graphs, queries, G, dijkstra, coefs = c4
    tight = [dict(q, eps=q["eps"] / 100) if q["op"] == 0 else q for q in queries]
    b0 = mt.run_batch(G, tight, mode=0)
    b3 = mt.run_batch(G, queries, mode=3)
    assert b3.stats()["converged"] == 1
    worst = 0.0
    for i, q in enumerate(queries):
        v3 = b3.state(i)
        if q["op"] == 2:
            np.testing.assert_array_equal(v3, dijkstra[i], err_msg=f"SSSP query {i}")
            continue
        g = graphs[q["graph"]]
        v0 = b0.state(i)
        r = oracle.linear_residual(g, coefs[q["graph"]], oracle.pagerank_c(g.n, D, q["seeds"]), v0)
        e = float(np.abs(v3 - v0).max() / v0.max() + np.abs(r).sum() / (1 - D) / v0.max())
        assert e <= 1e-6, f"PPR query {i}: norm-wise error bound {e}"
        worst = max(worst, e)
    print(f"mode 3: {b3.stats()['elapsed_ms']:.1f} ms against {b0.stats()['elapsed_ms']:.1f} ms "
          f"for mode 0, worst PPR bound {worst:.2e}")
    b0.close()
    b3.close()


@pytest.fixture(scope="module")
def scorers(mt):
    import bench
    net_pr, net_ss, info = bench.train_scorers(mt, device=0)
    return net_pr, net_ss


@pytest.mark.parametrize("opname,q", [("OP_SUM_F64", 0.1), ("OP_SUM_F64", 0.5),
                                      ("OP_SUM_MIXED", 0.5), ("OP_SUM_MIXED", 0.3)])
def test_learned_pagerank_scale24(mt, scorers, pagerank24, opname, q):
    # the mixed runs switch to FP32 deltas at 1e-3 of the initial residual,
    # as the learned benchmark does (a held-back hub's FP32 delta rounds its
    # many messages at a coarser step)
    g, v_f64, bound_f64 = pagerank24["g"], pagerank24["v"], pagerank24["bound"]
    G = pagerank24["G"]
    r = mt.run(G, getattr(mt, opname), damping=D, eps=4e-8, sched=mt.SCHED_LEARNED,
               top_frac=q, scorer=scorers[0], mixed_switch=1e-3)
    st = r.stats()
    assert st["converged"] == 1
    err = np.abs(r.state() - v_f64).max() + bound_f64
    assert err <= 1e-6 * v_f64.max(), (err, v_f64.max())
    r.close()


def test_learned_sssp_scale22(mt, scorers):
    g = graphgen.rmat(22, 16, weights=True)
    G = mt.Graph.from_csr(g)
    srcs = [int(s) for s in graphgen.sssp_sources(g, 4)]
    with ThreadPoolExecutor(THREADS) as ex:
        want = list(ex.map(lambda s: oracle.dijkstra(g, s), srcs))
    for s, w in zip(srcs, want):
        r = mt.run(G, mt.OP_MIN_U32, source=s, sched=mt.SCHED_LEARNED, top_frac=0.05,
                   scorer=scorers[1])
        np.testing.assert_array_equal(r.state(), w, err_msg=f"source {s}")
        r.close()
    G.close()
