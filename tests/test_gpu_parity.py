"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances:
  * SSSP (min over uint32): bit-exact against Dijkstra.
  * PageRank-style sums: norm-wise relative error max|v - v*| / max|v*| <= 1e-6.
    With termination at sum|Delta| < eps the distance to the fixed point obeys
    ||v - v*||_1 <= eps / (1 - d) (Delta is exactly what remains to be
    spread), so eps = 1e-8 bounds the per-entry error by 5e-8 absolute; the
    extra margin covers FP64 (or FP32-delta) rounding of the accumulation.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.8
TOL = 1e-6


@pytest.fixture(scope="module")
def mt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_05785_b300 as m
    m.lib()
    return m


# ------------------------------------------------------------- PageRank

@pytest.mark.parametrize("scale,ef", [(6, 4), (10, 8), (13, 8)])
def test_pagerank_f64_matches_power_iteration(mt, scale, ef):
    g = graphgen.rmat(scale, ef)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-8)
    vstar = oracle.pagerank(g, D)
    v = r.state()
    assert oracle.relative_error(v, vstar) <= TOL
    st = r.stats()
    assert st["converged"] == 1 and st["residual"] < 1e-8
    # the remaining delta really is what the residual says
    assert abs(r.delta().sum() - st["residual"]) <= 1e-12 + 1e-9 * st["residual"]
    # ||v* - v||_1 <= sum|Delta| / (1 - d)
    assert np.abs(vstar - v).sum() <= st["residual"] / (1 - D) * (1 + 1e-6) + 1e-12


def test_pagerank_mass_invariant_on_gpu_state(mt):
    # sum v + (sum Delta + d * leak) / (1-d) = n, leak = sum of v over dangling
    # vertices (everything folded there stays there); checked mid-run too.
    g = graphgen.rmat(12, 4)
    G = mt.Graph.from_csr(g)
    dangling = np.diff(g.row_ptr) == 0
    assert dangling.any()
    for rounds in [1, 3, 10, 1000]:
        r = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-9, max_rounds=rounds,
                   allow_not_converged=True)
        v, dl = r.state(), r.delta()
        inv = oracle.pagerank_mass_invariant(v, dl, v[dangling].sum(), g.n, D)
        assert abs(inv) < 1e-8 * g.n


def test_pagerank_threshold_schedule_same_fixed_point(mt):
    g = graphgen.rmat(13, 8)
    G = mt.Graph.from_csr(g)
    vstar = oracle.pagerank(g, D)
    r_all = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-8)
    r_thr = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-8, sched=mt.SCHED_THRESHOLD,
                   threshold=1e-4)
    assert oracle.relative_error(r_thr.state(), vstar) <= TOL
    assert oracle.relative_error(r_all.state(), vstar) <= TOL
    # every round activates at most n vertices, and the threshold run used it
    for st in (r_all.stats(), r_thr.stats()):
        assert 0 < st["activations"] <= st["rounds"] * g.n


def test_pagerank_threshold_too_high_still_terminates(mt):
    g = graphgen.rmat(10, 8)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-8, sched=mt.SCHED_THRESHOLD, threshold=10.0)
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= TOL


@pytest.mark.parametrize("scale,ef", [(13, 8), (16, 16)])
def test_pagerank_mixed_precision(mt, scale, ef):
    # FP64 deltas until the residual is 1/100 of its start, FP32 deltas after
    g = graphgen.rmat(scale, ef)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_MIXED, damping=D, eps=1e-8)
    assert r.state().dtype == np.float64 and r.delta().dtype == np.float32
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= TOL
    st = r.stats()
    assert st["converged"] == 1 and st["residual"] < 1e-8


def test_pagerank_pure_fp32_deltas_error_is_bounded(mt):
    # mixed_switch = 1: FP32 deltas from the first round.  Its error against the
    # FP64 oracle grows with hub in-degree; stated here, bounded loosely.
    g = graphgen.rmat(13, 8)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_MIXED, damping=D, eps=1e-8, mixed_switch=1.0)
    err = oracle.relative_error(r.state(), oracle.pagerank(g, D))
    assert err <= 2e-5
    # the FP64 phase cuts the error: the default schedule is well inside 1e-6
    r2 = mt.run(G, mt.OP_SUM_MIXED, damping=D, eps=1e-8)
    assert oracle.relative_error(r2.state(), oracle.pagerank(g, D)) <= 1e-7


def test_personalised_pagerank_with_explicit_delta0_and_coef(mt):
    g = graphgen.rmat(12, 8)
    G = mt.Graph.from_csr(g)
    seeds = graphgen.ppr_seed_sets(g.n, 1, seed=11)[0]
    c = oracle.pagerank_c(g.n, D, seeds)
    coef = oracle.pagerank_coef(g, D)
    r = mt.run(G, mt.OP_SUM_F64, coef=coef, v0=np.zeros(g.n), delta0=c, eps=1e-6 * 0.04 / len(seeds))
    vstar, _ = oracle.linear_power(g, coef, c)
    assert oracle.relative_error(r.state(), vstar) <= TOL


def test_device_inputs_and_result_reuse(mt):
    g = graphgen.rmat(11, 8)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    G = mt.Graph(rp, col)
    d0 = torch.full((g.n,), 1 - D, dtype=torch.float64, device="cuda")
    v0 = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    r = mt.run(G, mt.OP_SUM_F64, v0=v0, delta0=d0, eps=1e-9)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    r.state(out)
    vstar = oracle.pagerank(g, D)
    assert oracle.relative_error(out.cpu().numpy(), vstar) <= TOL
    # reuse the same result: no allocation, same answer
    r2 = mt.run(G, mt.OP_SUM_F64, eps=1e-9, result=r)
    assert r2 is r
    assert oracle.relative_error(r.state(), vstar) <= TOL


def test_resume_from_saved_state(mt):
    # (v, Delta) between kernels is a complete DAIC state: stop, resume, same answer
    g = graphgen.rmat(12, 8)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, eps=1e-9, max_rounds=4, allow_not_converged=True)
    assert r.stats()["converged"] == 0
    v, dl = r.state(), r.delta()
    r2 = mt.run(G, mt.OP_SUM_F64, v0=v, delta0=dl, eps=1e-9)
    assert oracle.relative_error(r2.state(), oracle.pagerank(g, D)) <= TOL


def test_round_cap_reports_not_converged(mt):
    g = graphgen.rmat(10, 8)
    G = mt.Graph.from_csr(g)
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_F64, eps=1e-12, max_rounds=2)
    assert ei.value.status == mt.ERR_NOT_CONVERGED


# ----------------------------------------------------------------- SSSP

@pytest.mark.parametrize("scale,ef", [(6, 4), (11, 8), (14, 16)])
def test_sssp_bit_exact_against_dijkstra(mt, scale, ef):
    g = graphgen.rmat(scale, ef, weights=True)
    G = mt.Graph.from_csr(g)
    for s in graphgen.sssp_sources(g, 3):
        r = mt.run(G, mt.OP_MIN_U32, source=int(s))
        np.testing.assert_array_equal(r.state(), oracle.dijkstra(g, int(s)))
        st = r.stats()
        assert st["converged"] == 1 and st["residual"] == 0


def test_sssp_full_size_eight_sources(mt):
    # R-MAT scale 20, edge factor 16, 8 sources one after another (the bench's
    # configuration and launch shape), every distance compared to Dijkstra.
    g = graphgen.rmat(20, 16, weights=True)
    G = mt.Graph.from_csr(g)
    r = None
    for s in graphgen.sssp_sources(g, 8):
        r = mt.run(G, mt.OP_MIN_U32, source=int(s), result=r)
        np.testing.assert_array_equal(r.state(), oracle.dijkstra(g, int(s)))


def test_sssp_unreachable_and_self_loops(mt):
    # 0 -> 1 (5), 1 -> 1 (1), 1 -> 2 (7), 3 isolated, 4 -> 0 (unreachable from 0)
    g = graphgen.small_graph(5, [(0, 1), (1, 1), (1, 2), (4, 0)], weights=[5, 1, 7, 2])
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_MIN_U32, source=0)
    np.testing.assert_array_equal(r.state(), [0, 5, 12, mt.INF32, mt.INF32])


def test_sssp_from_explicit_delta0_multi_source(mt):
    g = graphgen.rmat(12, 8, weights=True)
    G = mt.Graph.from_csr(g)
    s = graphgen.sssp_sources(g, 2)
    d0 = np.full(g.n, mt.INF32, dtype=np.uint32)
    d0[s] = 0
    r = mt.run(G, mt.OP_MIN_U32, delta0=d0)
    expect = np.minimum(oracle.dijkstra(g, int(s[0])), oracle.dijkstra(g, int(s[1])))
    np.testing.assert_array_equal(r.state(), expect)


# ----------------------------------------------------------- edge cases

def test_empty_and_edgeless_graphs(mt):
    G0 = mt.Graph(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    r0 = mt.run(G0, mt.OP_SUM_F64)
    assert r0.state().shape == (0,)
    G1 = mt.Graph(np.zeros(4, dtype=np.int64), np.zeros(0, dtype=np.int32))
    r1 = mt.run(G1, mt.OP_SUM_F64, eps=1e-12)
    np.testing.assert_allclose(r1.state(), [0.2, 0.2, 0.2])


def test_hub_vertex_uses_cta_path(mt):
    # one vertex with 50,000 out-edges (large bucket) plus a ragged tail
    n = 50001
    src = np.concatenate([np.zeros(n - 1, np.int64), np.arange(1, 40, dtype=np.int64)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int64), np.arange(2, 41, dtype=np.int64)])
    g = graphgen.csr_from_edges(n, src, dst)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, eps=1e-10)
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= TOL


def test_invalid_arguments_are_rejected(mt):
    with pytest.raises(mt.MaiterError) as ei:
        mt.Graph(np.array([0, 2, 1], dtype=np.int64), np.array([0, 1], dtype=np.int32))
    assert ei.value.status == mt.ERR_INVALID_ARG
    with pytest.raises(mt.MaiterError):
        mt.Graph(np.array([0, 1, 2], dtype=np.int64), np.array([0, 7], dtype=np.int32))
    g = graphgen.rmat(6, 4)
    G = mt.Graph.from_csr(g)
    with pytest.raises(mt.MaiterError):   # min without weights
        mt.run(G, mt.OP_MIN_U32, source=0)
    with pytest.raises(mt.MaiterError):   # bad eps
        mt.run(G, mt.OP_SUM_F64, eps=-1.0)


@pytest.mark.parametrize("cap", [1, 2, 3, 4, 5, 6, 7])
def test_round_cap_in_either_position_of_a_pass(mt, cap):
    # the graph loop runs three rounds per pass; a cap that falls on any of
    # them stops after exactly `cap` pushes with a valid DAIC state that resumes
    g = graphgen.rmat(11, 8, weights=True)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, eps=1e-10, max_rounds=cap, allow_not_converged=True)
    st = r.stats()
    assert st["rounds"] == cap and st["status"] == mt.ERR_NOT_CONVERGED
    v, dl = r.state(), r.delta()
    dangling = np.diff(g.row_ptr) == 0
    assert abs(oracle.pagerank_mass_invariant(v, dl, v[dangling].sum(), g.n, D)) < 1e-9 * g.n
    r2 = mt.run(G, mt.OP_SUM_F64, v0=v, delta0=dl, eps=1e-10)
    assert oracle.relative_error(r2.state(), oracle.pagerank(g, D)) <= TOL
    s = int(graphgen.sssp_sources(g, 1)[0])
    q = mt.run(G, mt.OP_MIN_U32, source=s, max_rounds=cap, allow_not_converged=True)
    assert q.stats()["rounds"] == cap
    exact = oracle.dijkstra(g, s)
    assert (q.state() >= exact).all()            # never below the true distance
    q2 = mt.run(G, mt.OP_MIN_U32, v0=q.state(), delta0=q.delta())
    np.testing.assert_array_equal(q2.state(), exact)
