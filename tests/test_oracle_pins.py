"""Pins for the CPU oracle: closed forms, independent routes, invariants and
values the paper prints.  Nothing here calls the CUDA path."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import scipy.sparse.linalg as spla

import graphgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")
D = 0.8


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------- PageRank closed forms

def test_cycle_fixed_point_is_one():
    # every vertex has in- and out-degree 1: v = (1-d) + d v  =>  v = 1
    n = 7
    g = graphgen.small_graph(n, [(i, (i + 1) % n) for i in range(n)])
    v = oracle.pagerank(g, D)
    np.testing.assert_allclose(v, np.ones(n), rtol=0, atol=1e-12)


def test_complete_digraph_fixed_point_is_one():
    n = 6
    g = graphgen.small_graph(n, [(i, j) for i in range(n) for j in range(n) if i != j])
    np.testing.assert_allclose(oracle.pagerank(g, D), np.ones(n), atol=1e-12)


def test_star_center_to_dangling_leaves():
    # center 0 -> leaves 1..L, leaves have no out-edges
    L = 5
    g = graphgen.small_graph(L + 1, [(0, k) for k in range(1, L + 1)])
    v = oracle.pagerank(g, D)
    assert v[0] == pytest.approx(1 - D, abs=1e-14)
    np.testing.assert_allclose(v[1:], (1 - D) + D * (1 - D) / L, atol=1e-14)


def test_single_edge():
    g = graphgen.small_graph(2, [(0, 1)])
    v = oracle.pagerank(g, D)
    np.testing.assert_allclose(v, [0.2, 0.36], atol=1e-14)


def test_sender_degree_reading_differs_from_receiver_degree():
    # Table 1 prints |N(j)|; the derivation of Section 3.1 uses |N(i)|.  On an
    # asymmetric graph the two readings give different fixed points, and the
    # closed form below (hand-derived with the sender's degree) must hold.
    # 0 -> 1, 0 -> 2, 1 -> 2, 2 -> 0
    g = graphgen.small_graph(3, [(0, 1), (0, 2), (1, 2), (2, 0)])
    v = oracle.pagerank(g, D)
    # v0 = .2 + .8 v2 ; v1 = .2 + .4 v0 ; v2 = .2 + .4 v0 + .8 v1
    A = np.array([[1, 0, -.8], [-.4, 1, 0], [-.4, -.8, 1]])
    np.testing.assert_allclose(v, np.linalg.solve(A, [.2, .2, .2]), atol=1e-13)
    # receiver-degree reading: edge i->k carries d/|N(k)|; its fixed point differs
    deg = np.diff(g.row_ptr)
    A_wrong = np.eye(3)
    for i in range(3):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            k = g.col[e]
            A_wrong[k, i] -= D / deg[k]
    assert np.abs(np.linalg.solve(A_wrong, [.2, .2, .2]) - v).max() > 1e-3


def test_multi_edges_count_with_multiplicity():
    # 0 -> 1 twice, 0 -> 2 once: 2/3 of 0's mass goes to 1
    g = graphgen.small_graph(3, [(0, 1), (0, 1), (0, 2)])
    v = oracle.pagerank(g, D)
    np.testing.assert_allclose(v, [0.2, 0.2 + D * 0.2 * 2 / 3, 0.2 + D * 0.2 / 3], atol=1e-14)


# ------------------------------------------------------- independent routes

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_power_iteration_matches_dense_lu(seed):
    g = graphgen.random_graph(300, 1500, seed)
    coef = oracle.pagerank_coef(g, D)
    c = oracle.pagerank_c(g.n, D)
    v, it = oracle.linear_power(g, coef, c)
    vd = oracle.dense_solve(g, coef, c)
    assert oracle.relative_error(v, vd) < 1e-12
    assert it > 10


def test_power_iteration_matches_sparse_solve_on_rmat():
    g = graphgen.rmat(12, 8)
    coef = oracle.pagerank_coef(g, D)
    c = oracle.pagerank_c(g.n, D)
    v, _ = oracle.linear_power(g, coef, c)
    P = sp.csr_matrix((coef[np.repeat(np.arange(g.n), np.diff(g.row_ptr))], g.col, g.row_ptr),
                      shape=(g.n, g.n))
    vs = spla.spsolve((sp.identity(g.n) - P.T).tocsc(), c)
    assert oracle.relative_error(v, vs) < 1e-12


def test_personalised_pagerank_matches_dense_lu():
    g = graphgen.random_graph(200, 900, 7)
    seeds = [3, 17, 150]
    coef = oracle.pagerank_coef(g, D)
    c = oracle.pagerank_c(g.n, D, seeds)
    assert c.sum() == pytest.approx(1 - D)
    v, _ = oracle.linear_power(g, coef, c)
    assert oracle.relative_error(v, oracle.dense_solve(g, coef, c)) < 1e-12


def test_linear_residual_zero_at_fixed_point_and_c_at_zero():
    g = graphgen.rmat(10, 8)
    coef = oracle.pagerank_coef(g, D)
    c = oracle.pagerank_c(g.n, D)
    v = oracle.pagerank(g, D)
    assert np.abs(oracle.linear_residual(g, coef, c, v)).max() < 1e-12
    np.testing.assert_array_equal(oracle.linear_residual(g, coef, c, np.zeros(g.n)), c)


# ---------------------------------------------------- DAIC (Theorems 1 and 3)

@pytest.mark.parametrize("sched", ["roundrobin", "priority"])
def test_async_daic_reaches_the_synchronous_fixed_point(sched):
    # Theorem 1 (round-robin) and Theorem 3 (priority scheduling)
    g = graphgen.rmat(10, 8)
    coef = oracle.pagerank_coef(g, D)
    ex = golden()["pagerank_init"]
    v0 = np.full(g.n, ex["v0"])
    d1 = np.full(g.n, ex["delta1"])
    r = oracle.daic_sum(g, coef, v0, d1, sched=sched, eps=1e-11)
    assert r["converged"]
    vstar = oracle.pagerank(g, D)
    assert oracle.relative_error(r["v"], vstar) < 1e-10


def test_worked_example_init_satisfies_fourth_condition():
    # v0 (+) Delta1 must equal one application of f to v0 (Section 3.1)
    ex = golden()["pagerank_init"]
    g = graphgen.rmat(9, 8)
    coef = oracle.pagerank_coef(g, ex["d"])
    c = oracle.pagerank_c(g.n, ex["d"])
    v0 = np.full(g.n, ex["v0"])
    f_v0 = v0 + oracle.linear_residual(g, coef, c, v0)
    np.testing.assert_allclose(v0 + ex["delta1"], f_v0, atol=0)


def test_progress_metric_rises_from_point_two_n_to_n_without_dangling():
    # Section 6.4: sum_j R_j goes from 0.2 N (after the first updates) to N
    ex = golden()["pagerank_progress"]
    n = 64
    edges = [(i, (i + 1) % n) for i in range(n)] + [(i, (5 * i + 3) % n) for i in range(n)]
    g = graphgen.small_graph(n, edges)
    assert np.diff(g.row_ptr).min() >= 1
    coef = oracle.pagerank_coef(g, ex["d"])
    # after the first synchronous DAIC step, v1 = v0 + Delta1
    assert (np.zeros(n) + np.full(n, 0.2)).sum() == pytest.approx(
        ex["start_fraction_of_N"] * n, abs=1e-12)
    r = oracle.daic_sum(g, coef, np.zeros(n), np.full(n, 0.2), eps=1e-13)
    assert r["v"].sum() == pytest.approx(ex["limit_fraction_of_N"] * n, rel=1e-12)


@pytest.mark.parametrize("sched", ["roundrobin", "priority"])
def test_mass_invariant_and_monotone_progress(sched):
    # The L1 norm of v rises monotonically (Section 3.5) and the mass
    # invariant holds at every cut, with dangling vertices present.
    g = graphgen.rmat(9, 4)
    assert (np.diff(g.row_ptr) == 0).any()
    coef = oracle.pagerank_coef(g, D)
    prev = -1.0
    for cut in [0, 1, 7, 100, 1000, 5000, 20000]:
        r = oracle.daic_sum(g, coef, np.zeros(g.n), np.full(g.n, 1 - D), sched=sched,
                            eps=0.0, max_updates=cut)
        assert abs(oracle.pagerank_mass_invariant(r["v"], r["delta"], r["leak"], g.n, D)) < 1e-9
        s = r["v"].sum()
        assert s >= prev - 1e-12
        prev = s


def test_priority_needs_no_more_updates_than_round_robin():
    # Theorem 4 in aggregate: priority order reaches the tolerance with fewer updates
    g = graphgen.rmat(11, 8)
    coef = oracle.pagerank_coef(g, D)
    a = oracle.daic_sum(g, coef, np.zeros(g.n), np.full(g.n, 0.2), "roundrobin", eps=1e-6)
    b = oracle.daic_sum(g, coef, np.zeros(g.n), np.full(g.n, 0.2), "priority", eps=1e-6)
    assert b["updates"] < a["updates"]


def test_residual_bounds_the_error():
    # ||v* - v||_1 <= sum|Delta| / (1-d): Delta is exactly what is still to be spread
    g = graphgen.rmat(10, 8)
    coef = oracle.pagerank_coef(g, D)
    vstar = oracle.pagerank(g, D)
    for cut in [100, 2000, 10000]:
        r = oracle.daic_sum(g, coef, np.zeros(g.n), np.full(g.n, 0.2), eps=0, max_updates=cut)
        assert np.abs(vstar - r["v"]).sum() <= r["delta"].sum() / (1 - D) * (1 + 1e-9)
        assert (vstar - r["v"] >= -1e-12).all()


# ------------------------------------------------------------------ SSSP

def _scipy_dist(g, s):
    # duplicate edges: keep the minimum weight (scipy would sum duplicates)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    order = np.lexsort((g.w, g.col, src))
    s_, c_, w_ = src[order], g.col[order], g.w[order]
    keep = np.ones(len(s_), bool)
    keep[1:] = (s_[1:] != s_[:-1]) | (c_[1:] != c_[:-1])
    A = sp.csr_matrix((w_[keep].astype(np.float64), (s_[keep], c_[keep])), shape=(g.n, g.n))
    d = csgraph.dijkstra(A, directed=True, indices=s)
    out = np.full(g.n, oracle.INF32, dtype=np.uint64)
    fin = np.isfinite(d)
    out[fin] = d[fin].astype(np.uint64)
    return out.astype(np.uint32)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_dijkstra_matches_bellman_ford_tiny(seed):
    g = graphgen.random_graph(48, 150, seed, weights=True)
    for s in [0, 5, 47]:
        np.testing.assert_array_equal(oracle.dijkstra(g, s), oracle.bellman_ford(g, s))


def test_dijkstra_matches_scipy_on_rmat():
    g = graphgen.rmat(13, 8, weights=True)
    for s in graphgen.sssp_sources(g, 3):
        np.testing.assert_array_equal(oracle.dijkstra(g, int(s)), _scipy_dist(g, int(s)))


@pytest.mark.parametrize("sched", ["roundrobin", "priority"])
def test_daic_min_equals_dijkstra(sched):
    g = graphgen.rmat(11, 8, weights=True)
    for s in graphgen.sssp_sources(g, 2):
        v0, d0 = oracle.sssp_init(g.n, int(s))
        r = oracle.daic_min(g, v0, d0, sched)
        assert r["converged"]
        np.testing.assert_array_equal(r["v"], oracle.dijkstra(g, int(s)))


def test_sssp_table1_init():
    ex = golden()["table1_sssp"]
    v, d = oracle.sssp_init(5, 2)
    assert (v == oracle.INF32).all() and ex["v0"] == "inf"
    assert d[2] == ex["delta1_source"] and (np.delete(d, 2) == oracle.INF32).all()


def test_sssp_monotone_progress():
    # Section 6.4: sum_j d_j only decreases (over reached vertices)
    g = graphgen.rmat(9, 8, weights=True)
    s = int(graphgen.sssp_sources(g, 1)[0])
    final = oracle.dijkstra(g, s)
    prev = None
    for cut in [1, 10, 100, 1000, 100000]:
        v0, d0 = oracle.sssp_init(g.n, s)
        r = oracle.daic_min(g, v0, d0, max_updates=cut)
        assert (r["v"].astype(np.int64) >= final.astype(np.int64)).all()
        if prev is not None:
            assert (r["v"] <= prev).all()
        prev = r["v"]


# ----------------------------------------------------------- top-fraction

def test_topfrac_selection_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(1, 200))
        delta = np.where(rng.random(n) < 0.3, 0.0, rng.choice([1e-3, 2e-3, 5e-3, 0.1], n))
        q = float(rng.choice([0.01, 0.1, 0.5, 1.0]))
        sel = set(oracle.topfrac_select(delta, q).tolist())
        key = np.abs(delta).astype(np.float32)
        nz = [j for j in range(n) if key[j] > 0]
        if not nz:
            assert sel == set()
            continue
        k = max(1, int(np.ceil(q * len(nz))))
        ranked = sorted(nz, key=lambda j: -key[j])
        kth = key[ranked[k - 1]]
        assert sel == {j for j in nz if key[j] >= kth}
        assert len(sel) >= k
    assert set(oracle.topfrac_select(np.array([0.0, 1.0, 2.0, 0.0]), 1.0).tolist()) == {1, 2}
