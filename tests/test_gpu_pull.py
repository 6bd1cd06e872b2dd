"""The receive-side engine (MAITER_ENGINE_PULL): dense rounds of + whose
messages are summed at the receivers over the transpose.  Every run is
checked against the oracle's fixed point (Theorem 1: any schedule, the
synchronous one included, reaches the fixed point of Eq. 1), at sizes around
the 32-row groups, with rows at and past the 2048-in-edge cut and over several
4096-edge chunks, with caller-given coefficients and start vectors, after a
round cap (the state left must be a valid DAIC state and resume to the same
answer), after a graph update, and in profiling mode.

Tolerance: the run stops at sum |Delta| < eps, and ||v - v*||_1 <= sum |Delta|
/ (1 - d) (the bound of the termination reading), so eps = 1e-8 keeps the
norm-wise relative error far below 1e-6 for PageRank (max v* >= 1 - d)."""
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


def pull(mt, G, op, **kw):
    return mt.run(G, op, engine=mt.ENGINE_PULL, **kw)


def reversed_star(leaves, into=0):
    """Every leaf 1..L points at the centre: in-degree L at the centre."""
    edges = np.stack([np.arange(1, leaves + 1), np.full(leaves, into)], axis=1)
    return graphgen.small_graph(leaves + 1, edges)


# scale 17: 131,072 receivers (4,096 groups), message slots for about half
# of them (the senders)
@pytest.mark.parametrize("scale,ef", [(6, 4), (10, 8), (13, 8), (16, 16), (17, 16)])
@pytest.mark.parametrize("opname", ["OP_SUM_F64", "OP_SUM_MIXED"])
def test_pull_pagerank_matches_oracle(mt, scale, ef, opname):
    g = graphgen.rmat(scale, ef)
    G = mt.Graph.from_csr(g)
    r = pull(mt, G, getattr(mt, opname), damping=D, eps=1e-8)
    st = r.stats()
    assert st["converged"] == 1 and st["residual"] < 1e-8
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= 1e-6


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 100, 1000, 40001])
def test_pull_sizes_around_groups(mt, n):
    g = graphgen.random_graph(n, 4 * n, seed=n)
    G = mt.Graph.from_csr(g)
    for op in (mt.OP_SUM_F64, mt.OP_SUM_MIXED):
        r = pull(mt, G, op, damping=D, eps=1e-9)
        assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= 1e-6, (n, op)


def test_pull_graph_without_edges(mt):
    g = graphgen.small_graph(5000, np.zeros((0, 2), dtype=np.int64))
    G = mt.Graph.from_csr(g)
    r = pull(mt, G, mt.OP_SUM_F64, damping=D, eps=1e-12)
    np.testing.assert_allclose(r.state(), np.full(5000, 1 - D), rtol=0, atol=1e-15)
    assert r.stats()["converged"] == 1


# a group holds rows of up to 2048 in-edges; a larger row is cut into chunks
# of 4096: at and past the cut, one chunk and a ragged second, many chunks
@pytest.mark.parametrize("leaves", [256, 2048, 2049, 4096, 4097, 200000])
def test_pull_rows_at_and_past_the_cut(mt, leaves):
    # centre of in-degree L (leaves of out-degree 1): v_leaf = 1 - d,
    # v_centre = (1 - d) + L d (1 - d) (closed form)
    g = reversed_star(leaves)
    G = mt.Graph.from_csr(g)
    for op in (mt.OP_SUM_F64, mt.OP_SUM_MIXED):
        v = pull(mt, G, op, damping=D, eps=1e-12).state()
        want_c = (1 - D) + leaves * D * (1 - D)
        assert abs(v[0] - want_c) <= 1e-6 * want_c, (leaves, op, v[0], want_c)
        np.testing.assert_allclose(v[1:], 1 - D, rtol=1e-7)


@pytest.mark.parametrize("leaves", [1, 300, 200000])
def test_pull_star_of_one_sender(mt, leaves):
    # the centre, the only sender (message slot 0), sends to every leaf; closed form:
    # v_centre = 1 - d, v_leaf = (1 - d) + d (1 - d) / L
    edges = np.stack([np.zeros(leaves, dtype=np.int64), np.arange(1, leaves + 1)], axis=1)
    g = graphgen.small_graph(leaves + 1, edges)
    G = mt.Graph.from_csr(g)
    for op in (mt.OP_SUM_F64, mt.OP_SUM_MIXED):
        v = pull(mt, G, op, damping=D, eps=1e-12).state()
        assert abs(v[0] - (1 - D)) <= 1e-12
        np.testing.assert_allclose(v[1:], (1 - D) + D * (1 - D) / leaves, rtol=1e-7)


def test_pull_hubs_inside_a_random_graph(mt):
    # extra in-edges at three receivers of a random graph: one over several
    # chunks, one of a single chunk, one summed inside its group
    base = graphgen.random_graph(60000, 240000, seed=5)
    rng = np.random.default_rng(6)
    src = np.repeat(np.arange(base.n, dtype=np.int64), np.diff(base.row_ptr))
    extra_dst = np.concatenate([np.full(150000, 8200), np.full(3000, 12345), np.full(700, 30001)])
    extra_src = rng.integers(0, base.n, extra_dst.size)
    g2 = graphgen.csr_from_edges(base.n, np.concatenate([src, extra_src]),
                                 np.concatenate([base.col, extra_dst]))
    G2 = mt.Graph.from_csr(g2)
    for op in (mt.OP_SUM_F64, mt.OP_SUM_MIXED):
        r = pull(mt, G2, op, damping=D, eps=1e-9)
        assert oracle.relative_error(r.state(), oracle.pagerank(g2, D)) <= 1e-6, op


def test_pull_caller_coefficients_and_start_vectors(mt):
    # Katz from a source (Table 1): coef = beta for every sender, Delta1 = e_s
    g = graphgen.rmat(12, 8)
    beta = 0.5 / max(1, int(np.diff(g.row_ptr).max()))
    s = int(graphgen.sssp_sources(g, 1)[0])
    G = mt.Graph.from_csr(g)
    d0 = np.zeros(g.n)
    d0[s] = 1.0
    r = pull(mt, G, mt.OP_SUM_F64, coef=np.full(g.n, beta), v0=np.zeros(g.n), delta0=d0,
             eps=1e-14)
    want = oracle.katz(g, beta, s)
    assert np.abs(r.state() - want).max() <= 1e-12 * np.abs(want).max()
    # personalised PageRank seeds as delta0 in the mixed op (FP32 coefficients)
    seeds = graphgen.ppr_seed_sets(g.n, 1, seed=3)[0]
    d0 = np.zeros(g.n)
    d0[seeds] = (1 - D) / len(seeds)
    coef = oracle.pagerank_coef(g, D).astype(np.float32)
    r2 = pull(mt, G, mt.OP_SUM_MIXED, coef=coef, v0=np.zeros(g.n), delta0=d0, eps=1e-13)
    vstar = oracle.pagerank(g, D, seeds=seeds)
    assert oracle.relative_error(r2.state(), vstar) <= 1e-6


@pytest.mark.parametrize("opname", ["OP_SUM_F64", "OP_SUM_MIXED"])
def test_pull_round_cap_leaves_a_resumable_daic_state(mt, opname):
    op = getattr(mt, opname)
    g = graphgen.rmat(10, 8)
    G = mt.Graph.from_csr(g)
    r = pull(mt, G, op, damping=D, eps=1e-10, max_rounds=4, allow_not_converged=True)
    st = r.stats()
    assert st["converged"] == 0 and st["rounds"] == 4
    v, dl = r.state(), r.delta().astype(np.float64)
    # a valid DAIC state: v + (I - d P^T)^{-1} Delta = v* (checked by a direct solve)
    coef = oracle.pagerank_coef(g, D)
    vstar = oracle.dense_solve(g, coef, oracle.pagerank_c(g.n, D))
    tol = 1e-12 if op == mt.OP_SUM_F64 else 1e-6
    assert np.abs(v + oracle.dense_solve(g, coef, dl) - vstar).max() <= tol * vstar.max()
    r2 = pull(mt, G, op, damping=D, eps=1e-10, v0=v, delta0=dl)
    assert oracle.relative_error(r2.state(), vstar) <= 1e-6


def test_pull_after_graph_update(mt):
    a = graphgen.random_graph(30000, 200000, seed=1)
    b = graphgen.random_graph(30000, 200000, seed=2)
    G = mt.Graph.from_csr(a)
    r = pull(mt, G, mt.OP_SUM_F64, damping=D, eps=1e-9)
    assert oracle.relative_error(r.state(), oracle.pagerank(a, D)) <= 1e-6
    G.update(b.row_ptr, b.col)
    r = pull(mt, G, mt.OP_SUM_F64, damping=D, eps=1e-9, result=r)
    assert oracle.relative_error(r.state(), oracle.pagerank(b, D)) <= 1e-6


def test_pull_profile_mode_and_agreement_with_the_round_engine(mt):
    g = graphgen.rmat(14, 16)
    G = mt.Graph.from_csr(g)
    prof = pull(mt, G, mt.OP_SUM_MIXED, damping=D, eps=1e-8, flags=mt.FLAG_PROFILE_KERNELS)
    st = prof.stats()
    assert st["push_launches"] == st["rounds"] > 0 and st["push_ms"] > 0
    plain = pull(mt, G, mt.OP_SUM_MIXED, damping=D, eps=1e-8)
    sync = mt.run(G, mt.OP_SUM_MIXED, damping=D, eps=1e-8)
    vstar = oracle.pagerank(g, D)
    for v in (prof.state(), plain.state(), sync.state()):
        assert oracle.relative_error(v, vstar) <= 1e-6
    # strict Jacobi rounds, like the binned engine's: the same round count
    # (up to the rounding of the sums); the push engine needs fewer, since a
    # vertex pushed late in a round already takes what arrived earlier in it
    binned = mt.run(G, mt.OP_SUM_MIXED, damping=D, eps=1e-8, engine=mt.ENGINE_BINNED)
    assert plain.stats()["rounds"] == st["rounds"]
    assert abs(plain.stats()["rounds"] - binned.stats()["rounds"]) <= 1
    assert plain.stats()["rounds"] >= sync.stats()["rounds"]


def test_pull_refuses_what_it_does_not_serve(mt):
    g = graphgen.rmat(8, 4, weights=True)
    G = mt.Graph.from_csr(g)
    with pytest.raises(mt.MaiterError) as e:
        mt.run(G, mt.OP_MIN_U32, source=0, engine=mt.ENGINE_PULL)
    assert e.value.status == mt.ERR_UNSUPPORTED
    with pytest.raises(mt.MaiterError) as e:
        mt.run(G, mt.OP_SUM_F64, sched=mt.SCHED_TOPFRAC, top_frac=0.1, engine=mt.ENGINE_PULL)
    assert e.value.status == mt.ERR_UNSUPPORTED
    with pytest.raises(mt.MaiterError) as e:
        mt.run(G, mt.OP_SUM_F64, edge_coef=np.ones(g.m), engine=mt.ENGINE_PULL)
    assert e.value.status == mt.ERR_UNSUPPORTED
