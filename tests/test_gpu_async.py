"""The persistent asynchronous engine (device work queue, no inter-CTA barrier)
against the oracle, and its bounded waits.  Same tolerances as the round
engine: SSSP bit-exact, PageRank norm-wise relative error <= 1e-6."""
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


@pytest.mark.parametrize("scale,ef", [(6, 4), (10, 8), (13, 8)])
def test_async_pagerank_matches_oracle(mt, scale, ef):
    g = graphgen.rmat(scale, ef)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, damping=D, eps=1e-8, engine=mt.ENGINE_ASYNC)
    v = r.state()
    vstar = oracle.pagerank(g, D)
    assert oracle.relative_error(v, vstar) <= TOL
    st = r.stats()
    assert st["converged"] == 1 and st["residual"] < 1e-8
    # nothing was lost: the mass invariant holds at the end of an async run
    dangling = np.diff(g.row_ptr) == 0
    inv = oracle.pagerank_mass_invariant(v, r.delta(), v[dangling].sum(), g.n, D)
    assert abs(inv) < 1e-7 * g.n


def test_async_pagerank_threshold(mt):
    g = graphgen.rmat(13, 8)
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, eps=1e-8, engine=mt.ENGINE_ASYNC,
               sched=mt.SCHED_THRESHOLD, threshold=1e-3)
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= TOL


@pytest.mark.parametrize("scale,ef", [(6, 4), (11, 8), (14, 16)])
def test_async_sssp_bit_exact(mt, scale, ef):
    g = graphgen.rmat(scale, ef, weights=True)
    G = mt.Graph.from_csr(g)
    for s in graphgen.sssp_sources(g, 3):
        r = mt.run(G, mt.OP_MIN_U32, source=int(s), engine=mt.ENGINE_ASYNC)
        np.testing.assert_array_equal(r.state(), oracle.dijkstra(g, int(s)))


def test_async_sssp_full_size(mt):
    g = graphgen.rmat(20, 16, weights=True)
    G = mt.Graph.from_csr(g)
    r = None
    for s in graphgen.sssp_sources(g, 8)[:4]:
        r = mt.run(G, mt.OP_MIN_U32, source=int(s), engine=mt.ENGINE_ASYNC, result=r)
        np.testing.assert_array_equal(r.state(), oracle.dijkstra(g, int(s)))


def test_async_and_sync_share_a_result(mt):
    g = graphgen.rmat(12, 8, weights=True)
    G = mt.Graph.from_csr(g)
    s = int(graphgen.sssp_sources(g, 1)[0])
    r = mt.run(G, mt.OP_MIN_U32, source=s, engine=mt.ENGINE_ASYNC)
    a = r.state().copy()
    mt.run(G, mt.OP_MIN_U32, source=s, result=r)
    np.testing.assert_array_equal(a, r.state())


def test_bounded_wait_reports_timeout_and_state_resumes(mt):
    # A phantom pending item (injected on the host side of the queue's counter)
    # makes the idle warps wait; they give up after timeout_ms, the run returns
    # TIMEOUT, the context stays usable and the state is a valid DAIC state.
    g = graphgen.rmat(12, 8)
    G = mt.Graph.from_csr(g)
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_F64, eps=1e-9, engine=mt.ENGINE_ASYNC, timeout_ms=200,
               flags=mt.FLAG_INJECT_STALL)
    assert ei.value.status == mt.ERR_TIMEOUT
    r = mt.run(G, mt.OP_SUM_F64, eps=1e-9, engine=mt.ENGINE_ASYNC, timeout_ms=200,
               flags=mt.FLAG_INJECT_STALL, allow_not_converged=True)
    assert r.stats()["status"] == mt.ERR_TIMEOUT
    v, dl = r.state(), r.delta()
    # no delta was dropped by the interrupted launch
    dangling = np.diff(g.row_ptr) == 0
    assert abs(oracle.pagerank_mass_invariant(v, dl, v[dangling].sum(), g.n, D)) < 1e-7 * g.n
    # the context still works, and the state resumes to the fixed point
    x = torch.zeros(1, device="cuda")
    assert float((x + 1).item()) == 1.0
    r2 = mt.run(G, mt.OP_SUM_F64, v0=v, delta0=dl, eps=1e-9)
    assert oracle.relative_error(r2.state(), oracle.pagerank(g, D)) <= TOL


def test_async_rejects_unsupported(mt):
    g = graphgen.rmat(8, 4)
    G = mt.Graph.from_csr(g)
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_MIXED, engine=mt.ENGINE_ASYNC)
    assert ei.value.status == mt.ERR_UNSUPPORTED
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_F64, engine=mt.ENGINE_ASYNC, sched=mt.SCHED_TOPFRAC)
    assert ei.value.status == mt.ERR_UNSUPPORTED
