"""The learned priority scorer on the GPU: its BF16 inference and training
kernels against the FP64 reference, traces, and learned scheduling (fixed
point unchanged, work compared with the scheduler without the network)."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import mlp as ref

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


def rand_params(seed):
    return np.random.default_rng(seed).normal(0, 0.4, ref.N_PARAMS).astype(np.float32)


def rand_x(n, seed):
    return np.random.default_rng(seed).uniform(0, 4, (n, 8)).astype(np.float32)


def test_forward_matches_fp64_reference(mt):
    net = mt.MLP(params=rand_params(1))
    x = rand_x(5000, 2)
    got = net.forward(x)
    want = ref.forward(net.params(), x)
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-4)


def test_gradients_match_fp64_reference(mt):
    p = rand_params(3)
    net = mt.MLP(params=p)
    x = rand_x(3000, 4)
    y = np.random.default_rng(5).normal(size=3000).astype(np.float32)
    g, loss = net.gradients(x, y)
    gref, lref = ref.mse_gradients(p, x, y)
    assert abs(loss - lref) <= 1e-4 * max(1.0, lref)
    # FP32 accumulation vs FP64 (a unit exactly at the ReLU kink could flip)
    assert np.linalg.norm(g - gref) <= 1e-3 * np.linalg.norm(gref)


def test_training_fits_a_known_function(mt):
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 3, (20000, 8)).astype(np.float32)
    x[:, 7] = 0
    y = (np.maximum(x[:, 0] - x[:, 3], 0) + 0.5 * x[:, 1]).astype(np.float32)
    net = mt.MLP(seed=7)
    before = float(np.mean((net.forward(x) - y) ** 2))
    net.train(x, y, epochs=25, batch=512, lr=3e-3, seed=8)
    after = float(np.mean((net.forward(x) - y) ** 2))
    assert after < 0.05 * before and after < 0.02


def test_trace_records_features_of_sampled_vertices(mt):
    g = graphgen.rmat(11, 8)
    G = mt.Graph.from_csr(g)
    sample = np.arange(0, g.n, 7, dtype=np.int32)
    tr, res = mt.trace(G, mt.OP_SUM_F64, sample, 20, sched=mt.SCHED_TOPFRAC, top_frac=0.2,
                       eps=1e-8, damping=D)
    R = tr["features"].shape[0]
    assert 1 <= R <= 20
    # features are BF16 roundings of FP32 logarithms taken with the hardware
    # log (a few FP32 ulps from the exact value): one BF16 ulp of slack, plus
    # an absolute 2e-6 where the value is near 0
    ulp = dict(rtol=2.0 ** -7, atol=2e-6)
    deg = np.diff(g.row_ptr)[sample]
    np.testing.assert_allclose(tr["features"][0, :, 3], ref.bf16(np.log1p(deg)), **ulp)
    indeg = np.bincount(g.col, minlength=g.n)[sample]
    np.testing.assert_allclose(tr["features"][0, :, 2], ref.bf16(np.log1p(indeg)), **ulp)
    # magnitudes on a log scale: ln(max(x, 2^-100)) / 16 of |Delta| n and
    # |v| n, and f6 = (ln(max(|Delta| n, 2^-100)) - log1p(outdeg)) / 16, in
    # FP32, rounded to BF16
    def ln(x):
        return np.log(np.maximum(np.asarray(x, dtype=np.float32), np.float32(2.0 ** -100)))
    def b(x):
        return ref.bf16(np.asarray(x, dtype=np.float32) / np.float32(16)).astype(np.float32)
    dl, vs = np.abs(tr["delta"]), np.abs(tr["v"])
    ad = (dl * g.n).astype(np.float32)
    for k, want in ((0, b(ln(ad))), (1, b(ln((vs * g.n).astype(np.float32)))),
                    (6, b(ln(ad) - np.log1p(deg).astype(np.float32)))):
        np.testing.assert_allclose(tr["features"][:, :, k], want, **ulp, err_msg=f"feature {k}")
    assert (np.diff(tr["last_update"].astype(np.int64), axis=0) >= 0).all()
    # the traced run still reaches the fixed point
    assert oracle.relative_error(res.state(), oracle.pagerank(g, D)) <= 1e-6


@pytest.mark.parametrize("seed", [0, 1])
def test_learned_schedule_keeps_the_fixed_point_even_with_a_random_network(mt, seed):
    g = graphgen.rmat(12, 8, weights=True)
    G = mt.Graph.from_csr(g)
    net = mt.MLP(seed=seed)
    r = mt.run(G, mt.OP_SUM_F64, eps=1e-8, sched=mt.SCHED_LEARNED, top_frac=0.2, scorer=net)
    assert oracle.relative_error(r.state(), oracle.pagerank(g, D)) <= 1e-6
    s = int(graphgen.sssp_sources(g, 1)[0])
    r2 = mt.run(G, mt.OP_MIN_U32, source=s, sched=mt.SCHED_LEARNED, top_frac=0.2, scorer=net)
    np.testing.assert_array_equal(r2.state(), oracle.dijkstra(g, s))


def test_trained_scorer_gain_over_the_schedule_without_it(mt):
    """Train on traces of one graph, apply to another: same fixed point, and
    the work (messages) compared with top-fraction scheduling by |Delta|
    (the same selection without the network)."""
    from paper_1710_05785_b300 import learned
    gt = graphgen.rmat(13, 16, seed=11, weights=True)
    ga = graphgen.rmat(14, 16, seed=12, weights=True)
    Gt, Ga = mt.Graph.from_csr(gt), mt.Graph.from_csr(ga)
    out = {}
    # SSSP: learn "is this tentative distance final"
    st = int(graphgen.sssp_sources(gt, 1)[0])
    X, y = learned.collect(mt, Gt, gt.row_ptr, mt.OP_MIN_U32, source=st, top_frac=0.1, records=64)
    net, _ = learned.train(mt, X, y, epochs=20)
    sa = int(graphgen.sssp_sources(ga, 1)[0])
    base = mt.run(Ga, mt.OP_MIN_U32, source=sa, sched=mt.SCHED_TOPFRAC, top_frac=0.1)
    lrn = mt.run(Ga, mt.OP_MIN_U32, source=sa, sched=mt.SCHED_LEARNED, top_frac=0.1, scorer=net)
    np.testing.assert_array_equal(lrn.state(), oracle.dijkstra(ga, sa))
    out["sssp"] = (base.stats()["edge_pushes"], lrn.stats()["edge_pushes"])
    # PageRank: learn the mass moved per message at the next update
    X, y = learned.collect(mt, Gt, gt.row_ptr, mt.OP_SUM_F64, top_frac=0.1, records=96, eps=1e-8)
    net2, _ = learned.train(mt, X, y, epochs=20)
    base2 = mt.run(Ga, mt.OP_SUM_F64, eps=1e-8, sched=mt.SCHED_TOPFRAC, top_frac=0.1)
    lrn2 = mt.run(Ga, mt.OP_SUM_F64, eps=1e-8, sched=mt.SCHED_LEARNED, top_frac=0.1, scorer=net2)
    assert oracle.relative_error(lrn2.state(), oracle.pagerank(ga, D)) <= 1e-6
    out["pagerank"] = (base2.stats()["edge_pushes"], lrn2.stats()["edge_pushes"])
    print("messages (top-q by |Delta|, learned):", out)
    # measured: SSSP 740,546 -> 534,090 messages, PageRank 48.8M -> 21.9M
    for k, (b, l) in out.items():
        assert l < b, (k, b, l)
