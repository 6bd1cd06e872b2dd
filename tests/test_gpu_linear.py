"""The other linear rows of Table 1 on the GPU: the Katz metric (per-source
coefficient beta) and the Jacobi method (one signed coefficient per edge,
g_{i,j}(x) = -A_ji / A_jj x, Delta^1_j = b_j / A_jj, v^0 = 0; Section 4.3),
against the oracle's Katz fixed point and a direct solve of A x = b.

Tolerance: with termination at sum |Delta| < eps the remaining error is
(I - M)^{-1} Delta; the test matrices are row diagonally dominant by a factor
1.5, so ||(I - M)^{-1}||_inf <= 3 and every entry is within 3 eps (plus FP64
rounding of the accumulation)."""
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


def jacobi_inputs(n, rows, cols, vals, diag, b):
    """The DAIC form of Table 1's Jacobi row for A = diag + off-diagonal
    entries A[rows, cols] = vals: an edge i -> j with coefficient
    -A_ji / A_jj for every off-diagonal A_ji, in CSR order."""
    src, dst = cols, rows
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    coef = -vals[order] / diag[dst]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    g = graphgen.CSRGraph(n, len(src), row_ptr, dst.astype(np.int32), None)
    return g, coef, b / diag


def random_dominant(n, per_row, seed):
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n), per_row)
    cols = rng.integers(0, n, size=n * per_row)
    keep = rows != cols
    rows, cols = rows[keep], cols[keep]
    pairs = np.unique(np.stack([rows, cols], 1), axis=0)
    rows, cols = pairs[:, 0], pairs[:, 1]
    vals = rng.uniform(-1.0, 1.0, size=len(rows))
    diag = 1.5 * np.bincount(rows, weights=np.abs(vals), minlength=n) + 1.0
    b = rng.uniform(-1.0, 1.0, size=n)
    return rows, cols, vals, diag, b


@pytest.mark.parametrize("sched", [0, 1, 2])
def test_jacobi_matches_direct_solve(mt, sched):
    n = 1500
    rows, cols, vals, diag, b = random_dominant(n, 8, seed=5)
    A = np.diag(diag)
    A[rows, cols] = vals
    xstar = oracle.solve_linear_system(A, b)
    g, coef, d0 = jacobi_inputs(n, rows, cols, vals, diag, b)
    G = mt.Graph.from_csr(g)
    kw = {0: {}, 1: dict(sched=mt.SCHED_THRESHOLD, threshold=1e-4),
          2: dict(sched=mt.SCHED_TOPFRAC, top_frac=0.05)}[sched]
    r = mt.run(G, mt.OP_SUM_F64, edge_coef=coef, v0=np.zeros(n), delta0=d0, eps=1e-12, **kw)
    assert np.max(np.abs(r.state() - xstar)) <= 1e-10
    assert r.stats()["converged"] == 1


def test_jacobi_larger_sparse_system(mt):
    # 2^15 unknowns, about 16 off-diagonal entries a row; reference by the
    # plain Jacobi iteration to 1e-15 (spectral radius <= 2/3)
    n = 1 << 15
    rows, cols, vals, diag, b = random_dominant(n, 16, seed=9)
    x = b / diag
    for _ in range(120):
        r = b - np.bincount(rows, weights=vals * x[cols], minlength=n)
        x = r / diag
    g, coef, d0 = jacobi_inputs(n, rows, cols, vals, diag, b)
    G = mt.Graph.from_csr(g)
    out = mt.run(G, mt.OP_SUM_F64, edge_coef=coef, v0=np.zeros(n), delta0=d0, eps=1e-11)
    assert np.max(np.abs(out.state() - x)) <= 1e-9


def test_katz_matches_oracle_and_closed_form(mt):
    g = graphgen.rmat(12, 8)
    beta = 0.5 / float(np.diff(g.row_ptr).max())
    s = int(np.argmax(np.diff(g.row_ptr)))
    c = np.zeros(g.n)
    c[s] = 1.0
    G = mt.Graph.from_csr(g)
    r = mt.run(G, mt.OP_SUM_F64, coef=np.full(g.n, beta), v0=np.zeros(g.n), delta0=c, eps=1e-14)
    assert oracle.relative_error(r.state(), oracle.katz(g, beta, s)) <= 1e-9
    p = graphgen.small_graph(6, [(i, i + 1) for i in range(5)])
    c = np.zeros(6)
    c[0] = 1.0
    rp = mt.run(mt.Graph.from_csr(p), mt.OP_SUM_F64, coef=np.full(6, 0.3), v0=np.zeros(6),
                delta0=c, eps=1e-15)
    np.testing.assert_allclose(rp.state(), 0.3 ** np.arange(6), rtol=1e-13)


def test_per_edge_coefficients_rejections(mt):
    g = graphgen.rmat(8, 4)
    G = mt.Graph.from_csr(g)
    coef = np.full(g.m, 0.1)
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_MIXED, edge_coef=coef)
    assert ei.value.status == mt.ERR_INVALID_ARG
    with pytest.raises(mt.MaiterError) as ei:
        mt.run(G, mt.OP_SUM_F64, edge_coef=coef, engine=mt.ENGINE_ASYNC)
    assert ei.value.status == mt.ERR_UNSUPPORTED
