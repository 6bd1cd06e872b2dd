"""The seeded input generator: determinism, sizes, and the R-MAT distribution."""
import numpy as np

import graphgen


def test_rmat_deterministic_and_exact_size():
    a = graphgen.rmat(10, 8, weights=True)
    b = graphgen.rmat(10, 8, weights=True)
    assert a.n == 1024 and a.m == 8192 and a.row_ptr[-1] == a.m
    np.testing.assert_array_equal(a.row_ptr, b.row_ptr)
    np.testing.assert_array_equal(a.col, b.col)
    np.testing.assert_array_equal(a.w, b.w)
    assert (np.diff(a.row_ptr) >= 0).all()
    assert a.col.min() >= 0 and a.col.max() < a.n
    assert a.w.min() >= 1 and a.w.max() <= 255


def test_rmat_seed_changes_graph():
    a = graphgen.rmat(10, 8, seed=1)
    b = graphgen.rmat(10, 8, seed=2)
    assert not np.array_equal(a.col, b.col)


def test_rmat_quadrant_frequencies():
    # top-level bit of (src, dst) before relabelling follows (a, b, c, d)
    scale = 14
    src, dst = graphgen.rmat_edges(scale, 16, seed=3)
    hs = (src >> (scale - 1)) & 1
    hd = (dst >> (scale - 1)) & 1
    q = 2 * hs + hd
    freq = np.bincount(q, minlength=4) / q.size
    np.testing.assert_allclose(freq, [0.57, 0.19, 0.19, 0.05], atol=0.005)


def test_rmat_skewed_degrees():
    g = graphgen.rmat(16, 16)
    deg = np.diff(g.row_ptr)
    assert deg.max() > 50 * deg.mean()
    assert (deg == 0).mean() > 0.2          # dangling vertices kept


def test_csr_is_canonical_under_edge_order():
    src = np.array([3, 1, 3, 0, 3], dtype=np.int32)
    dst = np.array([2, 0, 1, 3, 2], dtype=np.int32)
    w = np.array([5, 6, 7, 8, 1], dtype=np.uint32)
    g1 = graphgen.csr_from_edges(4, src, dst, w)
    p = np.array([4, 2, 0, 1, 3])
    g2 = graphgen.csr_from_edges(4, src[p], dst[p], w[p])
    np.testing.assert_array_equal(g1.col, g2.col)
    np.testing.assert_array_equal(g1.w, g2.w)
    np.testing.assert_array_equal(g1.row_ptr, [0, 1, 2, 2, 5])
    np.testing.assert_array_equal(g1.col[2:], [1, 2, 2])
    np.testing.assert_array_equal(g1.w[2:], [7, 1, 5])


def test_permutation_is_a_permutation():
    p = graphgen.permutation(1000, 9)
    np.testing.assert_array_equal(np.sort(p), np.arange(1000))


def test_sources_and_seed_sets():
    g = graphgen.rmat(12, 16)
    s = graphgen.sssp_sources(g, 8)
    assert len(set(s.tolist())) == 8
    assert (g.outdeg[s] >= 16).all()
    sets = graphgen.ppr_seed_sets(g.n, 200, seed=4)
    sizes = np.array([len(x) for x in sets])
    assert sizes.min() >= 1 and sizes.max() <= 64
    assert all(len(set(x.tolist())) == len(x) for x in sets)
    # log-uniform: about half of the sizes are <= 8 (= sqrt(64))
    assert 0.35 < (sizes <= 8).mean() < 0.65
