"""Pins of the float-weight shortest-path oracle and of the log-normal
generator (the paper's synthetic workload, Section 6.1), against facts fixed
outside the oracle: IEEE single rounding worked by hand, the integer oracle
on integer-valued weights, brute-force relaxation, and the distribution the
generator samples."""
import math

import numpy as np
import pytest

import graphgen
import oracle


def test_float_distances_round_left_to_right_from_the_source():
    # 0 -1.0-> 1 -2^-24-> 2 -2^-24-> 3, and a direct edge 0 -> 3 of weight
    # next_after(1, 2) = 1 + 2^-23.  In single precision 1 + 2^-24 is a tie and
    # rounds to even (1.0), so the path reaches 3 at 1.0 (its exact sum would be
    # 1 + 2^-23): the path wins, and every vertex on it sits at 1.0.
    tiny = np.float32(2.0 ** -24)
    direct = np.nextafter(np.float32(1.0), np.float32(2.0))
    w = np.array([1.0, tiny, tiny, direct], dtype=np.float32)
    g = graphgen.small_graph(4, [(0, 1), (1, 2), (2, 3), (0, 3)], weights=w.view(np.uint32))
    d = oracle.dijkstra_f32(g, 0)
    assert d.dtype == np.float32
    np.testing.assert_array_equal(d, np.array([0.0, 1.0, 1.0, 1.0], dtype=np.float32))
    np.testing.assert_array_equal(oracle.bellman_ford_f32(g, 0), d)


def test_float_oracle_matches_integer_oracle_on_integer_weights():
    # small integers are exact in single precision and so are their sums below 2^24
    g = graphgen.rmat(10, 8, weights=True)
    gf = graphgen.CSRGraph(g.n, g.m, g.row_ptr, g.col, g.w.astype(np.float32).view(np.uint32))
    for s in graphgen.sssp_sources(g, 3):
        di = oracle.dijkstra(g, int(s))
        df = oracle.dijkstra_f32(gf, int(s))
        expect = np.where(di == oracle.INF32, np.inf, di.astype(np.float64)).astype(np.float32)
        np.testing.assert_array_equal(df, expect)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_float_dijkstra_matches_brute_force(seed):
    g = graphgen.lognormal(48, seed=seed, weights=True)
    for s in range(0, 48, 7):
        np.testing.assert_array_equal(oracle.dijkstra_f32(g, s), oracle.bellman_ford_f32(g, s))


def test_lognormal_generator_samples_its_distribution():
    n = 1 << 16
    mu, sigma = -0.5, 2.3
    g = graphgen.lognormal(n, weights=True)
    indeg = np.bincount(g.col, minlength=n)
    # P(round(X) = 0) = P(X < 1/2) = Phi((ln 1/2 - mu) / sigma)
    p0 = 0.5 * (1.0 + math.erf((math.log(0.5) - mu) / sigma / math.sqrt(2.0)))
    assert abs((indeg == 0).mean() - p0) < 0.01
    # P(round(X) >= 10) = P(X >= 9.5)
    p10 = 0.5 * math.erfc((math.log(9.5) - mu) / sigma / math.sqrt(2.0))
    assert abs((indeg >= 10).mean() - p10) < 0.01
    lw = np.log(graphgen.float_weights(g).astype(np.float64))
    assert abs(lw.mean()) < 0.01 and abs(lw.std() - 1.0) < 0.01
    # sources are uniform: the out-degrees' mean equals the in-degrees'
    assert g.m == indeg.sum() and abs(np.diff(g.row_ptr).mean() - g.m / n) < 1e-9
    # seeded: the same call gives the same graph
    h = graphgen.lognormal(n, weights=True)
    assert np.array_equal(h.col, g.col) and np.array_equal(h.w, g.w)
