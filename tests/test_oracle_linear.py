"""Pins of the oracle for the other linear rows of Table 1: the Katz metric
(closed forms on a path and a cycle) and the linear system the Jacobi method
solves (a system worked by hand)."""
import numpy as np

import graphgen
import oracle


def test_katz_on_a_path_is_powers_of_beta():
    # 0 -> 1 -> 2 -> 3 -> 4: one path of length k reaches k, so x_k = beta^k
    g = graphgen.small_graph(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    beta = 0.3
    np.testing.assert_allclose(oracle.katz(g, beta, 0), beta ** np.arange(5), rtol=1e-12)


def test_katz_on_a_cycle_sums_the_geometric_series():
    # on a directed n-cycle the paths from 0 to k have lengths k, k + n, ...
    n, beta = 7, 0.6
    g = graphgen.small_graph(n, [(i, (i + 1) % n) for i in range(n)])
    expect = beta ** np.arange(n) / (1.0 - beta ** n)
    np.testing.assert_allclose(oracle.katz(g, beta, 0), expect, rtol=1e-12)


def test_katz_counts_multi_edges_and_branches():
    # 0 -> 1 twice, 0 -> 2, 1 -> 2: two paths 0-1 (length 1), paths to 2 of
    # length 1 (once) and 2 (twice)
    g = graphgen.small_graph(3, [(0, 1), (0, 1), (0, 2), (1, 2)])
    b = 0.25
    np.testing.assert_allclose(oracle.katz(g, b, 0), [1.0, 2 * b, b + 2 * b * b], rtol=1e-12)


def test_linear_system_solution_by_hand():
    # [[4, 1], [2, 3]] x = [1, 2]: det 10, x = (1*3 - 1*2, 4*2 - 2*1) / 10
    x = oracle.solve_linear_system([[4.0, 1.0], [2.0, 3.0]], [1.0, 2.0])
    np.testing.assert_allclose(x, [0.1, 0.6], rtol=1e-14)
