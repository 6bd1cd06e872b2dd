"""Pins of the oracle for the other rows of Table 1: the Katz metric (closed
forms on a path and a cycle), the linear system the Jacobi method solves (a
system worked by hand), and connected-components labels (by hand, by
transitive closure, and two independent algorithms on symmetric graphs)."""
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


def test_per_edge_iteration_solves_the_jacobi_system():
    # A = [[4, 1, 0], [2, 5, 1], [0, 1, 3]], b = [1, 2, 3]: the Jacobi form has an
    # edge j -> k with coefficient -A_kj / A_kk for each off-diagonal A_kj
    A = np.array([[4.0, 1.0, 0.0], [2.0, 5.0, 1.0], [0.0, 1.0, 3.0]])
    b = np.array([1.0, 2.0, 3.0])
    edges, coef = [], []
    for j in range(3):
        for k in range(3):
            if k != j and A[k, j] != 0.0:
                edges.append((j, k))
                coef.append(-A[k, j] / A[k, k])
    g = graphgen.small_graph(3, edges)   # rows sorted by target, as listed above
    x, it = oracle.linear_power_edges(g, np.array(coef), b / np.diag(A))
    np.testing.assert_allclose(x, oracle.solve_linear_system(A, b), rtol=1e-12)
    # the definition itself: A x = b
    np.testing.assert_allclose(A @ x, b, rtol=1e-12)
    assert it > 1


def test_per_edge_iteration_equals_per_source_when_coefficients_agree():
    g = graphgen.rmat(9, 4)
    coef_src = np.where(np.diff(g.row_ptr) > 0, 0.8 / np.maximum(np.diff(g.row_ptr), 1), 0.0)
    ecoef = np.repeat(coef_src, np.diff(g.row_ptr))
    c = np.full(g.n, 0.2)
    a, _ = oracle.linear_power_edges(g, ecoef, c)
    b, _ = oracle.linear_power(g, coef_src, c)
    np.testing.assert_allclose(a, b, rtol=1e-11)


# ------------------------------------------ connected components (Table 1)

def test_component_labels_by_hand():
    # {0, 1, 2} joined both ways, {3, 4}, and 5 alone
    e = [(0, 1), (1, 0), (1, 2), (2, 1), (3, 4), (4, 3)]
    g = graphgen.small_graph(6, e)
    np.testing.assert_array_equal(oracle.max_reach_labels(g), [2, 2, 2, 4, 4, 5])
    np.testing.assert_array_equal(oracle.component_labels(g), [2, 2, 2, 4, 4, 5])


def test_max_reach_follows_edge_direction():
    up = graphgen.small_graph(3, [(0, 1), (1, 2)])
    down = graphgen.small_graph(3, [(2, 1), (1, 0)])
    np.testing.assert_array_equal(oracle.max_reach_labels(up), [0, 1, 2])
    np.testing.assert_array_equal(oracle.max_reach_labels(down), [2, 2, 2])


def test_max_reach_by_transitive_closure_and_union_find():
    for trial in range(6):
        n = 24
        g = graphgen.random_graph(n, 30, seed=trial)
        # brute force: reachability by repeated boolean products
        R = np.eye(n, dtype=bool)
        A = np.zeros((n, n), dtype=bool)
        for j in range(n):
            A[j, g.col[g.row_ptr[j]:g.row_ptr[j + 1]]] = True
        for _ in range(n):
            R = R | (R.astype(np.int64) @ A.astype(np.int64) > 0)
        expect = np.array([np.nonzero(R[:, j])[0].max() for j in range(n)], dtype=np.int32)
        np.testing.assert_array_equal(oracle.max_reach_labels(g), expect)
        s = graphgen.symmetrize(g)
        np.testing.assert_array_equal(oracle.max_reach_labels(s), oracle.component_labels(s))
