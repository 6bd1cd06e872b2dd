"""The bench's own result checks (numpy, no oracle on the timed path) against
the oracle: they accept the exact answer and reject plausible wrong ones."""
import numpy as np

import bench
import graphgen
import oracle

D = 0.8


def test_sssp_check_accepts_dijkstra_and_rejects_perturbations():
    g = graphgen.rmat(10, 8, weights=True)
    s = int(graphgen.sssp_sources(g, 1)[0])
    d = oracle.dijkstra(g, s)
    assert bench.sssp_is_exact(g, s, d)
    fin = np.nonzero((d != 0xFFFFFFFF) & (np.arange(g.n) != s))[0]
    k = int(fin[len(fin) // 2])
    for delta in (+1, -1):
        bad = d.copy()
        bad[k] = np.uint32(int(bad[k]) + delta)
        assert not bench.sssp_is_exact(g, s, bad), delta
    unreach = np.nonzero(d == 0xFFFFFFFF)[0]
    if len(unreach):
        bad = d.copy()
        bad[unreach[0]] = 7
        assert not bench.sssp_is_exact(g, s, bad)
    bad = d.copy()
    bad[k] = 0xFFFFFFFF
    assert not bench.sssp_is_exact(g, s, bad)


def test_residual_bound_is_small_at_the_fixed_point_only():
    g = graphgen.rmat(10, 8)
    v = oracle.pagerank(g, D)
    c = oracle.pagerank_c(g.n, D)
    assert bench.linear_residual_bound(g, v, c, D) <= 1e-10
    seeds = graphgen.ppr_seed_sets(g.n, 1, seed=3)[0]
    vp = oracle.pagerank(g, D, seeds=seeds)
    assert bench.linear_residual_bound(g, vp, oracle.pagerank_c(g.n, D, seeds), D) <= 1e-10
    bad = v.copy()
    bad[int(np.argmax(v))] *= 1 + 1e-5
    assert bench.linear_residual_bound(g, bad, c, D) > 1e-6


def test_traffic_table_holds_every_capture_the_bench_lines_read():
    # the lines' roofline.traffic comes from these captures; a missing or
    # renamed key would turn it into null without an error
    tab = bench.load_traffic()
    for key in ("k_pull_pagerank_f32_rmat24", "k_push_pagerank_mixed_rmat24",
                "k_push_sssp_rmat20", "k_vec_pull_ppr64_rmat22"):
        assert isinstance(tab.get(key), int) and tab[key] > 0, key


def test_millisecond_workloads_default_to_regions_the_clock_sampler_sees():
    # every short workload has its own default step count, long enough for
    # several 50 ms sampler periods at its per-step time
    names = set(bench.PR_WORKLOADS) | set(bench.ROW_WORKLOADS) | {"sssp-rmat20"}
    assert set(bench.SHORT_STEPS) <= names
    assert all(steps >= 60 for steps in bench.SHORT_STEPS.values())
