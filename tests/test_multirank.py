"""The multi-rank path of bench.py on CPU (two gloo ranks, 127.0.0.1): each
rank takes its own consecutive slice of the seeded SSSP sources (independent
problems: together the ranks cover the first 8 x world sources exactly once),
the job time is the slowest rank's, and the whole-job value counts every
rank's edges.  No data-path collective exists to test: the sources share
nothing but the timing."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    import bench
    import graphgen
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=__import__("datetime").timedelta(seconds=60))
    try:
        g = graphgen.rmat(10, 4, weights=True)
        mine = bench.rank_sources(g, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        slowest = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        out.put((rank, gathered, slowest, bench.weak_value(slowest, g.m, world),
                 bench.rank_sources(g, 0, 1)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_sources_and_take_the_slowest_time():
    import bench
    import graphgen
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = graphgen.rmat(10, 4, weights=True)
    expect = [int(s) for s in graphgen.sssp_sources(g, bench.NSRC * world)]
    for rank, gathered, slowest, value, single in results:
        assert gathered[rank] == bench.rank_sources(g, rank, world)
        flat = [s for part in gathered for s in part]
        assert flat == expect and len(set(flat)) == len(flat)      # each source once
        assert all(len(part) == bench.NSRC for part in gathered)
        assert slowest == 2.5                                       # the slower rank
        np.testing.assert_allclose(value, bench.NSRC * g.m * world / 2.5e-3 / 1e9)
        # one rank alone runs the first NSRC of the same seeded list
        assert single == expect[:bench.NSRC]


def test_thread_errors_reach_the_caller():
    import bench
    done = []
    bench.run_in_threads([lambda: done.append(1), lambda: done.append(2)])
    assert sorted(done) == [1, 2]

    def boom():
        raise RuntimeError("step failed")
    with pytest.raises(RuntimeError, match="step failed"):
        bench.run_in_threads([lambda: None, boom])


def test_clock_summary_reports_median_clock_and_throttle_reasons():
    import bench
    c = bench.ClockSampler(0)
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    c.lines = ["0, 2032, 2032, 700.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2032, 1090.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2010, 2032, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2032.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2032, 500.0, 0x8, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                           "samples_in_region": 0}
    # the sample taken as the region starts counts in samples, not in the region's
    c.first = ["0, 2032, 2032, 600.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c.lines = c.first + ["0, 2032, 2032, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["samples"] == 2 and s["samples_in_region"] == 1
