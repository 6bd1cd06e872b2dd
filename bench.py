"""Benchmark of DAIC delta propagation on one B300.

Default workload: PageRank in DAIC form (d = 0.8, v0 = 0, Delta1 = 0.2) on a
seeded R-MAT graph of scale 24, edge factor 16 (16.8 M vertices, 268 M
edges), FP32 deltas and messages with FP64 state and residual reduction, run
to sum |Delta| < 4e-8 on the receive-side engine; one step = one run from the
initial state to the tolerance.  Metric: GTEPS = m / time-to-tolerance, with
the graph resident in HBM.  Beside it: the plain FP64 form and the other
engines and precisions as checked variants, the dominant kernel's fraction of
the measured HBM copy bandwidth (and the push kernel's), an end-to-end figure
through the C ABI from pinned host buffers, the CPU oracle on the machine's host
and the clocks seen during the timed region.  The SSSP record (R-MAT scale
20, 8 sources one after another, exact) is nested in the same line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload NAME]

Multi-GPU (torchrun): the runs are independent problems, so each rank runs
its own copy (weak scaling, no collective on the data path; a barrier and a
max over ranks frame the timing).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402

METRIC = "GTEPS and time-to-tolerance (1e-6 / exact) vs plain form, % of HBM roofline"
SCALE, EF, NSRC = 20, 16, 8
# algorithmic bytes of the SSSP push kernel (an atomic read-modify-write counts
# as a read plus a write):
#   per edge push:      4 B target + 4 B weight + 8 B Delta_k RMW       = 16 B
#   per updated vertex: 8 B row offsets + 8 B Delta_j + 8 B v_j RMW     = 24 B
BYTES_PER_EDGE = 16
BYTES_PER_VERTEX = 24
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def random_access(mt, kind, n, device, edge_ops, push_ms, what):
    """The push's edge loop against the rate this device sustains for
    single-word operations at random addresses of an array of Delta's size
    (maiter_probe_random_rate, measured now): every edge push makes one such
    operation on Delta_k, so this is the ceiling of the edge loop while Delta
    fits in L2, where the DRAM roofline says little."""
    lg = max(10, min(28, int(np.ceil(np.log2(max(n, 2))))))
    ceiling = mt.probe_random_rate(kind, lg, device)
    achieved = edge_ops / (push_ms * 1e-3) / 1e9
    return {"achieved_gops": achieved, "ceiling_gops": ceiling,
            "frac": achieved / ceiling if ceiling > 0 else None,
            "ceiling_kind": f"measured: {what} at random addresses of 2^{lg} words",
            "unit": "G edge pushes/s vs G ops/s"}


def rank_sources(g, rank, world):
    """This rank's NSRC sources: the first NSRC * world seeded sources of the
    graph, cut into consecutive slices in rank order (independent problems,
    so ranks share nothing but the timing)."""
    all_src = graphgen.sssp_sources(g, NSRC * world)
    return [int(s) for s in all_src[rank * NSRC:(rank + 1) * NSRC]]


def max_over_ranks(x, dist, device):
    """The slowest rank's value (the job ends when its last rank does)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(ms_per_step, m, world):
    """Whole-job GTEPS: every rank's NSRC sources over the slowest rank's time."""
    return NSRC * m * world / (ms_per_step * 1e-3) / 1e9


def run_in_threads(fns):
    """Runs each callable on a thread of its own and waits for all of them;
    an exception on any thread is raised here (a failed step must not leave
    a throughput figure behind)."""
    import threading
    errors = []

    def wrap(fn):
        try:
            fn()
        except BaseException as e:  # noqa: BLE001 - re-raised on the caller's thread
            errors.append(e)

    threads = [threading.Thread(target=wrap, args=(fn,)) for fn in fns]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region (every 50 ms).  The timed region starts only once the first sample
    is in, so a region shorter than the interval still has the sample taken
    at its start; `samples_in_region` counts those taken after it began."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.first = []

    def __enter__(self):
        import select
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        if self.proc is not None:
            ready, _, _ = select.select([self.proc.stdout], [], [], 10.0)
            if ready:
                line = self.proc.stdout.readline()
                if line.strip():
                    self.first = [line]
        return self

    def __exit__(self, *exc):
        self.lines = list(self.first)
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines += [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sm),
                "samples_in_region": max(0, len(sm) - len(self.first))}


def cpu_baseline(g, sources, budget_s=25.0):
    """The oracle as it stands (Dijkstra, binary heap, one core) on a bounded
    sample of the same workload: as many of the sources as fit the budget."""
    import oracle
    oracle.dijkstra(g, int(sources[0]))  # load the library, warm the caches
    t0 = time.perf_counter()
    done = 0
    for s in sources:
        oracle.dijkstra(g, int(s))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done * g.m / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"Dijkstra from {done} of the {len(sources)} sources on the full "
                      f"R-MAT scale-{SCALE} graph ({dt:.1f} s)"}


def run_reference(args):
    """Reference arm: the CPU oracle on the host cores, one bounded sample of
    the workload per step.  PageRank workloads: one synchronous iteration of
    the oracle over the full graph per step, the iterations to tolerance
    projected from the measured residual decay; SSSP: Dijkstra from one source
    per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    if args.workload in PR_WORKLOADS:
        cfg = dict(PR_WORKLOADS[args.workload])
        if args.scale:
            cfg["scale"] = args.scale
        g = graphgen.rmat(cfg["scale"], cfg["ef"])
        per_iter, n_tol, done = oracle_pagerank_sample(g, D_PR, cfg["eps"], iters=args.steps,
                                                       warmup=args.warmup)
        ms = per_iter * n_tol * 1e3
        value = g.m / (ms * 1e-3) / 1e9
        sample = (f"{done} synchronous iterations of the oracle over the full graph, one per "
                  f"step ({per_iter:.2f} s each, one core); {n_tol} iterations to tolerance "
                  f"projected from the measured residual decay")
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": pagerank_config(args.workload, cfg, g, 1),
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    g = graphgen.rmat(SCALE, EF, weights=True)
    sources = graphgen.sssp_sources(g, NSRC)
    for k in range(args.warmup):
        oracle.dijkstra(g, int(sources[k % NSRC]))
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.dijkstra(g, int(sources[k % NSRC]))
    dt = time.perf_counter() - t0
    value = args.steps * g.m / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": sssp_config(g, 1),
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": "Dijkstra from one source of the full graph per step"},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def sssp_config(g, world):
    return {"workload": f"sssp-rmat{SCALE}-ef{EF}-{NSRC}src: SSSP in DAIC form, weights u32 "
                        f"uniform [1, 255], {NSRC} sources one after another, exact",
            "n": g.n, "m": g.m, "sources_per_rank": NSRC,
            "l2": f"{L2_FLUSH_BYTES >> 20} MiB write between steps (outside the events)",
            "parallelism": f"independent sources x{world}"}


def load_traffic():
    """profiles/traffic.json: DRAM bytes (read + write) per launch of the
    captured kernels, by capture name ({} when the file is absent)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


PR_WORKLOADS = {
    # FP64 PageRank on R-MAT scale 13, to sum |Delta| < 1e-8
    "pagerank-rmat13": dict(scale=13, ef=8, op="f64", eps=1e-8),
    # mixed precision at R-MAT scale 24: FP32 deltas / FP64 state and residual; eps = 4e-8
    # bounds the per-entry relative error by 25 * eps = 1e-6 (v* >= 1 - d)
    "pagerank-mixed-rmat24": dict(scale=24, ef=16, op="mixed", eps=4e-8),
}
# algorithmic bytes of a PageRank message and of a vertex update (an atomic
# or any read-modify-write counts as a read plus a write):
#   FP64 deltas:  4 B target + 16 B Delta_k RMW = 20 B per message;
#                 8 B offsets + 16 B Delta_j take + 16 B v_j RMW = 40 B per update
#   FP32 deltas:  4 + 8 = 12 B per message; 8 + 8 + 16 = 32 B per update
PR_BYTES = {"f64": (20, 40), "f32": (12, 32)}
D_PR = 0.8


def pagerank_alg_bytes(st, mixed):
    """Algorithmic bytes of a run's messages and updates (per the table above);
    a mixed run's FP64 warm-up phase is counted at the FP64 rates."""
    if not mixed:
        return PR_BYTES["f64"][0] * st["edge_pushes"] + PR_BYTES["f64"][1] * st["activations"]
    w_e, w_v = st["warm_edge_pushes"], st["warm_activations"]
    return (PR_BYTES["f64"][0] * w_e + PR_BYTES["f64"][1] * w_v
            + PR_BYTES["f32"][0] * (st["edge_pushes"] - w_e)
            + PR_BYTES["f32"][1] * (st["activations"] - w_v))


def oracle_pagerank_sample(g, d, eps, budget_s=None, iters=None, warmup=0):
    """The oracle's synchronous iteration (Eq. 1) from v = 0 on the full graph,
    one iteration being v <- v + r with r = c + P^T v - v (the oracle's
    residual routine, one core), timed per iteration.  Runs `iters`
    iterations (after `warmup` untimed ones) or as many as fit `budget_s`.
    The iterations to ||r||_1 < eps are counted if reached, else projected
    from the measured geometric decay of ||r||_1 over the last iterations.
    Returns (seconds per iteration, iterations to tolerance, iterations run)."""
    import oracle
    coef = oracle.pagerank_coef(g, d)
    c = oracle.pagerank_c(g.n, d)
    v = np.zeros(g.n)
    norms, times = [], []
    t_start = time.perf_counter()
    k = 0
    while True:
        t0 = time.perf_counter()
        r = oracle.linear_residual(g, coef, c, v)
        v += r
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
        norms.append(float(np.abs(r).sum()))
        k += 1
        if norms[-1] < eps:
            break
        if iters is not None and k >= warmup + iters:
            break
        if budget_s is not None and time.perf_counter() - t_start > budget_s and k >= 3:
            break
    per_iter = float(np.median(times)) if times else dt
    # iteration i computes r from v^i, so r is below eps once i = len - 1 holds;
    # the run needs that many iterations plus the one that meets the test
    if norms[-1] < eps:
        n_tol = len(norms)
    else:
        span = min(4, len(norms) - 1)
        rho = (norms[-1] / norms[-1 - span]) ** (1.0 / span)
        n_tol = len(norms) + int(np.ceil(np.log(eps / norms[-1]) / np.log(rho)))
    return per_iter, n_tol, len(times)


def pagerank_cpu_baseline(g, d, eps, budget_s=15.0):
    per_iter, n_tol, done = oracle_pagerank_sample(g, d, eps, budget_s=budget_s)
    return {"value": g.m / (per_iter * n_tol) / 1e9, "unit": "GTEPS", "cores": 1,
            "kind": "oracle",
            "sample": f"{done} synchronous iterations of the oracle (Eq. 1) over the full graph, "
                      f"{per_iter:.2f} s each on one core; {n_tol} iterations to "
                      f"sum |r| < {eps:g} projected from the measured decay of the residual"}


def pagerank_config(wl, cfg, g, world):
    """The workload as both arms of the bench name it."""
    return {"workload": f"{wl}: PageRank in DAIC form, d = 0.8, v0 = 0, Delta1 = 0.2, R-MAT "
                        f"scale {cfg['scale']} edge factor {cfg['ef']}, to sum |Delta| < "
                        f"{cfg['eps']:g}",
            "n": g.n, "m": g.m, "eps": cfg["eps"],
            "l2": f"inputs larger than L2 (CSR {(4 * g.m + 4 * g.n) / 1e9:.2f} GB); the GPU arm "
                  f"also writes {L2_FLUSH_BYTES >> 20} MiB before every run",
            "parallelism": f"independent replicas x{world}"}


def run_pagerank(args, wl, dist=None, nested=None):
    """PageRank workloads: one step = one run from v0 = 0, Delta1 = 1 - d to
    sum |Delta| < eps; value = m / time-to-tolerance (GTEPS per solution).
    The headline at scale 24 is the receive-side engine with FP32 deltas and
    messages (FP64 state and residual); beside it the plain form (FP64 round
    engine), the round engine in mixed precision, the receive-side engine in
    the other precisions, the binned engine and top-q scheduling."""
    import torch
    import paper_1710_05785_b300 as mt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cfg = dict(PR_WORKLOADS[wl])
    if args.scale:
        cfg["scale"] = args.scale   # a smaller case of the same kernels (profiling)
    mixed = cfg["op"] == "mixed"
    g = graphgen.rmat(cfg["scale"], cfg["ef"])
    G = mt.Graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev), device=local)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    eps = cfg["eps"]
    # the headline: the receive-side engine (every receiver sums its
    # in-messages over the transpose: no atomic per edge) with FP32 deltas
    # and messages from the first round (no delta accumulates under atomics,
    # so no FP64 warm-up is needed); beside it the plain form (FP64), the
    # round engine (frontier scan + push with L2 atomics) in mixed precision,
    # the binned engine and top-q
    head = "pull_f32" if mixed else "plain_f64_sync"
    variants = {
        "pull_f32": dict(op=mt.OP_SUM_MIXED, engine=mt.ENGINE_PULL, mixed_switch=1.0),
        "mixed_sync": dict(op=mt.OP_SUM_MIXED),
        "plain_f64_sync": dict(op=mt.OP_SUM_F64),
        "pull_mixed": dict(op=mt.OP_SUM_MIXED, engine=mt.ENGINE_PULL),
        "pull_f64": dict(op=mt.OP_SUM_F64, engine=mt.ENGINE_PULL),
        "binned_f32": dict(op=mt.OP_SUM_MIXED, engine=mt.ENGINE_BINNED, mixed_switch=1.0),
        "f64_topq10_sync": dict(op=mt.OP_SUM_F64, sched=mt.SCHED_TOPFRAC, top_frac=0.1),
    }
    if not mixed:
        del variants["pull_f32"]
    variants["f64_async"] = dict(op=mt.OP_SUM_F64, engine=mt.ENGINE_ASYNC)
    if args.head_only:
        variants = {head: variants[head]}
    res = {}
    states = {}

    def one(name, kw, record=None):
        r = mt.run(G, eps=eps, damping=D_PR, stream=stream.cuda_stream, result=res.get(name),
                   **kw)
        res[name] = r
        return r.stats()

    # the headline: W warm-up runs, then K timed runs (device events on the
    # launching stream, max over ranks), an L2 flush before each
    for _ in range(max(args.warmup, 1)):
        flush.fill_(1)
        one(head, variants[head])
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(k)
            ev[k][0].record(stream)
            stats.append(one(head, variants[head]))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, dev)
    ms = total_ms / args.steps
    hs = stats[-1]
    if not all(s["converged"] == 1 and s["residual"] < eps for s in stats):
        raise RuntimeError("a timed PageRank run did not reach its tolerance")
    v_head = res[head].state()
    results = {head: dict(time_to_tolerance_ms=ms, rounds=hs["rounds"],
                          edge_pushes=hs["edge_pushes"], residual=hs["residual"],
                          kernel_launches=hs["kernel_launches"])}
    for name, kw in variants.items():
        if name == head:
            continue
        reps = 2
        one(name, kw)
        best = None
        for _ in range(reps):
            flush.fill_(1)
            st = one(name, kw)
            best = st if best is None or st["elapsed_ms"] < best["elapsed_ms"] else best
        results[name] = dict(time_to_tolerance_ms=best["elapsed_ms"], rounds=best["rounds"],
                             edge_pushes=best["edge_pushes"], residual=best["residual"],
                             kernel_launches=best["kernel_launches"])
        states[name] = res[name].state()
        res[name].close()
        del res[name]
    plain_t = results["plain_f64_sync"]["time_to_tolerance_ms"] if "plain_f64_sync" in results else None
    # Checks without the oracle.  An FP64 state is bounded by its own residual,
    # ||v* - v||_1 <= ||c + P^T v - v||_1 / (1 - d); for states with FP32
    # rounding that L1 bound sums the rounding of every vertex, so they are
    # bounded through the FP64 one: max|v - v*| <= max|v - v_f64| + bound_f64.
    v_f64 = v_head if not mixed else states.get("plain_f64_sync")
    if v_f64 is None:
        v_f64 = mt.run(G, op=mt.OP_SUM_F64, eps=eps, damping=D_PR,
                       stream=stream.cuda_stream).state()
    bound_f64 = linear_residual_bound(g, v_f64, np.full(g.n, 1 - D_PR), D_PR)

    def error_bound(v):
        return float(np.abs(v - v_f64).max() / v_f64.max()) + bound_f64

    for name, v in [(head, v_head)] + list(states.items()):
        results[name]["error_bound"] = error_bound(v)
        if results[name]["error_bound"] > 1e-6:
            raise RuntimeError(f"PageRank result of {name} misses the 1e-6 bound: "
                               f"{results[name]['error_bound']:.3g}")
    bound = results[head]["error_bound"]
    # kernel-level roofline: the headline run again with per-kernel events
    peaks, peak_kind = measured_peaks()
    traffic_tab = load_traffic()

    def kernel_roofline(kw, kernel, kind, what, traffic_key, note):
        pf = mt.run(G, eps=eps, damping=D_PR, stream=stream.cuda_stream,
                    flags=mt.FLAG_PROFILE_KERNELS, **kw).stats()
        is_mixed = kw["op"] == mt.OP_SUM_MIXED
        alg = pagerank_alg_bytes(pf, is_mixed)
        launches = max(pf["push_launches"], 1)
        achieved = alg / (pf["push_ms"] * 1e-3) / 1e9
        out = {"bound": "hbm", "kernel": kernel,
               "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": achieved / peaks["hbm_gbs"], "traffic": traffic_tab.get(traffic_key),
               "peak_kind": f"{peak_kind} copy bandwidth",
               "launches": pf["push_launches"],
               "ms_per_launch": pf["push_ms"] / launches,
               "alg_bytes_per_launch": alg / launches,
               "random_access": random_access(mt, kind, g.n, local, pf["edge_pushes"],
                                              pf["push_ms"], what),
               "note": note}
        if pf["scan_launches"]:
            out["scan_ms_per_launch"] = pf["scan_ms"] / pf["scan_launches"]
        return out

    if head == "pull_f32":
        roofline = kernel_roofline(
            variants[head], "k_pull<float,float> (a warp per 32 receivers or per 1024-edge "
            "chunk of a receiver of in-degree > 256)", mt.PROBE_LOAD_32,
            "32-bit loads", f"k_pull_pagerank_f32_rmat{cfg['scale']}",
            "achieved = algorithmic bytes (12 B per FP32 message, 32 B per update, the same "
            "definition as the push's) / device time of the pull launches")
        push_roofline = None if "mixed_sync" not in variants else kernel_roofline(
            variants["mixed_sync"], "k_push<OpSumMixed> (warm-up rounds k_push<OpSumWarm>)",
            mt.PROBE_RED_F32, "f32 atomicAdd", f"k_push_pagerank_mixed_rmat{cfg['scale']}",
            "achieved = algorithmic bytes of the push (12 B per FP32 message, 32 B per update; "
            "FP64 warm-up rounds at 20 / 40 B) / device time of the push launches")
    else:
        roofline = kernel_roofline(
            variants[head], "k_push<OpSumF64>", mt.PROBE_RED_F64, "f64 atomicAdd",
            f"k_push_pagerank_f64_rmat{cfg['scale']}",
            "achieved = algorithmic bytes of the push (20 B per FP64 message, 40 B per update) "
            "/ device time of the push launches")
        push_roofline = None
    bprof = None
    if "binned_f32" in variants:
        bp = mt.run(G, eps=eps, damping=D_PR, stream=stream.cuda_stream,
                    flags=mt.FLAG_PROFILE_KERNELS, **variants["binned_f32"]).stats()
        br = max(bp["push_launches"], 1)
        balg = pagerank_alg_bytes(bp, True)
        bprof = {"kernel": "k_bin_scatter + k_bin_gather (FP32 deltas, exact 64-bit sums)",
                 "achieved": balg / (bp["push_ms"] * 1e-3) / 1e9,
                 "frac": balg / (bp["push_ms"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                 "rounds": bp["push_launches"], "scatter_ms_per_round": bp["bin_scatter_ms"] / br,
                 "gather_ms_per_round": bp["bin_gather_ms"] / br, "slots": bp["slots"],
                 "l2_atomics_per_edge": 0}
    e2e = None if args.no_e2e else pagerank_e2e(mt, g, G, eps, variants[head], dev, local, world,
                                                 args, error_bound)
    line = {
        "metric": METRIC, "value": world * g.m / (ms * 1e-3) / 1e9, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if mixed else "f64", "data": "synthetic",
        "config": pagerank_config(wl, cfg, g, world),
        "headline": head,
        "engine": ("receive-side engine: every receiver sums the messages of its in-neighbours "
                   "over the transpose (no atomic per edge), then folds; CUDA graph with a "
                   "device-side WHILE") if head == "pull_f32" else
                  "round engine: frontier scan + degree-bucketed push with L2 atomics; CUDA "
                  "graph with a device-side WHILE",
        "precision": ("FP32 deltas and messages from the first round; FP64 state and residual "
                      "reduction") if mixed else "FP64",
        "time_to_tolerance_ms": ms,
        "vs_plain_form": plain_t / ms if plain_t else None,
        "error_bound": bound,
        "variants": results,
        "gteps_work": hs["edge_pushes"] / (ms * 1e-3) / 1e9,
        "roofline": roofline,
        "push_roofline": push_roofline,
        "binned_roofline": bprof,
        "e2e": e2e,
        # every timed run's kernels, + one L2 flush fill per step
        "gpu_launches": int(sum(x["kernel_launches"] for x in stats)) + args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = pagerank_cpu_baseline(g, D_PR, eps)
    for r in res.values():
        r.close()
    G.close()
    del G, flush
    torch.cuda.empty_cache()
    if nested is not None:
        line.update(nested(dist))
    if rank == 0:
        print(json.dumps(line), flush=True)


def pagerank_e2e(mt, g, G0, eps, kw, dev, local, world, args, error_bound):
    """End to end through the C ABI from pinned host buffers, per step: the CSR
    uploaded into a graph's buffers (maiter_graph_update; the binned layout is
    rebuilt from it), the run, and every state read back into pinned memory.
    Two steps in flight, each on its own graph, result and stream driven by
    its own host thread, with a lock that keeps the runs one after another."""
    import threading
    import torch
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    h2d = rp_h.numel() * 8 + col_h.numel() * 4
    d2h = g.n * 8
    slots = []
    for _ in range(2):
        s_k = torch.cuda.Stream(dev)
        G_k = mt.Graph(rp_h, col_h, device=local)
        r_k = mt.run(G_k, eps=eps, damping=D_PR, stream=s_k.cuda_stream, **kw)
        slots.append({"G": G_k, "s": s_k, "r": r_k,
                      "out": torch.empty(g.n, dtype=torch.float64).pin_memory()})
    torch.cuda.synchronize()
    lock = threading.Lock()

    def e2e_step(sl):
        sl["G"].update(rp_h, col_h, stream=sl["s"].cuda_stream)
        with lock:
            sl["r"] = mt.run(sl["G"], eps=eps, damping=D_PR, stream=sl["s"].cuda_stream,
                             result=sl["r"], **kw)
        sl["r"].state(sl["out"])

    per = max(1, min(args.steps, 4))
    t0 = time.perf_counter()
    for _ in range(per):
        e2e_step(slots[0])
    serial_s = (time.perf_counter() - t0) / per
    t0 = time.perf_counter()
    run_in_threads([lambda sl=sl: [e2e_step(sl) for _ in range(per)] for sl in slots])
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / (2 * per)
    bound = error_bound(slots[1]["out"].numpy())
    if bound > 1e-6:
        raise RuntimeError(f"end-to-end PageRank result misses the 1e-6 bound: {bound:.3g}")
    for sl in slots:
        sl["r"].close()
        sl["G"].close()
    return {"value": world * g.m / e2e_s / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps_in_flight": 2,
            "one_step_at_a_time": world * g.m / serial_s / 1e9,
            "ms_per_step": e2e_s * 1e3}


BATCH_SCALES = [16, 17, 18, 19, 20, 21, 22, 22]   # the last scale-22 graph on a second seed


def batch_workload(scales=BATCH_SCALES, ppr_per_graph=64, sssp_per_graph=16, ef=16, d=0.8):
    """The batch workload: 512 personalised-PageRank queries (seed sets of 1-64
    vertices, sizes log-uniform) and 128 SSSP sources over 8 R-MAT graphs."""
    graphs, queries = [], []
    for gi, s in enumerate(scales):
        seed = graphgen.DEFAULT_SEED_BASE + s + (1000 if gi == len(scales) - 1 else 0)
        g = graphgen.rmat(s, ef, seed=seed, weights=True)
        graphs.append(g)
        for S in graphgen.ppr_seed_sets(g.n, ppr_per_graph, seed=seed + 7):
            queries.append(dict(op=0, graph=gi, seeds=S, damping=d, eps=1e-6 * (1 - d) ** 2 / len(S)))
        for src in graphgen.sssp_sources(g, sssp_per_graph, seed=seed + 11):
            queries.append(dict(op=2, graph=gi, seeds=[int(src)]))
    return graphs, queries


def run_batch_bench(args):
    """One step = every query of the batch workload to its own termination, in
    one CUDA-graph launch; value = sum over queries of m / step time.  The
    headline runs the PageRank queries of each graph as receive-side groups of
    64 (batch mode 3: FP32 deltas, FP64 state); beside it the autotuner's pick
    among the per-query modes (FP64) and the untuned sparse mode."""
    import torch
    import paper_1710_05785_b300 as mt
    from paper_1710_05785_b300 import autotune

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev).cuda_stream
    graphs, queries = batch_workload()
    G = [mt.Graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                  torch.from_numpy(g.w.view(np.int32)).to(dev), device=local) for g in graphs]
    tuned = autotune.tune_batch(mt, graphs, G, queries, cache=autotune.Cache(None), sample=48)
    # the untuned arm: sparse (query, vertex) frontiers with default cut-offs
    untuned = dict(mode=1, cut_large=1024, chunk=1024, push_blocks_per_sm=0)
    edges = float(sum(graphs[q["graph"]].m for q in queries))
    groups = dict(mode=mt.BATCH_PULL_GROUPS)
    head = "pull_groups"
    out = {}
    for name, cfg in [(head, groups), ("tuned", tuned), ("default", untuned)]:
        b = None
        for _ in range(max(args.warmup, 1) if name == head else 1):
            b = mt.run_batch(G, queries, batch=b, stream=stream, **cfg)
        reps = args.steps if name == head else 1
        times = []
        with ClockSampler(local) as clk:
            for _ in range(reps):
                b = mt.run_batch(G, queries, batch=b, stream=stream, **cfg)
                times.append(b.stats()["elapsed_ms"])
        st = b.stats()
        qr = b.query_rounds()
        out[name] = dict(ms=float(np.mean(times)), stats=st, qrounds=qr, cfg=cfg)
        if name == head:
            clocks = clk.summary()
            bad, worst = check_batch_sample_ref(mt, G, graphs, queries, b, stream)
            if bad:
                raise RuntimeError(f"batch queries miss their answers: {bad[:5]}")
            prof = mt.run_batch(G, queries, batch=b, stream=stream,
                                flags=mt.FLAG_PROFILE_KERNELS, **cfg).stats()
        elif name == "tuned":
            bad = check_batch_sample(graphs, queries, b)
            if bad:
                raise RuntimeError(f"batch queries of the tuned arm miss their answers: {bad[:5]}")
        b.close()
    ms = out[head]["ms"]
    st = out[head]["stats"]
    peaks, peak_kind = measured_peaks()
    # the group pull's algorithmic bytes: per in-edge a 4 B sender id and the
    # sender's 64-query message vector (256 B); per vertex and round the
    # 64 states (16 B read + write each), deltas (8 B) and messages (4 B), its
    # coefficient and row offset (8 B); every group of this workload is full
    # (64 PPR queries per graph), so edge_pushes / 64 = sum of rounds x m
    nppr = [sum(1 for q in queries if q["graph"] == gi and q["op"] == 0) for gi in range(len(graphs))]
    assert all(c == 64 for c in nppr), nppr
    alg = 260.0 * prof["edge_pushes"] / 64 + 1800.0 * prof["activations"] / 64
    achieved = alg / (prof["push_ms"] * 1e-3) / 1e9
    # DRAM traffic per launch from the scale-22 capture, scaled by in-edges
    # (every graph of the workload has m = 16 n, so traffic grows with m)
    vec_cap = load_traffic().get("k_vec_pull_ppr64_rmat22")
    vec_traffic = None
    if vec_cap and prof["push_launches"]:
        vec_traffic = vec_cap / float(1 << 26) * (prof["edge_pushes"] / 64) / prof["push_launches"]
    qr = out[head]["qrounds"]
    line = {
        "metric": METRIC, "value": edges / (ms * 1e-3) / 1e9, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64/u32", "data": "synthetic",
        "config": {"workload": "batch: 512 PPR (seed sets 1-64, log-uniform) + 128 SSSP over 8 "
                               "R-MAT graphs, scales 16-22 (22 twice), edge factor 16",
                   "queries": len(queries), "graphs": len(graphs),
                   "ppr_eps": "1e-6 (1-d)^2 / |S| per query", "launch": "one CUDA graph per batch",
                   "headline": "PageRank queries in receive-side groups of 64 per graph "
                               "(batch mode 3; FP32 deltas and messages, FP64 states and "
                               "residuals); SSSP queries as round-engine branches",
                   "tuned": tuned},
        "queries_per_s": len(queries) / (ms * 1e-3),
        "rounds": st["rounds"], "query_rounds": {"min": int(qr.min()), "median": float(np.median(qr)),
                                                 "max": int(qr.max())},
        "edge_pushes": st["edge_pushes"],
        "vs_untuned": out["default"]["ms"] / ms,
        "untuned_ms": out["default"]["ms"],
        "tuned_ms": out["tuned"]["ms"], "vs_tuned": out["tuned"]["ms"] / ms,
        "ppr_error_bound": worst,
        "roofline": {"bound": "hbm", "kernel": "k_vec_pull (a warp per row, 64-query vectors)",
                     "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": vec_traffic, "peak_kind": f"{peak_kind} copy bandwidth",
                     "push_launches": prof["push_launches"],
                     "push_ms_per_launch": prof["push_ms"] / max(prof["push_launches"], 1),
                     "note": "achieved = the group pull's algorithmic bytes (260 B per in-edge, "
                             "1800 B per vertex and round) / device time of its launches; the "
                             "SSSP branches are not in it; traffic = the scale-22 capture's DRAM "
                             "bytes per in-edge x this workload's in-edges per launch"},
        "gpu_launches": int(st["kernel_launches"]) * args.steps,
        "checked": "2 SSSP (exact) and 4 PPR queries per graph from the last timed batch: "
                   "PPR bounded through a round-engine FP64 run to eps_q / 100 and its residual "
                   "bound (<= 1e-6); the tuned arm's sample by the residual bound",
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(graphs, queries, edges)
    if rank == 0:
        print(json.dumps(line), flush=True)


def check_batch_sample_ref(mt, G, graphs, queries, b, stream, sssp_per_graph=2, ppr_per_graph=4):
    """As check_batch_sample, for states with FP32 deltas: a PPR state v is
    bounded through a reference v_ref, the library's FP64 round engine run to
    eps_q / 100 from the same seeds, as max|v - v_ref| / max v_ref + the
    residual bound of v_ref.  Returns the failures and the worst bound."""
    bad, worst = [], 0.0
    seen = {}
    for i, q in enumerate(queries):
        key = (q["graph"], q["op"])
        cap = sssp_per_graph if q["op"] == 2 else ppr_per_graph
        if seen.get(key, 0) >= cap:
            continue
        seen[key] = seen.get(key, 0) + 1
        g = graphs[q["graph"]]
        v = b.state(i)
        if q["op"] == 2:
            if not sssp_is_exact(g, int(q["seeds"][0]), v):
                bad.append(i)
            continue
        c = np.zeros(g.n)
        c[np.asarray(q["seeds"])] = (1 - q["damping"]) / len(q["seeds"])
        r = mt.run(G[q["graph"]], mt.OP_SUM_F64, damping=q["damping"], eps=q["eps"] / 100,
                   v0=np.zeros(g.n), delta0=c, stream=stream)
        vref = r.state()
        r.close()
        e = float(np.abs(v - vref).max() / vref.max()) + linear_residual_bound(g, vref, c, q["damping"])
        worst = max(worst, e)
        if e > 1e-6:
            bad.append(i)
    return bad, worst


def check_batch_sample(graphs, queries, b, sssp_per_graph=2, ppr_per_graph=4):
    """The first few SSSP and PPR queries of every graph checked without the
    oracle (exact distances; residual bound <= 1e-6).  Returns the failures."""
    bad = []
    seen = {}
    for i, q in enumerate(queries):
        key = (q["graph"], q["op"])
        cap = sssp_per_graph if q["op"] == 2 else ppr_per_graph
        if seen.get(key, 0) >= cap:
            continue
        seen[key] = seen.get(key, 0) + 1
        g = graphs[q["graph"]]
        v = b.state(i)
        if q["op"] == 2:
            if not sssp_is_exact(g, int(q["seeds"][0]), v):
                bad.append(i)
        else:
            c = np.zeros(g.n)
            c[np.asarray(q["seeds"])] = (1 - q["damping"]) / len(q["seeds"])
            if linear_residual_bound(g, v, c, q["damping"]) > 1e-6:
                bad.append(i)
    return bad


def batch_cpu_baseline(graphs, queries, edges, budget_s=20.0):
    """The oracle on one core over a bounded sample of the batch: Dijkstra for
    SSSP queries and the synchronous iteration to tolerance for PPR queries,
    taken round-robin from the smallest graph up until the budget is spent;
    value = the sampled queries' edges (m of their graph each) / time."""
    import oracle
    order = sorted(range(len(queries)), key=lambda i: (graphs[queries[i]["graph"]].n, i))
    t0 = time.perf_counter()
    done, sampled_edges = 0, 0
    for i in order:
        q = queries[i]
        g = graphs[q["graph"]]
        if q["op"] == 2:
            oracle.dijkstra(g, int(q["seeds"][0]))
        else:
            oracle.pagerank(g, q["damping"], seeds=q["seeds"], tol=q["eps"])
        done += 1
        sampled_edges += g.m
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": sampled_edges / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{done} of the {len(queries)} queries, smallest graphs first "
                      f"({dt:.1f} s; PPR by synchronous iteration to the query's eps)"}


def train_scorers(mt, device=0, q=0.1, epochs=20, samples=8192, records=320):
    """The learned workload's scorers: one trained on the activation trace of a
    PageRank run (d = 0.8, top-q scheduling) on an R-MAT scale-20 graph, one
    on an SSSP run's trace on another scale-20 graph; both trained on the GPU
    by the library's own kernels.  Returns (pagerank net, sssp net, info)."""
    import torch
    from paper_1710_05785_b300 import learned

    dev = torch.device("cuda", device)

    def upload(g):
        w = torch.from_numpy(g.w.view(np.int32)).to(dev) if g.w is not None else None
        return mt.Graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev), w,
                        device=device)

    t0 = time.perf_counter()
    gtp = graphgen.rmat(20, 16, seed=graphgen.DEFAULT_SEED_BASE + 5020)
    Gtp = upload(gtp)
    Xp, yp = learned.collect(mt, Gtp, gtp.row_ptr, mt.OP_SUM_F64, samples=samples,
                             records=records, top_frac=q, eps=1e-8)
    net_pr, loss_pr = learned.train(mt, Xp, yp, epochs=epochs, device=device)
    Gtp.close()
    gts = graphgen.rmat(20, 16, seed=graphgen.DEFAULT_SEED_BASE + 6020, weights=True)
    Gts = upload(gts)
    Xs, ys = learned.collect(mt, Gts, gts.row_ptr, mt.OP_MIN_U32, samples=samples,
                             records=records, top_frac=q,
                             source=int(graphgen.sssp_sources(gts, 1)[0]))
    net_ss, loss_ss = learned.train(mt, Xs, ys, epochs=epochs, device=device)
    Gts.close()
    info = {"seconds": time.perf_counter() - t0, "pagerank_examples": int(len(yp)),
            "pagerank_final_loss": loss_pr, "sssp_examples": int(len(ys)),
            "sssp_final_loss": loss_ss}
    return net_pr, net_ss, info


# ------------------------------------------------ result checks (no oracle)
# The bench checks what it timed with properties that pin the exact answer at
# any size, in numpy: a failed check fails the run instead of leaving a figure.

def sssp_is_exact(g, source, dist):
    """Distances from `source` are exactly the shortest-path distances iff
    dist[source] = 0, no edge can shorten a distance (dist[k] <= dist[j] + w),
    and every other finite distance is attained by an edge (positive weights
    make the tight edges lead back to the source)."""
    INF = 0xFFFFFFFF
    d = np.asarray(dist, dtype=np.uint64)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    dj = d[src]
    cand = np.where(dj == INF, np.uint64(INF), dj + g.w.astype(np.uint64))
    k = g.col
    if d[source] != 0 or np.any(d[k] > cand):
        return False
    best = np.full(g.n, np.uint64(INF) + np.uint64(1), dtype=np.uint64)
    np.minimum.at(best, k, cand)
    fin = (d != INF)
    fin[source] = False
    return bool(np.all(best[fin] == d[fin]))


def linear_residual_bound(g, v, c, d):
    """||v* - v||_1 <= ||c + d P^T v - v||_1 / (1 - d) for PageRank-type
    fixed points (P the out-degree-normalised adjacency); returns that bound
    divided by max v (the norm-wise relative error it admits)."""
    deg = np.diff(g.row_ptr).astype(np.float64)
    coef = np.divide(d, deg, out=np.zeros_like(deg), where=deg > 0)
    send = np.repeat(coef * v, np.diff(g.row_ptr))
    r = np.asarray(c, dtype=np.float64) - v
    r += np.bincount(g.col, weights=send, minlength=g.n)
    return float(np.abs(r).sum() / (1 - d) / max(float(np.max(v)), 1e-300))


def run_learned_bench(args):
    """Learned scheduling: scorers trained on traces of scale-20 runs (PageRank
    with d = 0.8, and SSSP), applied to PageRank at scale 24 and SSSP at scale
    22 (edge factor 16); messages and time to the same tolerance against the
    plain form (all pending vertices, FP64 round engine), top-q by |Delta| and
    the binned engine.  The learned schedule selects the fraction q of the
    pending vertices with the highest scores (q = 0.5 and 0.3 for PageRank,
    0.8 for SSSP).  Every timed result is checked (residual bound, exact
    distances)."""
    import torch
    import paper_1710_05785_b300 as mt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def upload(g):
        w = torch.from_numpy(g.w.view(np.int32)).to(dev) if g.w is not None else None
        return mt.Graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev), w,
                        device=local)

    q = 0.1            # traces: top-q by |Delta|; also the top-q schedule compared
    q_pr, q_pr_low, q_ss = 0.5, 0.3, 0.8
    # FP32 deltas once the residual is 1e-3 of its start (1e-2 for the plain
    # form): a priority schedule holds hubs back, and a held-back hub's FP32
    # delta takes its many messages at a coarser rounding step
    sw = 1e-3
    net_pr, net_ss, training = train_scorers(mt, device=local, q=q)

    def measure(G, reps, check, **kw):
        r = mt.run(G, stream=stream, **kw)
        best = None
        for _ in range(reps):
            r = mt.run(G, stream=stream, result=r, **kw)
            st = r.stats()
            best = st if best is None or st["elapsed_ms"] < best["elapsed_ms"] else best
        if not check(r):
            raise RuntimeError(f"learned workload: a result misses its answer ({kw})")
        r.close()
        out = {"time_to_tolerance_ms": best["elapsed_ms"], "edge_pushes": best["edge_pushes"],
               "rounds": best["rounds"], "converged": best["converged"]}
        if "err" in ref:
            out["error_bound"] = ref.pop("err")
        return out

    gp = graphgen.rmat(24, 16)
    Gp = upload(gp)
    eps = 4e-8
    c_pr = np.full(gp.n, 1 - D_PR)
    ref = {}

    def f64_ok(r):
        # the FP64 state by its own residual bound; kept as the reference
        ref["v"] = r.state()
        ref["bound"] = linear_residual_bound(gp, ref["v"], c_pr, D_PR)
        ref["err"] = ref["bound"]
        return ref["bound"] <= 1e-6

    def pr_ok(r):
        # other states through the FP64 one (their L1 residual sums the FP32
        # rounding of every vertex): max |v - v*| / max v* bounded by the
        # distance to the FP64 state plus that state's own bound
        v = r.state()
        ref["err"] = float(np.abs(v - ref["v"]).max() / ref["v"].max()) + ref["bound"]
        return ref["err"] <= 1e-6

    with ClockSampler(local) as clk:
        pr = {
            "plain_f64": measure(Gp, 2, f64_ok, op=mt.OP_SUM_F64, eps=eps),
            "topq_f64": measure(Gp, 1, pr_ok, op=mt.OP_SUM_F64, eps=eps, sched=mt.SCHED_TOPFRAC,
                                top_frac=q),
            "learned_f64": measure(Gp, 2, pr_ok, op=mt.OP_SUM_F64, eps=eps,
                                   sched=mt.SCHED_LEARNED, top_frac=q_pr, scorer=net_pr),
            "mixed": measure(Gp, 2, pr_ok, op=mt.OP_SUM_MIXED, eps=eps),
            "learned_mixed": measure(Gp, 2, pr_ok, op=mt.OP_SUM_MIXED, eps=eps,
                                     sched=mt.SCHED_LEARNED, top_frac=q_pr, scorer=net_pr,
                                     mixed_switch=sw),
            "learned_mixed_q03": measure(Gp, 2, pr_ok, op=mt.OP_SUM_MIXED, eps=eps,
                                         sched=mt.SCHED_LEARNED, top_frac=q_pr_low,
                                         scorer=net_pr, mixed_switch=sw),
            "binned_mixed": measure(Gp, 2, pr_ok, op=mt.OP_SUM_MIXED, eps=eps,
                                    engine=mt.ENGINE_BINNED),
        }
        Gp.close()
        gs = graphgen.rmat(22, 16, weights=True)
        Gs = upload(gs)
        srcs = [int(s) for s in graphgen.sssp_sources(gs, 4)]
        ss = {}
        for name, kw in [("plain", {}), ("topq", dict(sched=mt.SCHED_TOPFRAC, top_frac=q_ss)),
                         ("learned", dict(sched=mt.SCHED_LEARNED, top_frac=q_ss, scorer=net_ss))]:
            tot = {"time_to_tolerance_ms": 0.0, "edge_pushes": 0, "rounds": 0}
            for s in srcs:
                m = measure(Gs, 1, lambda r, s=s: sssp_is_exact(gs, s, r.state()),
                            op=mt.OP_MIN_U32, source=s, **kw)
                for k in tot:
                    tot[k] += m[k]
            ss[name] = tot
        Gs.close()
    head = min(("learned_f64", "learned_mixed"), key=lambda k: pr[k]["time_to_tolerance_ms"])
    ms = pr[head]["time_to_tolerance_ms"]
    line = {
        "metric": METRIC, "value": gp.m / (ms * 1e-3) / 1e9, "unit": "GTEPS",
        "n_gpus": world, "steps": 2, "warmup": 1, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "learned_f64" else "f32/f64", "data": "synthetic",
        "config": {"workload": "learned scheduling: scorers trained on R-MAT scale-20 traces; "
                               "PageRank at scale 24 (eps 4e-8), SSSP at scale 22 (4 sources)",
                   "top_frac": {"pagerank": q_pr, "pagerank_low": q_pr_low, "sssp": q_ss,
                                "topq_pagerank": q},
                   "headline": head, "learned_mixed_switch": sw,
                   "l2": "inputs larger than L2 (scale-24 CSR 1.14 GB)"},
        "vs_plain_form": pr["plain_f64"]["time_to_tolerance_ms"] / ms,
        "pagerank_scale24": pr, "sssp_scale22_4_sources": ss,
        "training": training,
        "checked": "every timed result: PageRank by the residual bound (<= 1e-6 norm-wise), "
                   "SSSP distances exact",
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = pagerank_cpu_baseline(gp, D_PR, eps)
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------- the other rows

def _jacobi_system(n, per_row, seed):
    """A row diagonally dominant sparse system (factor 1.5) in the DAIC form of
    the Jacobi row of Table 1: edge i -> j with coefficient -A_ji / A_jj."""
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n, dtype=np.int64), per_row)
    cols = rng.integers(0, n, size=n * per_row)
    keep = rows != cols
    rows, cols = rows[keep], cols[keep]
    vals = rng.uniform(-1.0, 1.0, size=rows.size)
    diag = 1.5 * np.bincount(rows, weights=np.abs(vals), minlength=n) + 1.0
    b = rng.uniform(-1.0, 1.0, size=n)
    order = np.lexsort((rows, cols))            # CSR of out-edges: by source i, then target j
    src, dst = cols[order], rows[order]
    coef = -vals[order] / diag[dst]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    g = graphgen.CSRGraph(n, int(src.size), row_ptr, dst.astype(np.int32), None, "jacobi")
    return g, coef, b / diag


ROW_WORKLOADS = ["sssp-f32-lognormal20", "components-rmat20", "jacobi-2e20"]
# default step counts of the millisecond-scale workloads (0.4-5 ms a step): a
# timed region of about 0.2-0.5 s, several periods of the 50 ms clock sampler
SHORT_STEPS = {"pagerank-rmat13": 200, "components-rmat20": 500, "jacobi-2e20": 100,
               "sssp-f32-lognormal20": 60, "sssp-rmat20": 60}


def run_row(args, name):
    """The rows beyond the headline, each on its own synthetic workload: float
    SSSP on the paper's log-normal graph (8 sources), connected components on a
    symmetric R-MAT graph, the Jacobi method on a sparse diagonally dominant
    system.  value = (runs x m) / device time of the step (GTEPS)."""
    import torch
    import paper_1710_05785_b300 as mt
    import oracle

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev).cuda_stream
    if name == "sssp-f32-lognormal20":
        g = graphgen.lognormal(1 << 20, weights=True)
        srcs = [int(s) for s in np.argsort(-np.diff(g.row_ptr), kind="stable")[:NSRC]]
        runs = [dict(op=mt.OP_MIN_F32, source=s) for s in srcs]
        # bytes as for the integer push: 4 B target + 4 B weight + 8 B Delta_k RMW
        b_edge, b_vertex, dtype = 16, 24, "f32"
        cfg = {"workload": "sssp-f32-lognormal20: in-degrees LN(-0.5, 2.3), weights LN(0, 1) "
                           "in IEEE single, 8 sources (highest out-degree)"}
        kernel = "k_push<OpMinF32>"

        def cpu(budget):
            t0, done = time.perf_counter(), 0
            for s in srcs:
                oracle.dijkstra_f32(g, s)
                done += 1
                if time.perf_counter() - t0 > budget:
                    break
            dt = time.perf_counter() - t0
            return done * g.m / dt / 1e9, f"float Dijkstra from {done} of the {NSRC} sources ({dt:.1f} s)"
    elif name == "components-rmat20":
        g = graphgen.symmetrize(graphgen.rmat(20, 8))
        runs = [dict(op=mt.OP_MAX_I32)]
        # 4 B target + 8 B Delta_k RMW per edge; 8 B offsets + 8 B Delta_j + 8 B v_j RMW
        b_edge, b_vertex, dtype = 12, 24, "i32"
        cfg = {"workload": "components-rmat20: R-MAT scale 20, edge factor 8, every edge "
                           "also reversed (m = 16.8 M), max-label propagation"}
        kernel = "k_push<OpMaxI32>"

        def cpu(budget):
            t0 = time.perf_counter()
            oracle.max_reach_labels(g)
            dt = time.perf_counter() - t0
            return g.m / dt / 1e9, f"the oracle's labelling of the whole graph ({dt:.1f} s)"
    else:
        g, ecoef, d0 = _jacobi_system(1 << 20, 16, seed=graphgen.DEFAULT_SEED_BASE + 7)
        # timed runs read coefficients, v0 and Delta0 already in HBM; the
        # end-to-end leg passes the host arrays
        runs = [dict(op=mt.OP_SUM_F64, edge_coef=torch.from_numpy(ecoef).to(dev),
                     v0=torch.zeros(g.n, dtype=torch.float64, device=dev),
                     delta0=torch.from_numpy(d0).to(dev), eps=1e-10)]
        host_runs = [dict(op=mt.OP_SUM_F64, edge_coef=torch.from_numpy(ecoef).pin_memory(),
                          v0=torch.zeros(g.n, dtype=torch.float64).pin_memory(),
                          delta0=torch.from_numpy(d0).pin_memory(), eps=1e-10)]
        # 4 B target + 8 B coefficient + 16 B Delta_k RMW; 8 + 16 + 16 B per vertex
        b_edge, b_vertex, dtype = 28, 40, "f64"
        cfg = {"workload": "jacobi-2e20: 2^20 unknowns, 16 off-diagonal entries a row drawn "
                           "uniformly, row dominance 1.5, Jacobi in DAIC form, sum |Delta| < 1e-10"}
        kernel = "k_push<OpSumEdge>"
        rounds_holder = {}

        def cpu(budget):
            t0, it = time.perf_counter(), 0
            while time.perf_counter() - t0 < budget and it < 40:
                oracle.linear_power_edges(g, ecoef, d0, tol=0.0, max_iter=1)
                it += 1
            per = (time.perf_counter() - t0) / it
            r = rounds_holder.get("rounds", 1)
            return g.m / (per * r) / 1e9, (f"{it} synchronous iterations of the oracle "
                                           f"({per * 1e3:.0f} ms each), projected to the {r} "
                                           f"rounds the GPU needed")
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    w_d = torch.from_numpy(g.w.view(np.int32)).to(dev) if g.w is not None else None
    G = mt.Graph(rp_d, col_d, w_d, device=local)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    res = {}

    def step(record=None):
        for i, kw in enumerate(runs):
            res[i] = mt.run(G, result=res.get(i), stream=stream, **kw)
            if record is not None:
                record.append(res[i].stats())

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    stats = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(k)
            ev[k][0].record()
            step(stats)
            ev[k][1].record()
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    units = len(runs) * g.m
    prof = [mt.run(G, flags=mt.FLAG_PROFILE_KERNELS, stream=stream, **kw).stats() for kw in runs]
    push_ms = sum(p["push_ms"] for p in prof)
    launches = sum(p["push_launches"] for p in prof)
    alg = sum(b_edge * p["edge_pushes"] + b_vertex * p["activations"] for p in prof)
    peaks, peak_kind = measured_peaks()
    achieved = alg / (push_ms * 1e-3) / 1e9
    if name == "jacobi-2e20":
        rounds_holder["rounds"] = stats[-1]["rounds"]
    # end to end from pinned host buffers, per step: upload the graph into a
    # graph's buffers (maiter_graph_update), run, read every state back.  Two
    # steps in flight, each on its own graph, results and stream, driven by
    # its own host thread, with a lock that keeps the runs one after another;
    # graphs and results are allocated before the timed steps.
    import threading
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    w_h = torch.from_numpy(g.w.view(np.int32)).pin_memory() if g.w is not None else None
    e2e_runs = host_runs if name == "jacobi-2e20" else runs
    slots = []
    for _ in range(2):
        s_k = torch.cuda.Stream(dev)
        G_k = mt.Graph(rp_h, col_h, w_h, device=local)
        slots.append({"G": G_k, "s": s_k,
                      "res": [mt.run(G_k, stream=s_k.cuda_stream, **kw) for kw in e2e_runs],
                      "out": torch.empty(g.n * 8, dtype=torch.uint8).pin_memory()})
    torch.cuda.synchronize()
    run_lock = threading.Lock()

    def e2e_step(slot):
        slot["G"].update(rp_h, col_h, w_h, stream=slot["s"].cuda_stream)
        with run_lock:
            for i, kw in enumerate(e2e_runs):
                slot["res"][i] = mt.run(slot["G"], result=slot["res"][i],
                                        stream=slot["s"].cuda_stream, **kw)
        for i, kw in enumerate(e2e_runs):
            slot["res"][i].state(slot["out"].view(
                torch.float64 if kw["op"] == mt.OP_SUM_F64 else torch.int32)[:g.n])

    per_slot = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(per_slot):
        e2e_step(slots[0])
    e2e_serial_s = (time.perf_counter() - t0) / per_slot
    t0 = time.perf_counter()
    run_in_threads([lambda sl=sl: [e2e_step(sl) for _ in range(per_slot)] for sl in slots])
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / (2 * per_slot)
    for sl in slots:
        for rr in sl["res"]:
            rr.close()
        sl["G"].close()
    h2d = rp_h.numel() * 8 + col_h.numel() * 4 + (w_h.numel() * 4 if w_h is not None else 0)
    if name == "jacobi-2e20":
        h2d += g.m * 8 + g.n * 16   # coefficients, v0 and Delta0
    d2h = len(runs) * g.n * (8 if dtype == "f64" else 4)
    line = {
        "metric": METRIC, "value": units / (ms * 1e-3) / 1e9, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": dict(cfg, n=g.n, m=g.m, runs_per_step=len(runs),
                       l2=f"{L2_FLUSH_BYTES >> 20} MiB write between steps"),
        "rounds_per_run": float(np.mean([s["rounds"] for s in stats[-len(runs):]])),
        "edge_pushes_per_step": int(sum(s["edge_pushes"] for s in stats[-len(runs):])),
        "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": None, "peak_kind": f"{peak_kind} copy bandwidth",
                     "push_launches": launches, "push_ms_per_launch": push_ms / max(launches, 1),
                     "alg_bytes_per_launch": alg / max(launches, 1)},
        "e2e": {"value": units / e2e_s / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps_in_flight": 2,
                "one_step_at_a_time": units / e2e_serial_s / 1e9},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats) / args.steps),
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        v, sample = cpu(20.0)
        line["cpu_baseline"] = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 10; the millisecond-scale workloads "
                         "default to enough steps for a timed region of a few tenths of a "
                         "second, so that the clock sampler sees it)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-sssp", action="store_true",
                    help="default workload: leave out the nested SSSP record")
    ap.add_argument("--scale", type=int, default=0,
                    help="PageRank workloads: R-MAT scale instead of the workload's "
                         "(a smaller case of the same kernels, for profiling)")
    ap.add_argument("--head-only", action="store_true",
                    help="PageRank workloads: time only the headline variant")
    ap.add_argument("--workload", default="pagerank-mixed-rmat24",
                    choices=["sssp-rmat20", "batch", "learned"] + sorted(PR_WORKLOADS)
                    + ROW_WORKLOADS,
                    help="pagerank-mixed-rmat24 (default: PageRank, mixed precision, R-MAT "
                         "scale 24, with the SSSP scale-20 record nested) or another workload")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = SHORT_STEPS.get(args.workload, 10) if args.impl == "ours" else 10
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        if args.workload in PR_WORKLOADS:
            nested = None
            if args.workload == "pagerank-mixed-rmat24" and not args.no_sssp and not args.scale:
                def nested(d):
                    # its own step count: 10 steps of ~4.4 ms would end inside one
                    # period of the clock sampler
                    sub = argparse.Namespace(**vars(args))
                    sub.steps = max(args.steps, SHORT_STEPS["sssp-rmat20"])
                    return {"sssp_rmat20_8src": run_sssp(sub, d, emit=False)}
            run_pagerank(args, args.workload, dist, nested)
        elif args.workload == "batch":
            run_batch_bench(args)
        elif args.workload == "learned":
            run_learned_bench(args)
        elif args.workload in ROW_WORKLOADS:
            run_row(args, args.workload)
        else:
            run_sssp(args, dist, emit=True)
    finally:
        if dist:
            dist.destroy_process_group()


def run_sssp(args, dist, emit=True):
    """SSSP on R-MAT scale 20 (edge factor 16, weights U[1, 255]), 8 sources one
    after another, every run to the exact fixed point; one step = the 8
    sources.  value = 8 m / step time (GTEPS).  Prints the line (emit) or
    returns it as a record."""
    import torch
    import paper_1710_05785_b300 as mt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    g = graphgen.rmat(SCALE, EF, weights=True)
    sources = rank_sources(g, rank, world)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    w_d = torch.from_numpy(g.w.view(np.int32)).to(dev)
    G = mt.Graph(rp_d, col_d, w_d, device=local)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    # One step: the 8 sources one after another, chained inside one graph
    # launch (maiter_run_batch, dense mode 2: each query is a round-engine run
    # of its own, started when the one before it has stopped).
    queries = [dict(op=mt.OP_MIN_U32, graph=0, seeds=[s]) for s in sources]
    bat = [None]
    stats, qrounds = [], []

    def step(record=False):
        bat[0] = mt.run_batch([G], queries, stream=stream.cuda_stream,
                              mode=mt.BATCH_DENSE_CHAINED, batch=bat[0])
        if record:
            stats.append(bat[0].stats())
            qrounds.append(bat[0].query_rounds())

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k)                      # evict the graph from L2 between steps
            ev[k][0].record(stream)
            step(record=True)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = weak_value(ms_per_step, g.m, world)

    # kernel-level roofline: the same 8 runs with per-kernel events
    prof = []
    for s in sources:
        r = mt.run(G, mt.OP_MIN_U32, source=s, flags=mt.FLAG_PROFILE_KERNELS,
                   stream=stream.cuda_stream)
        prof.append(r.stats())
        r.close()
    push_ms = sum(p["push_ms"] for p in prof)
    push_launches = sum(p["push_launches"] for p in prof)
    alg_bytes = sum(BYTES_PER_EDGE * p["edge_pushes"] + BYTES_PER_VERTEX * p["activations"]
                    for p in prof)
    peaks, peak_kind = measured_peaks()
    achieved = alg_bytes / (push_ms * 1e-3) / 1e9
    traffic = load_traffic().get("k_push_sssp_rmat20")

    # the other schedules and the asynchronous engine on the same 8 sources
    # (one warm pass, then the best of two timed passes)
    variant_kw = {
        "async": dict(engine=mt.ENGINE_ASYNC),
        "topq05_sync": dict(sched=mt.SCHED_TOPFRAC, top_frac=0.05),
        "bucket64_sync": dict(sched=mt.SCHED_BUCKET, threshold=64.0),
    }
    variants = {"plain_sync": {"ms_per_8_sources": ms_per_step,
                               "edge_pushes": int(sum(s["edge_pushes"] for s in stats) / args.steps)}}
    # the same 8 sources as 8 maiter_run calls (a host round trip after each
    # run), and as one batch whose 8 runs go side by side (mode 0)
    tts = []
    for name in ("separate_runs", "batch8_side_by_side"):
        best = None
        rv = None
        for rep in range(3):
            flush.fill_(rep)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if name == "separate_runs":
                for s in sources:
                    rv = mt.run(G, mt.OP_MIN_U32, source=s, result=rv, stream=stream.cuda_stream)
                    if rep == 2:
                        tts.append(rv.stats()["elapsed_ms"])
            else:
                rv = mt.run_batch([G], queries, stream=stream.cuda_stream, mode=mt.BATCH_DENSE,
                                  batch=rv)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
        rv.close()
        variants[name] = {"ms_per_8_sources": best, "vs_plain": ms_per_step / best}
    for name, kw in variant_kw.items():
        rv = None
        best, pushes = None, 0
        for rep in range(3):
            t0 = time.perf_counter()
            tot, pushes = 0.0, 0
            for s in sources:
                rv = mt.run(G, mt.OP_MIN_U32, source=s, result=rv, stream=stream.cuda_stream, **kw)
                st = rv.stats()
                tot += st["elapsed_ms"]
                pushes += st["edge_pushes"]
            if rep > 0:
                best = tot if best is None else min(best, tot)
        rv.close()
        variants[name] = {"ms_per_8_sources": best, "edge_pushes": int(pushes),
                          "vs_plain": ms_per_step / best}

    # end to end through the C ABI from pinned host buffers, per step: upload
    # the CSR into a graph's buffers (maiter_graph_update), run the 8 sources
    # chained in one launch, read every distance vector back.  Two steps are
    # in flight, each on its own graph, batch and stream, driven by its own
    # host thread: one step's upload and read-back overlap the other's runs,
    # while a lock keeps the runs themselves one after another.  Buffers and
    # batches are allocated before the timed steps.
    import threading
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    w_h = torch.from_numpy(g.w.view(np.int32)).pin_memory()
    h2d = rp_h.numel() * 8 + col_h.numel() * 4 + w_h.numel() * 4
    d2h = NSRC * g.n * 4
    e2e_steps = 0 if args.no_e2e else 2 * max(1, min(args.steps, 5))
    slots = []
    for _ in range(2):
        s_k = torch.cuda.Stream(dev)
        G_k = mt.Graph(rp_h, col_h, w_h, device=local)
        b_k = mt.run_batch([G_k], queries, stream=s_k.cuda_stream, mode=mt.BATCH_DENSE_CHAINED)
        slots.append({"G": G_k, "s": s_k, "b": b_k,
                      "out": torch.empty(g.n, dtype=torch.int32).pin_memory()})
    torch.cuda.synchronize()
    run_lock = threading.Lock()

    def e2e_step(slot):
        slot["G"].update(rp_h, col_h, w_h, stream=slot["s"].cuda_stream)
        with run_lock:
            slot["b"] = mt.run_batch([slot["G"]], queries, stream=slot["s"].cuda_stream,
                                     mode=mt.BATCH_DENSE_CHAINED, batch=slot["b"])
        for i in range(NSRC):
            slot["b"].state(i, slot["out"])

    def e2e_worker(slot, count):
        for _ in range(count):
            e2e_step(slot)

    # one step at a time (no overlap), then two in flight
    t0 = time.perf_counter()
    for _ in range(e2e_steps // 2):
        e2e_step(slots[0])
    e2e_serial_s = (time.perf_counter() - t0) / max(e2e_steps // 2, 1)
    t0 = time.perf_counter()
    run_in_threads([lambda k=k: e2e_worker(slots[k], e2e_steps // 2) for k in range(2)])
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / max(e2e_steps, 1)
    for sl in slots:
        sl["b"].close()
        sl["G"].close()
    e2e_value = NSRC * g.m * world / e2e_s / 1e9 if e2e_steps else None
    e2e_serial = NSRC * g.m * world / e2e_serial_s / 1e9 if e2e_steps else None

    launches = sum(s["kernel_launches"] for s in stats) + args.steps  # + the L2 flush fill
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": sssp_config(g, world),
        "engine": "sync (CUDA graph, device-side WHILE); the 8 runs chained in one graph "
                  "launch (maiter_run_batch mode 2)", "sched": "all pending",
        "time_to_solution_ms": {"mean": float(np.mean(tts)), "max": float(np.max(tts))},
        "gteps_work": float(sum(s["edge_pushes"] for s in stats) / (total_ms * 1e-3) / 1e9),
        "rounds_per_source": float(np.mean(np.concatenate(qrounds))),
        "roofline": {"bound": "hbm", "kernel": "k_push<OpMinU32>", "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "push_launches": push_launches,
                     "push_ms_per_launch": push_ms / max(push_launches, 1),
                     "scan_ms_per_launch": sum(p["scan_ms"] for p in prof) / max(push_launches, 1),
                     "alg_bytes_per_launch": alg_bytes / max(push_launches, 1),
                     # each edge push reads Delta_k once (the filter); the
                     # atomicMin follows only where the distance improves
                     "random_access": random_access(
                         mt, mt.PROBE_LOAD_32, g.n, local,
                         sum(p["edge_pushes"] for p in prof), push_ms, "4-byte L2 loads")},
        "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps_in_flight": 2,
                "one_step_at_a_time": e2e_serial},
        "variants": variants,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
    }
    # every source's distances of the last timed step, checked exactly
    for i, s in enumerate(sources):
        if not sssp_is_exact(g, s, bat[0].state(i)):
            raise RuntimeError(f"SSSP distances from source {s} are not exact")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, sources)
    bat[0].close()
    G.close()
    if emit and rank == 0:
        print(json.dumps(line), flush=True)
    return line


if __name__ == "__main__":
    main()
