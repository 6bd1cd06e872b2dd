"""Autotuner host logic (no GPU): candidate spaces, the search, the cache and
graph signatures."""
import json

import graphgen
from paper_1710_05785_b300 import autotune


def test_candidates_respect_cut_order():
    cs = autotune.candidates(autotune.RUN_SPACE)
    assert cs and all(c["cut_warp"] <= c["cut_cta"] for c in cs)
    assert len({json.dumps(c, sort_keys=True) for c in cs}) == len(cs)
    # sparse mode: 3 x 3 x 2; dense mode ignores cut_large / chunk: 2
    assert len(autotune.candidates(autotune.BATCH_SPACE)) == 3 * 3 * 2 + 2


def test_search_picks_the_fastest_and_warms_up():
    calls = []

    def measure(c):
        calls.append(c)
        # fastest at cut_large 1024, chunk 512, push_blocks_per_sm 4
        return abs(c["cut_large"] - 1024) / 100 + abs(c["chunk"] - 512) / 100 + \
            (0 if c["push_blocks_per_sm"] == 4 else 1)

    best, timings = autotune.search(autotune.BATCH_SPACE, measure, repeats=2)
    assert best == {"mode": 1, "cut_large": 1024, "chunk": 512, "push_blocks_per_sm": 4}
    assert len(calls) == 3 * len(timings)          # one warm call + two timed per config
    assert timings[0][0] <= timings[-1][0]


def test_cache_round_trip(tmp_path):
    p = tmp_path / "tune.json"
    c = autotune.Cache(str(p))
    assert c.get("k") is None
    c.put("k", {"config": {"chunk": 1024}})
    c2 = autotune.Cache(str(p))
    assert c2.get("k") == {"config": {"chunk": 1024}}


def test_graph_signature_tracks_shape_not_seed_noise():
    a = graphgen.rmat(10, 8, seed=1)
    b = graphgen.rmat(10, 8, seed=1)
    c = graphgen.rmat(11, 8, seed=1)
    assert autotune.graph_signature(a) == autotune.graph_signature(b)
    assert autotune.graph_signature(a) != autotune.graph_signature(c)
    assert autotune.graph_signature(a, c) != autotune.graph_signature(c, a)
