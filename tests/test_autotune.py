"""Host logic of the autotuner (no GPU): the search, the cache and its keys.

The library's knob setters are replaced by a dictionary, and timings by a
cost function with a known minimum, so the search can be checked exactly.
"""
import itertools
import json

import pytest

from paper_2602_14084_gb300 import autotune as at


@pytest.fixture
def knobs(monkeypatch):
    """A fake of the library's tuning state (ubt_set_tuning / ubt_get_tuning)."""
    state = {"hub_threshold": 128, "block_work": 1 << 14, "pull": 1, "count_visitor": 0, "block_unit": 16,
             "small_batch": 4,
             "blocks_per_sm": 32, "block_threads": 512, "warp_threads": 128, "smem_table_max": 8192,
             "world_words_per_pass": 8, "long_min": 64, "long_tail": 1}

    def get(name):
        return state[name]

    def set_(name, v):
        if name not in state:
            raise RuntimeError("unknown knob")
        state[name] = int(v)

    monkeypatch.setattr(at, "_lib", lambda: (get, set_))
    return state


def separable_cost(best):
    # each knob adds (log-distance from its optimum)^2; the minimum is `best`
    import math
    def f(cfg):
        return 1.0 + sum((math.log2(cfg[k]) - math.log2(v)) ** 2 for k, v in best.items())
    return f


def test_descent_finds_the_minimum_of_a_separable_cost():
    space = {"a": [1, 2, 4, 8, 16], "b": [32, 64, 128, 256], "c": [1, 2, 3]}
    best = {"a": 4, "b": 256, "c": 1}
    res = at.coordinate_descent(separable_cost(best), {"a": 16, "b": 32, "c": 3}, space)
    assert res.config == best
    assert res.ms == pytest.approx(1.0)
    assert res.start_ms > res.ms
    # every configuration is measured at most once
    keys = [tuple(sorted(t["config"].items())) for t in res.trials]
    assert len(keys) == len(set(keys))


def test_descent_keeps_the_incumbent_within_the_noise_margin():
    space = {"a": [1, 2, 3]}
    cost = {1: 1.00, 2: 0.99, 3: 1.5}  # 1 % better: below the 2 % margin
    res = at.coordinate_descent(lambda c: cost[c["a"]], {"a": 1}, space, min_gain=0.02)
    assert res.config == {"a": 1}
    res = at.coordinate_descent(lambda c: cost[c["a"]], {"a": 1}, space, min_gain=0.005)
    assert res.config == {"a": 2}


def test_descent_handles_interacting_knobs_over_rounds():
    # the best b depends on a: a second round is needed to reach the optimum
    space = {"a": [1, 2], "b": [1, 2]}
    cost = {(1, 1): 5.0, (2, 1): 4.0, (1, 2): 6.0, (2, 2): 1.0}
    res = at.coordinate_descent(lambda c: cost[(c["a"], c["b"])], {"a": 1, "b": 1}, space, order=["b", "a"])
    assert res.config == {"a": 2, "b": 2}
    assert res.rounds >= 2


def test_descent_skips_infeasible_configurations():
    space = {"a": [1, 2, 4]}

    def m(c):
        if c["a"] == 4:
            raise ValueError("rejected by the library")
        return {1: 3.0, 2: 2.0}[c["a"]]

    res = at.coordinate_descent(m, {"a": 1}, space)
    assert res.config == {"a": 2}
    assert any(t["ms"] == float("inf") for t in res.trials)


def test_descent_stops_at_the_time_budget():
    ticks = itertools.count()
    space = {"a": list(range(1, 50))}
    res = at.coordinate_descent(lambda c: 100.0 - c["a"], {"a": 1}, space, budget_s=10,
                                clock=lambda: float(next(ticks)))
    assert res.stopped == "budget"
    assert len(res.trials) < 49


def test_signature_buckets():
    base = {"n": 1_000_000, "m": 9_119_924, "wedges": 1_084_451_115, "max_out_degree": 322, "hub_vertices": 4956,
            "kind": 0}
    near = dict(base, m=9_300_000, wedges=1_100_000_000, hub_vertices=5100, max_out_degree=330)
    far = dict(base, m=2 * base["m"])
    assert at.signature(base) == at.signature(near)
    assert at.signature(base) != at.signature(far)
    assert at.signature(base, n_graphs=10000) != at.signature(base)
    assert at.signature(base) != at.signature(dict(base, kind=1))


def test_count_variant_follows_the_visitor_classes():
    assert at.count_variant(1, True) == "nt1-pruned"
    assert at.count_variant(3, True) == "nt4-pruned"
    assert at.count_variant(4, False) == "nt4-full"
    assert at.count_variant(8, True) == "nt8-pruned"
    assert at.count_variant(9, True) == at.count_variant(64, True) == "nt64-pruned"


def test_cache_merge_and_reload(tmp_path):
    p = str(tmp_path / "sub" / "cache.json")
    at.save_cache(p, {"k1": {"config": {"a": 1}, "ms": 2.0}})
    at.save_cache(p, {"k2": {"config": {"a": 2}, "ms": 1.0}})
    d = at.load_cache(p)
    assert set(d) == {"k1", "k2"} and d["k1"]["config"] == {"a": 1}
    with open(p, "w") as f:
        f.write("{not json")
    assert at.load_cache(p) == {}
    assert at.load_cache(str(tmp_path / "missing.json")) == {}


def test_tune_searches_applies_and_caches(knobs, tmp_path):
    info = {"n": 1000, "m": 10000, "wedges": 10 ** 6, "max_out_degree": 50, "hub_vertices": 3, "kind": 0}
    best = {"hub_threshold": 64, "block_unit": 4}
    cost = separable_cost(best)
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        return cost(cfg)

    path = str(tmp_path / "c.json")
    rec = at.tune(None, None, "count", info, variant="nt4-pruned", knobs=["hub_threshold", "block_unit"],
                  cache_path=path, device="FakeGPU-sm2", measure=measure)
    assert rec["source"] == "search"
    assert rec["config"] == best
    assert knobs["hub_threshold"] == 64 and knobs["block_unit"] == 4  # applied
    assert knobs["block_work"] == 1 << 14  # untouched
    stored = json.load(open(path))
    assert rec["key"] in stored and "FakeGPU-sm2|count:nt4-pruned|" in rec["key"]
    # second call: served from the cache, nothing measured, configuration applied again
    knobs["hub_threshold"] = 128
    calls.clear()
    rec2 = at.tune(None, None, "count", info, variant="nt4-pruned", knobs=["hub_threshold", "block_unit"],
                   cache_path=path, device="FakeGPU-sm2", measure=measure)
    assert rec2["source"] == "cache" and not calls
    assert knobs["hub_threshold"] == 64


def test_tuning_scope_restores(knobs):
    with at.tuning_scope({"block_unit": 2, "small_batch": 1}):
        assert knobs["block_unit"] == 2 and knobs["small_batch"] == 1
    assert knobs["block_unit"] == 16 and knobs["small_batch"] == 4


def test_candidate_values_are_within_the_library_limits():
    # the limits ubt_set_tuning enforces (include/ubt.h)
    lim = {"hub_threshold": (2, 4096), "block_work": (1, 1 << 40), "pull": (0, 1), "count_visitor": (0, 1), "block_unit": (1, 32),
           "small_batch": (1, 1024),
           "block_threads": (64, 512), "warp_threads": (64, 512), "blocks_per_sm": (1, 32),
           "smem_table_max": (64, 1 << 20), "world_words_per_pass": (1, 64), "long_min": (1, 1 << 20),
           "long_tail": (0, 1)}
    for k, vals in at.ALL_KNOBS.items():
        lo, hi = lim[k]
        assert all(lo <= v <= hi for v in vals), k
    for q, ks in at.QUERY_KNOBS.items():
        assert set(ks) <= set(at.ALL_KNOBS), q
