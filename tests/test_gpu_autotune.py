"""The autotuner on the GPU: a real search over the library's knobs, with
every candidate's counts checked against the starting configuration's, and
the tuned counts checked against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

TAUS = [0.55, 0.7, 0.85, 0.95]


def test_tune_count_searches_caches_and_keeps_results(tmp_path):
    ubt = require_gpu()
    from paper_2602_14084_gb300 import autotune as at
    n = 20000
    s, d = synth.chung_lu(n, 2.1, 20.0, 2000.0, 3)
    k = synth.quantise(synth.p_beta(s.size, 0.5, 0.5, 4))
    want_b, want_u = oracle.count_threshold(n, s, d, k, TAUS)
    saved = at.current()
    path = str(tmp_path / "tune.json")
    try:
        rec = at.tune_count(n, s, d, k, TAUS, prune=True, cache_path=path, rounds=1, budget_s=60,
                            knobs=["hub_threshold", "block_work", "block_unit", "blocks_per_sm"])
        assert rec["source"] == "search" and rec["ms"] <= rec["start_ms"]
        assert at.current(list(rec["config"])) == rec["config"]
        G = ubt.Graph(n, s, d, k=k)  # built under the tuned knobs
        gb, gu = G.count_threshold(TAUS, prune=True)
        assert np.array_equal(gb, want_b) and np.array_equal(gu, want_u)
        assert G.guard() == 0
        G.close()
        at.apply(saved)
        rec2 = at.tune_count(n, s, d, k, TAUS, prune=True, cache_path=path,
                             knobs=["hub_threshold", "block_work", "block_unit", "blocks_per_sm"])
        assert rec2["source"] == "cache" and rec2["config"] == rec["config"]
    finally:
        at.apply(saved)


def test_tuner_rejects_a_configuration_that_changes_results():
    require_gpu()
    import torch
    from paper_2602_14084_gb300 import autotune as at
    calls = {"n": 0}

    def run(G):
        calls["n"] += 1
        return torch.tensor([calls["n"]])  # a "result" that changes between configurations

    qt = at.QueryTuner(lambda: None, run, reps=1, warmup=1)
    saved = at.current()
    try:
        qt.measure({"block_unit": 16})
        with pytest.raises(RuntimeError, match="changed the query result"):
            qt.measure({"block_unit": 8})
    finally:
        at.apply(saved)
