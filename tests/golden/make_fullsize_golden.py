"""Writes the full-size expected values that tests/test_gpu_fullsize.py
compares the GPU path with, on workloads where the oracle needs minutes
(too long to run inside the GPU test suite).  Calls only oracle/ (the
values) and synth/ (the seeded inputs); nothing from the CUDA path.

  rmat22_sweep32.json  R-MAT scale 22 (edge factor 16, P+ ~ 0.5 Beta(8,2) +
                       0.5 Beta(2,8) quantised), seed 1: the number of
                       triangles and the t-balanced / t-unbalanced counts at
                       the 32 thresholds t_i = 0.51 + i 0.48/31 (Defs. 4-5,
                       Def. 8), by the oracle's resident multi-threaded pass
                       (pinned equal to its serial pass).
  rmat20_worlds.json   R-MAT scale 20 (edge factor 16, k ~ U{0..65536}), seed
                       1: balanced counts (Def. 3) in every world of four
                       seeded world words drawn with seed 7, and the sum of
                       the balanced counts over all 4,096 worlds (64 words).

Each file records a digest of the input arrays, so a test can tell whether
its generator produced the same graph.  Run from the repository root:

    python tests/golden/make_fullsize_golden.py [rmat22] [rmat20]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SWEEP32 = [0.51 + i * (0.48 / 31) for i in range(32)]
WORLD_SEED = 7
W = 4096


def input_digest(g):
    h = hashlib.sha256()
    for a in (g.src, g.dst, g.k):
        h.update(np.ascontiguousarray(a, dtype=np.uint32).tobytes())
    return h.hexdigest()[:24]


def world_words():
    """The four world words checked one by one (seeded, distinct, in 0..63)."""
    return sorted(int(x) for x in synth.rng(20).choice(W // 64, size=4, replace=False))


def make_rmat22():
    g = synth.config_graph("rmat22", seed=1)
    t0 = time.time()
    R = oracle.ResidentGraph(g.n, g.src, g.dst)
    b, u, T = R.count(g.k, SWEEP32, threads=oracle.threads())
    R.close()
    rec = {"graph": "rmat22", "graph_seed": 1, "n": g.n, "m": g.m, "input_digest": input_digest(g),
           "taus": SWEEP32, "triangles": T, "balanced": b.tolist(), "unbalanced": u.tolist(),
           "made_by": "oracle.ResidentGraph.count, %d threads, %.0f s" % (oracle.threads(), time.time() - t0)}
    with open(os.path.join(HERE, "rmat22_sweep32.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print("rmat22: T = %d (%.0f s)" % (T, time.time() - t0), flush=True)


def _world_counts_rmat20(words):
    """One oracle call in a worker process (the graph is regenerated there)."""
    g = synth.config_graph("rmat20", seed=1)
    return oracle.world_counts(g.n, g.src, g.dst, g.k, WORLD_SEED, list(words))


def make_rmat20():
    import multiprocessing as mp
    g = synth.config_graph("rmat20", seed=1)
    t0 = time.time()
    words = world_words()
    # four words per oracle call (bounds its sign table), the calls in parallel processes
    chunks = [words] + [list(range(w0, w0 + 4)) for w0 in range(0, W // 64, 4)]
    with mp.get_context("spawn").Pool(max(1, min(len(chunks), os.cpu_count() or 1))) as pool:
        res = pool.map(_world_counts_rmat20, chunks)
    per = res[0]
    total = int(sum(int(r.sum()) for r in res[1:]))
    rec = {"graph": "rmat20", "graph_seed": 1, "n": g.n, "m": g.m, "input_digest": input_digest(g),
           "world_seed": WORLD_SEED, "W": W, "words": words,
           "per_world": {str(w): per[i * 64:(i + 1) * 64].tolist() for i, w in enumerate(words)},
           "balanced_sum_over_all_worlds": total,
           "made_by": "oracle.world_counts, %.0f s" % (time.time() - t0)}
    with open(os.path.join(HERE, "rmat20_worlds.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print("rmat20: total %d (%.0f s)" % (total, time.time() - t0), flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["rmat22", "rmat20"]
    oracle.build()
    if "rmat22" in which:
        make_rmat22()
    if "rmat20" in which:
        make_rmat20()
