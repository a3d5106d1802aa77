"""Autotuner for the traversal's work partition and launch shape.

The traversal kernels (ubt_traverse.cuh) split the forward lists into task
classes and launch persistent blocks; how the work is cut is set by the
library's tuning knobs (``ubt_set_tuning``).  None of them changes a result --
they only move work between task kinds, warps and blocks -- but the best
setting depends on the graph's degree distribution, the query and the GPU.
This module picks them by measurement:

* knobs that act when a graph is built (``BUILD_KNOBS``: the pair
  partition, the block-task limits on list length and streamed work, the
  shared-memory table limit) and knobs that
  act on every query (``RUN_KNOBS``: block shapes, blocks per SM, work-grab
  sizes, sign-world words per pass);
* coordinate descent over a small candidate list per knob, starting from the
  current settings: one knob at a time, every candidate timed with CUDA events
  on the query's stream (median of ``reps`` runs after ``warmup``), the best
  kept when it beats the incumbent by more than ``min_gain``; rounds repeat
  until a round changes nothing or the time budget is spent;
* every candidate's output is compared with the starting configuration's
  output (bit-equal for integer results), so a tuning that changed a result
  fails loudly instead of being cached;
* results are cached in a JSON file keyed by GPU, query and a coarse graph
  signature (log2 buckets of the sizes that decide the task split), so a
  graph of the same shape reuses the tuning without searching again.

Only host logic lives here; every timed step runs in the library's kernels.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

# candidate values per knob (the library validates each against its limits)
BUILD_KNOBS: Dict[str, List[int]] = {
    "pull": [1, 0],
    "hub_threshold": [32, 64, 128, 256, 512],
    "block_work": [1 << 12, 1 << 14, 1 << 16, 1 << 18, 1 << 20],
    "smem_table_max": [4096, 8192, 16384],
}
RUN_KNOBS: Dict[str, List[int]] = {
    "count_visitor": [0, 1],
    "block_unit": [1, 2, 4, 8, 16, 32],
    "small_batch": [1, 2, 4, 8, 16],
    "block_threads": [128, 256, 512],
    "warp_threads": [64, 128],
    "blocks_per_sm": [1, 2, 4, 32],
    "world_words_per_pass": [1, 2, 4, 8, 16, 32, 64],
    "long_min": [32, 48, 64, 96, 128],
    "long_tail": [1, 0],
}
# knobs that matter per query kind (others are left as they are)
QUERY_KNOBS: Dict[str, List[str]] = {
    "count": ["count_visitor", "hub_threshold", "block_work", "block_unit", "small_batch", "blocks_per_sm",
              "block_threads", "warp_threads", "smem_table_max", "pull", "long_min", "long_tail"],
    "expected": ["hub_threshold", "block_work", "block_unit", "small_batch", "blocks_per_sm", "block_threads",
                 "warp_threads", "smem_table_max", "pull"],
    "worlds": ["world_words_per_pass", "hub_threshold", "block_work", "block_unit", "small_batch",
               "blocks_per_sm", "long_tail", "long_min"],
    "batch": ["block_threads", "hub_threshold", "block_work", "block_unit", "small_batch", "warp_threads",
              "blocks_per_sm", "long_tail", "long_min"],
}
ALL_KNOBS = {**BUILD_KNOBS, **RUN_KNOBS}


def _lib():
    from . import get_tuning, set_tuning
    return get_tuning, set_tuning


def current(names: Optional[Sequence[str]] = None) -> Dict[str, int]:
    """The library's current value of each knob."""
    get_tuning, _ = _lib()
    return {k: get_tuning(k) for k in (names or ALL_KNOBS)}


def apply(config: Dict[str, int]) -> None:
    """Sets every knob of `config` in the library."""
    _, set_tuning = _lib()
    for k, v in config.items():
        set_tuning(k, int(v))


class tuning_scope:
    """Context manager: applies a configuration and restores the previous one."""

    def __init__(self, config: Dict[str, int]):
        self.config = dict(config)
        self.saved: Dict[str, int] = {}

    def __enter__(self):
        self.saved = current(list(self.config))
        apply(self.config)
        return self

    def __exit__(self, *exc):
        apply(self.saved)
        return False


def _bucket(x: int) -> int:
    return 0 if x <= 0 else int(round(math.log2(x)))


def signature(info: Dict[str, int], n_graphs: int = 1) -> str:
    """Coarse shape of a built graph: the sizes that decide the task split, in
    log2 buckets (graphs that differ only by seed share a signature)."""
    parts = [
        "kind%d" % int(info.get("kind", 0)),
        "n%d" % _bucket(info["n"]),
        "m%d" % _bucket(info["m"]),
        "w%d" % _bucket(info.get("wedges", 0)),
        "d%d" % _bucket(info.get("max_out_degree", 0)),
        "h%d" % _bucket(info.get("hub_vertices", 0)),
    ]
    if n_graphs > 1:
        parts.append("g%d" % _bucket(n_graphs))
    return "-".join(parts)


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s-sm%d" % (p.name.replace(" ", "_"), p.multi_processor_count)


def cache_key(device: str, query: str, sig: str) -> str:
    return "%s|%s|%s" % (device, query, sig)


def default_cache_path() -> str:
    return os.environ.get("UBT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ubt_autotune.json"))


def shipped_cache_path() -> str:
    """Tunings measured for the package's benchmark workloads."""
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, entries: Dict[str, dict]) -> None:
    """Merges `entries` into the cache file (written atomically)."""
    d = load_cache(path)
    d.update(entries)
    os.makedirs(os.path.dirname(os.path.abspath(path)) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


@dataclass
class SearchResult:
    config: Dict[str, int]
    ms: float
    start_ms: float
    trials: List[dict] = field(default_factory=list)
    rounds: int = 0
    stopped: str = ""

    @property
    def speedup(self) -> float:
        return self.start_ms / self.ms if self.ms > 0 else 1.0


def coordinate_descent(measure: Callable[[Dict[str, int]], float], start: Dict[str, int],
                       space: Dict[str, List[int]], order: Optional[Sequence[str]] = None, rounds: int = 2,
                       min_gain: float = 0.02, budget_s: float = float("inf"),
                       clock: Callable[[], float] = time.monotonic) -> SearchResult:
    """Minimises measure(config) one knob at a time.

    measure returns a time (lower is better) or raises ValueError for an
    infeasible configuration (skipped).  A candidate replaces the incumbent
    only if it is faster by more than `min_gain` (relative), which keeps
    timing noise from wandering the search.  Each configuration is measured
    at most once."""
    t0 = clock()
    order = list(order or space)
    best = dict(start)
    seen: Dict[tuple, float] = {}
    trials: List[dict] = []

    def key(cfg):
        return tuple(sorted(cfg.items()))

    def run(cfg):
        k = key(cfg)
        if k not in seen:
            try:
                seen[k] = float(measure(cfg))
            except ValueError:
                seen[k] = float("inf")
            trials.append({"config": dict(cfg), "ms": seen[k]})
        return seen[k]

    best_ms = run(best)
    start_ms = best_ms
    stopped = "converged"
    r = 0
    for r in range(1, rounds + 1):
        changed = False
        for name in order:
            for v in space[name]:
                if clock() - t0 > budget_s:
                    stopped = "budget"
                    break
                if v == best.get(name):
                    continue
                cand = dict(best)
                cand[name] = v
                ms = run(cand)
                if ms < best_ms * (1.0 - min_gain):
                    best, best_ms, changed = cand, ms, True
            if stopped == "budget":
                break
        if stopped == "budget" or not changed:
            break
    return SearchResult(config=best, ms=best_ms, start_ms=start_ms, trials=trials, rounds=r, stopped=stopped)


def _same(a, b) -> bool:
    import torch
    if isinstance(a, (list, tuple)):
        return len(a) == len(b) and all(_same(x, y) for x, y in zip(a, b))
    if isinstance(a, torch.Tensor):
        if a.dtype.is_floating_point:
            return bool(torch.allclose(a, b, rtol=1e-12, atol=0.0))
        return bool(torch.equal(a, b))
    return a == b


class QueryTuner:
    """Times one query on graphs built under each candidate configuration.

    make_graph() builds a Graph with the library's current knobs (called
    again only when a build-time knob changes); run(G) launches the query on
    the current stream and returns its output tensors (results are compared
    with those of the starting configuration)."""

    def __init__(self, make_graph: Callable[[], object], run: Callable[[object], object], reps: int = 5,
                 warmup: int = 2):
        self.make_graph = make_graph
        self.run = run
        self.reps = reps
        self.warmup = warmup
        self._graphs: Dict[tuple, object] = {}
        self._want = None

    def _graph(self, cfg):
        bkey = tuple(sorted((k, v) for k, v in cfg.items() if k in BUILD_KNOBS))
        if bkey not in self._graphs:
            # keep one built graph at a time: large graphs hold a lot of memory
            for g in self._graphs.values():
                g.close()
            self._graphs.clear()
            self._graphs[bkey] = self.make_graph()
        return self._graphs[bkey]

    def measure(self, cfg: Dict[str, int]) -> float:
        import torch
        try:
            apply(cfg)
        except Exception as e:  # a value the library rejects
            raise ValueError(str(e))
        G = self._graph(cfg)
        out = None
        for _ in range(self.warmup):
            out = self.run(G)
        torch.cuda.synchronize()
        if self._want is None:
            self._want = _clone(out)
        elif not _same(out, self._want):
            raise RuntimeError("tuning configuration %r changed the query result" % (cfg,))
        ts = []
        s = torch.cuda.current_stream()
        for _ in range(self.reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            self.run(G)
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    def close(self):
        for g in self._graphs.values():
            g.close()
        self._graphs.clear()


def _clone(x):
    import torch
    if isinstance(x, (list, tuple)):
        return type(x)(_clone(y) for y in x)
    if isinstance(x, torch.Tensor):
        return x.clone()
    return x


def lookup(query: str, info: Dict[str, int], variant: str = "", n_graphs: int = 1,
           paths: Optional[Sequence[str]] = None, device: Optional[str] = None) -> Optional[dict]:
    """The cached tuning of `query` for graphs shaped like `info`, or None
    (user cache first, then the package's shipped tunings)."""
    key = cache_key(device or device_key(), query + (":" + variant if variant else ""), signature(info, n_graphs))
    for p in (paths or (default_cache_path(), shipped_cache_path())):
        hit = load_cache(p).get(key)
        if hit:
            rec = dict(hit)
            rec.update(source="cache", cache=p, key=key)
            return rec
    return None


def count_variant(n_tau: int, prune: bool) -> str:
    """Threshold counts run different visitors by threshold count (register
    counters up to 8, binned beyond), and pruning changes the work."""
    nt = 1 if n_tau <= 1 else 2 if n_tau <= 2 else 4 if n_tau <= 4 else 8 if n_tau <= 8 else 64
    return "nt%d-%s" % (nt, "pruned" if prune else "full")


def tune(make_graph, run, query: str, info: Dict[str, int], variant: str = "", n_graphs: int = 1,
         knobs: Optional[Sequence[str]] = None, cache_path: Optional[str] = None, use_cache: bool = True,
         reps: int = 5, warmup: int = 2, rounds: int = 2, min_gain: float = 0.02, budget_s: float = 120.0,
         log: Optional[Callable[[str], None]] = None, device: Optional[str] = None,
         measure: Optional[Callable[[Dict[str, int]], float]] = None) -> dict:
    """Finds (or loads) the best knob setting of `query` (a QUERY_KNOBS key;
    `variant` refines the cache key) for graphs shaped like `info` (a
    Graph.info() dict), applies it and returns a record {"config", "ms",
    "start_ms", "source", "key", ...}.  The search starts from the library's
    current setting.  `device` overrides the GPU part of the cache key and
    `measure` the timing of one configuration (both for tests)."""
    knobs = list(knobs or QUERY_KNOBS[query])
    space = {k: ALL_KNOBS[k] for k in knobs}
    key = cache_key(device or device_key(), query + (":" + variant if variant else ""), signature(info, n_graphs))
    path = cache_path or default_cache_path()
    if use_cache:
        rec = lookup(query, info, variant, n_graphs, paths=(path, shipped_cache_path()), device=device)
        if rec:
            apply(rec["config"])
            return rec
    start = current(knobs)
    qt = QueryTuner(make_graph, run, reps=reps, warmup=warmup) if measure is None else None
    try:
        res = coordinate_descent(measure or qt.measure, start, space, order=knobs, rounds=rounds,
                                 min_gain=min_gain, budget_s=budget_s)
    finally:
        if qt is not None:
            qt.close()
    apply(res.config)
    rec = {"config": res.config, "ms": res.ms, "start_ms": res.start_ms, "trials": len(res.trials),
           "rounds": res.rounds, "stopped": res.stopped, "key": key, "source": "search"}
    if log:
        log("autotune %s: %.3f ms -> %.3f ms with %s" % (key, res.start_ms, res.ms, res.config))
    if use_cache:
        save_cache(path, {key: {k: rec[k] for k in ("config", "ms", "start_ms", "trials", "rounds", "stopped")}})
    return rec


def tune_count(n, src, dst, k, taus, prune=True, **kw) -> dict:
    """Tunes the threshold count of a FIXED graph given as COO arrays (host
    or device; copied to the device once, rebuilt per build-time setting)."""
    import torch
    from . import Graph, _dev_u32
    dev = torch.device("cuda")
    src_d, dst_d, k_d = _dev_u32(src, dev), _dev_u32(dst, dev), _dev_u32(k, dev)
    out = torch.empty(2 * len(taus), dtype=torch.int64, device=dev)
    make = lambda: Graph(n, src_d, dst_d, k=k_d)
    G0 = make()
    info = G0.info()
    G0.close()
    return tune(make, lambda G: G.count_threshold_(taus, out, prune=prune), "count", info,
                variant=count_variant(len(taus), prune), **kw)
