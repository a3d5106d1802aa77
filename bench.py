"""Benchmark of the exact t-count path on one GB300 (or N replicas).

Workload (one "step" = one threshold-count query over the whole graph):
  rmat22: R-MAT scale 22, edge factor 16, (a, b, c) = (0.57, 0.19, 0.19),
  symmetrised and deduplicated (4,194,304 vertices, 64.2M edges, 2.11e9
  triangles), P+ ~ 0.5 Beta(8,2) + 0.5 Beta(2,8) quantised to k/65536; the 32
  thresholds t_i = 0.51 + i 0.48/31 (i = 0..31) answered in one traversal
  with probability pruning.  The unpruned query runs too (not timed as the
  headline) and must give identical counts.

value  = triangles of the graph / query time (triangles per second), the
         graph already built and resident in HBM (the paper pre-sorts its data
         and times queries, Sec. 7.2).  L2 is flushed between timed steps.
e2e    = the same metric through ubt_count_host from pinned host buffers:
         H2D copy of (src, dst, k), graph build, query, D2H of the counts.
extras = the t = 0.9 enumeration on the same graph, the Chung-Lu n=1e6
         4-threshold query, MC sign worlds, the ego-net batch, expected counts
         forward + backward, Alg. 2, the samplers, top-k and the distribution
         study (--extras, on by default; --no-extras skips).

cpu_baseline / --impl reference: the CPU oracle (plain C, Alg. 1's outer
loop over all host cores) on a bounded sample of the same workload: the
triangles whose earliest vertex in Node Order falls in one of 16 hash classes
of the vertices.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEP32 = [0.51 + i * (0.48 / 31) for i in range(32)]   # 32 thresholds in [0.51, 0.99]
TAUS = SWEEP32
WORKLOAD = "rmat22"
METRIC = "exact t-count triangles/s (R-MAT scale 22, 32 thresholds in one launch, pruned)"
UNIT = "triangles/s"
CL1M_TAUS = [0.55, 0.70, 0.85, 0.95]
CPU_SAMPLE_MOD = 16   # the CPU arms count one of 16 hash classes of the vertices per pass


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "ubt_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources the counting traversal (k_traverse) and the graph layout it
# reads are built from; the AEO, sampling, world and no-allocation kernels
# live in the others
COUNT_SOURCES = ("ubt_api.cu", "ubt_build.cu", "ubt_internal.cuh", "ubt_query.cu", "ubt_scan.cu",
                 "ubt_traverse.cuh")


def csrc_digest(files=None):
    """Digest of the CUDA sources (all, or the named files): ncu counters
    apply only to the kernels they were taken on."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2602_14084_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")) and (files is None or f in files):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def tuned(ubt, query, variant, make, run, args, budget_s=None):
    """Knob setting of one benchmark query: from the package's shipped tunings
    when this GPU and graph shape are in it, else by a bounded autotuner
    search (written to the package's tunings with --tune).  Applies it and
    returns the autotuner's record (without the trial list)."""
    from paper_2602_14084_gb300 import autotune as at
    G0 = make()
    info, ng = G0.info(), getattr(G0, "n_graphs", 1)
    G0.close()
    del G0
    if args.no_tune:
        return {"source": "defaults", "config": at.current(at.QUERY_KNOBS[query])}
    path = at.shipped_cache_path() if args.tune else at.default_cache_path()
    rec = at.tune(make, run, query, info, variant=variant, n_graphs=ng, cache_path=path,
                  use_cache=not args.tune, budget_s=budget_s or args.tune_budget,
                  reps=3 if query in ("worlds", "batch") else 5, warmup=1 if query in ("worlds", "batch") else 2,
                  log=lambda msg: print(msg, file=sys.stderr, flush=True))
    if args.tune:
        at.save_cache(path, {rec["key"]: {k: rec[k] for k in ("config", "ms", "start_ms", "trials", "rounds",
                                                                "stopped")}})
    return rec




def merge_model_bytes(n, src, dst):
    """Bytes of Alg. 1 under the merge model of its analysis (Sec. 4): every
    forward edge u -> v reads both forward lists once, 8 B per entry, i.e.
    8 * sum over forward edges of (d+(u) + d+(v)).  Forward = from the earlier
    endpoint in Node Order (degree, then id)."""
    a, b = np.asarray(src, dtype=np.int64), np.asarray(dst, dtype=np.int64)
    deg = np.bincount(a, minlength=n) + np.bincount(b, minlength=n)
    a_first = (deg[a] < deg[b]) | ((deg[a] == deg[b]) & (a < b))
    u, v = np.where(a_first, a, b), np.where(a_first, b, a)
    dplus = np.bincount(u, minlength=n)
    return 8 * int(dplus[u].sum() + dplus[v].sum())


def alg_bytes_of(st):
    """Algorithmic bytes of one traversal (ubt_traversal_stats sizes): 8 B per
    table entry, 24 B per pair (its pair word, its edge's CSR entry and the
    streamed list's two offsets), 8 B per streamed entry."""
    return 8 * st["table_entries"] + 24 * st["pairs"] + 8 * st["streamed"]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch (read + write) from the committed ncu summary of
    this kernel and workload, or None when the kernels changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f).get("%s %s" % (kernel, workload))
    except Exception:
        return None
    if not rec or rec.get("count_sources_digest") != csrc_digest(COUNT_SOURCES):
        return None
    return rec["dram_bytes_per_launch"]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device="cuda"):
    """The largest of every rank's x: the job takes as long as its slowest
    replica (all ranks call this; one all-reduce)."""
    if ws == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, t_max, ws):
    """Weak scaling, replicas only: every rank processes the same workload, so
    the job's throughput is all ranks' units over the slowest rank's time."""
    return ws * units_per_rank / t_max


def make_graph(name):
    import synth
    return synth.config_graph(name, seed=1)


def workload_config(g, T, ws):
    """The `config` of the benchmark line (both arms time this workload)."""
    return {"workload": "rmat22: R-MAT scale 22, edge factor 16, (0.57,0.19,0.19,0.05), symmetrised and "
                        "deduplicated, P+ ~ 0.5 Beta(8,2) + 0.5 Beta(2,8) -> k/65536; 32 thresholds "
                        "t_i = 0.51 + i 0.48/31 in one traversal, pruned",
            "n": g.n, "m": g.m, "triangles": T, "n_taus": len(TAUS), "taus": "0.51 + i*0.48/31, i = 0..31",
            "l2": "inputs larger than L2 (513 MB of forward lists) and L2 flushed between steps (512 MB write)",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def golden_sweep(g):
    """The oracle's stored counts of the headline workload (written by
    tests/golden/make_fullsize_golden.py), if they were made for this input."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "rmat22_sweep32.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    import hashlib
    h = hashlib.sha256()
    for a in (g.src, g.dst, g.k):
        h.update(np.ascontiguousarray(a, dtype=np.uint32).tobytes())
    return rec if rec.get("input_digest") == h.hexdigest()[:24] else None


def count_kernel_name(ubt, n_tau):
    """The counting traversal the current tuning launches."""
    v = ubt.get_tuning("count_visitor")
    if v == 1:
        return "k_traverse<CountReg<%d>>" % (1 if n_tau <= 1 else 2 if n_tau <= 2 else 4 if n_tau <= 4 else 8) \
            if n_tau <= 8 else "k_traverse<CountMulti>"
    return "k_traverse<CountBins>"


def cpu_sample_desc(tri, mod=CPU_SAMPLE_MOD):
    return ("R-MAT scale 22, 32 thresholds: the %d triangles whose earliest vertex in Node Order falls in one of "
            "%d hash classes of the vertices (Alg. 1's outer loop over that class), graph built beforehand"
            % (tri, mod))


class no_gc:
    """Python's garbage collector off inside a timed loop (as timeit does), so
    that a collection pause between two launches is not timed as GPU work."""

    def __enter__(self):
        import gc
        self.was = gc.isenabled()
        gc.disable()

    def __exit__(self, *exc):
        import gc
        if self.was:
            gc.enable()


def time_steps(fn, steps, warmup, flush=None):
    """W untimed warm-up calls, then `steps` calls each bracketed by CUDA
    events on the current stream, with an L2 flush before each (untimed)."""
    with no_gc():
        return _time_steps(fn, steps, warmup, flush)


def _time_steps(fn, steps, warmup, flush=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    s = torch.cuda.current_stream()
    for _ in range(steps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    return times


def reference_arm(args):
    """CPU oracle as the comparison arm (rank 0 only): each step counts one
    hash class of 16 of the workload's vertices (Alg. 1 from those vertices,
    all host cores), on the graph built beforehand."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    g = make_graph(WORKLOAD)
    R = oracle.ResidentGraph(g.n, g.src, g.dst)
    th = oracle.threads()
    for i in range(args.warmup):
        R.count(g.k, TAUS, threads=th, sample_mod=CPU_SAMPLE_MOD, sample_rem=i % CPU_SAMPLE_MOD)
    times, tris = [], []
    for i in range(args.steps):
        t0 = time.perf_counter()
        _, _, tri = R.count(g.k, TAUS, threads=th, sample_mod=CPU_SAMPLE_MOD, sample_rem=i % CPU_SAMPLE_MOD)
        times.append(time.perf_counter() - t0)
        tris.append(tri)
    R.close()
    v = float(np.sum(tris)) / float(np.sum(times))
    ms = 1e3 * float(np.mean(times))
    T = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", "rmat22_sweep32.json")) as f:
            T = json.load(f)["triangles"]
    except Exception:
        pass
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(g, T, 1),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "cpu": cpu_model(),
                         "sample": "per step " + cpu_sample_desc(int(np.mean(tris)))},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--extras", dest="extras", action="store_true", default=True)
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu", action="store_false", default=True)
    ap.add_argument("--only", default=None,
                    choices=["count", "count32", "count-unpruned", "worlds", "expected", "backward", "enumerate",
                             "aeo", "aeo-tables", "edge-sampling", "vertex-sampling", "topk", "build", "batch"],
                    help="profiling driver: build the --workload graph, run one form of the query "
                         "--warmup + --steps times, print its mean time and exit")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="graph of the profiling driver: cl1m, rmat22, rmat20, cl4m, er2k, or a smaller "
                         "rmat<s> (k uniform) / rmat<s>m (rmat22's probability mixture)")
    ap.add_argument("--knob", action="append", default=[], metavar="NAME=VALUE",
                    help="profiling driver: set a tuning knob after the shipped tuning is applied (repeatable)")
    ap.add_argument("--digest", action="store_true", help="print the CUDA-source digest and exit")
    ap.add_argument("--tune", action="store_true",
                    help="search the knobs of every benchmark query (no cache) and store the results in the "
                         "package's shipped tunings, then run the benchmark with them")
    ap.add_argument("--no-tune", dest="no_tune", action="store_true", help="run with the library's default knobs")
    ap.add_argument("--tune-budget", type=float, default=60.0, help="seconds of autotuner search per query "
                    "when the shipped tunings do not cover this GPU and graph")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.digest:
        print(csrc_digest())
        return 0
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_14084_gb300 as ubt

    if args.only:
        return profile_driver(ubt, args)
    from paper_2602_14084_gb300 import autotune as at
    args.lib_defaults = at.current()
    g = make_graph(WORKLOAD)
    src_d = torch.from_numpy(g.src.view(np.int32)).cuda()
    dst_d = torch.from_numpy(g.dst.view(np.int32)).cuda()
    k_d = torch.from_numpy(g.k.view(np.int32)).cuda()
    counts = torch.empty(2 * len(TAUS), dtype=torch.int64, device="cuda")
    tuning = tuned(ubt, "count", at.count_variant(len(TAUS), True), lambda: ubt.Graph(g.n, src_d, dst_d, k=k_d),
                   lambda G_: G_.count_threshold_(TAUS, counts, prune=True), args)
    t0 = time.perf_counter()
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    # rebuild timed with events (first build includes library/context warm-up)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    G2 = ubt.Graph(g.n, src_d, dst_d, k=k_d)
    b.record()
    b.synchronize()
    build_ms = a.elapsed_time(b)
    del G2

    info = G.info()
    _, _, T, _ = G.expected_counts(with_exact=True)
    cb, cu = G.count_threshold(TAUS, prune=True)
    ub_, uu_ = G.count_threshold(TAUS, prune=False)
    assert np.array_equal(cb, ub_) and np.array_equal(cu, uu_), "pruned and unpruned counts differ"

    flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def flush():
        flush_buf.fill_(1)

    def step():
        G.count_threshold_(TAUS, counts, prune=True)

    def step_unpruned():
        G.count_threshold_(TAUS, counts, prune=False)

    clocks = Clocks(dev if ws == 1 else local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = time_steps(step, args.steps, args.warmup, flush)
    clk = clocks.stop()
    t_step = max_over_ranks(float(np.mean(times)), ws)
    times_unpruned = time_steps(step_unpruned, max(3, args.steps // 4), 1, flush)

    # roofline of the dominant kernel (the traversal): algorithmic bytes =
    # 8 B per table entry loaded + 24 B per pair (pair word, its edge's entry,
    # the streamed list's offsets) + 8 B per streamed entry
    st = G.traversal_stats(TAUS, prune=True)
    alg_bytes = alg_bytes_of(st)
    pk, pk_kind = peaks()
    achieved = alg_bytes / t_step / 1e9
    kname = count_kernel_name(ubt, len(TAUS))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": ncu_traffic(kname, WORKLOAD),
                "kernel": kname, "peak_kind": pk_kind,
                "alg_bytes_per_launch": alg_bytes, "streamed_entries": st["streamed"],
                "table_entries": st["table_entries"], "pairs": st["pairs"],
                "alg1_probes": info["wedges"],
                "merge_model_bytes": merge_model_bytes(g.n, g.src, g.dst)}
    st0 = G.traversal_stats(TAUS, prune=False)
    golden = golden_sweep(g)
    if golden is not None:
        assert np.array_equal(cb, golden["balanced"]) and np.array_equal(cu, golden["unbalanced"]), \
            "GPU counts differ from the oracle's stored counts"
        assert T == golden["triangles"]

    # the enumeration of C3 (t = 0.9, both classes) on the same graph
    nb9, nu9 = G.count_threshold([0.9])
    cap = int(nb9[0] + nu9[0])
    recbuf = torch.empty(max(cap, 1) * ubt.TRI_REC_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    found = ctypes.c_int64(0)

    def enum():
        r = ubt.lib().ubt_enumerate(G.handle, 0.9, 3, 1, ctypes.c_void_p(recbuf.data_ptr()), cap,
                                    ctypes.byref(found), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert r == 0, r

    enum_ms = _events_ms(enum, max(3, args.steps // 4), 1, flush)
    assert found.value == cap
    del recbuf

    # end to end through the C ABI from pinned host buffers
    hs = torch.from_numpy(g.src.view(np.int32)).pin_memory()
    hd = torch.from_numpy(g.dst.view(np.int32)).pin_memory()
    hk = torch.from_numpy(g.k.view(np.int32)).pin_memory()
    L = ubt.lib()
    nb = ctypes.c_size_t(0)
    L.ubt_count_host_workspace_size(g.n, g.m, ctypes.byref(nb))
    ews = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    tau_arr = np.asarray(TAUS, dtype=np.float64)
    hout = torch.zeros(2 * len(TAUS), dtype=torch.int64).pin_memory()

    def e2e_step():
        stv = L.ubt_count_host(g.n, g.m, ctypes.c_void_p(hs.data_ptr()), ctypes.c_void_p(hd.data_ptr()),
                               ctypes.c_void_p(hk.data_ptr()), tau_arr.ctypes.data_as(ctypes.c_void_p),
                               len(TAUS), 1, ctypes.c_void_p(hout.data_ptr()), ctypes.c_void_p(ews.data_ptr()),
                               ews.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert stv == 0, stv

    e2e_times = []
    e2e_clocks = Clocks(dev if ws == 1 else local)
    e2e_clocks.start()
    with no_gc():
        for i in range(args.warmup + max(10, args.steps)):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e2e_step()
            t2 = time.perf_counter()
            if i >= args.warmup:
                e2e_times.append(t2 - t1)
    e2e_clk = e2e_clocks.stop()
    assert np.array_equal(hout.numpy()[:len(TAUS)], cb)
    e2e_t = max_over_ranks(float(np.mean(e2e_times)), ws)
    # the copy part alone: the same three pinned arrays to device buffers
    dsrc, ddst, dk = torch.empty_like(src_d), torch.empty_like(dst_d), torch.empty_like(k_d)

    def h2d():
        dsrc.copy_(hs, non_blocking=True)
        ddst.copy_(hd, non_blocking=True)
        dk.copy_(hk, non_blocking=True)

    h2d_ms = _events_ms(h2d, 5, 1)
    del dsrc, ddst, dk

    line = {
        "metric": METRIC, "value": job_throughput(T, t_step, ws), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(g, T, ws),
        "roofline": roofline,
        "e2e": {"value": job_throughput(T, e2e_t, ws), "unit": UNIT, "h2d_bytes_per_step": 12 * g.m,
                "d2h_bytes_per_step": 16 * len(TAUS), "ms_per_step": 1e3 * e2e_t,
                "ms_per_step_min": 1e3 * float(np.min(e2e_times)),
                "ms_per_step_all": [round(1e3 * x, 2) for x in e2e_times], "h2d_ms": h2d_ms, "clocks": e2e_clk,
                "includes": "H2D of src/dst/k, graph build (validate, orient, CSR, sort), query, D2H"},
        # per query: the block-task traversal (giant / hub owners), the
        # warp-task traversal (medium owners; this workload has both) and the
        # kernel that turns the bins into counts
        "gpu_launches": args.steps * ((1 if info["hub_vertices"] > 0 else 0) + 1 + 1),
        "clocks": clk,
        "build_ms": build_ms,
        "tuning": {k: tuning[k] for k in ("source", "config", "key") if k in tuning},
        "unpruned": {"ms_per_step": 1e3 * float(np.mean(times_unpruned)),
                     "value": T / float(np.mean(times_unpruned)), "streamed_entries": st0["streamed"],
                     "alg_bytes": alg_bytes_of(st0)},
        "counts_match_oracle": ("equal to the oracle's stored counts (tests/golden/rmat22_sweep32.json)"
                                if golden is not None else "stored oracle counts are for another input"),
        "enumerate_0.9": {"ms": enum_ms, "records": cap, "record_bytes": 24 * cap,
                          "triangles_per_s": T / (enum_ms / 1e3)},
        "graph": info,
    }

    if args.extras and rank == 0:
        del G, ews, hs, hd, hk, src_d, dst_d, k_d
        _release()
        line["extras"] = extras(ubt, None, g, T, args, flush)
    if args.cpu and rank == 0:
        # the oracle as it stands, on all host cores, one hash class of 16 of
        # the vertices (about 1/16 of the work), the graph built beforehand
        import oracle
        oracle.build()
        R = oracle.ResidentGraph(g.n, g.src, g.dst)
        th = oracle.threads()
        t1 = time.perf_counter()
        _, _, tri = R.count(g.k, TAUS, threads=th, sample_mod=CPU_SAMPLE_MOD, sample_rem=0)
        dt = time.perf_counter() - t1
        R.close()
        line["cpu_baseline"] = {"value": tri / dt, "unit": UNIT, "cores": th, "kind": "oracle", "cpu": cpu_model(),
                                "sample": cpu_sample_desc(tri) + " (%.1f s)" % dt}
    if ws > 1:
        torch.distributed.barrier()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _events_ms(fn, steps, warmup, flush=None):
    return 1e3 * float(np.mean(time_steps(fn, steps, warmup, flush)))


def _release():
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def profile_driver(ubt, args):
    """One form of the query on one workload graph, for ncu captures."""
    import torch
    import synth
    from paper_2602_14084_gb300 import autotune as at
    g = make_graph(args.workload)
    taus = SWEEP32 if args.only == "count32" else CL1M_TAUS

    def build():
        if args.only in ("expected", "backward"):
            p = g.p if g.p is not None else synth.p_uniform_f32(g.m, 5)
            return ubt.Graph(g.n, g.src, g.dst, p=torch.from_numpy(np.ascontiguousarray(p)).cuda())
        k = g.k if g.k is not None else synth.quantise(g.p)
        return ubt.Graph(g.n, g.src, g.dst, k=k,
                         undirected=args.only in ("aeo", "aeo-tables", "edge-sampling", "vertex-sampling"),
                         edge_index=args.only in ("aeo", "vertex-sampling"))

    # the knobs the benchmark would use (cached tunings only: no search here)
    G = build()
    q = {"count": "count", "count32": "count", "count-unpruned": "count", "worlds": "worlds"}.get(args.only)
    rec = None
    if q and not args.no_tune:
        var = {"count": at.count_variant(len(CL1M_TAUS), True), "count32": at.count_variant(32, True),
               "count-unpruned": at.count_variant(len(CL1M_TAUS), False), "worlds": "W4096"}[args.only]
        rec = at.lookup(q, G.info(), var)
        if rec:
            at.apply(rec["config"])
    if rec or args.knob:
        at.apply({kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.knob})
        G.close()
        G = build()
    counts = torch.empty(2 * len(taus), dtype=torch.int64, device="cuda")
    eo = torch.empty(2, dtype=torch.float64, device="cuda")
    gout = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda")
    grad = torch.empty(g.m, dtype=torch.float32, device="cuda")
    W = 4096
    if args.only == "worlds":
        wws = torch.empty(G.sample_worlds_workspace(W), dtype=torch.uint8, device="cuda")
        wout = torch.empty(W, dtype=torch.int64, device="cuda")
    if args.only == "enumerate":
        nb, nu = G.count_threshold([0.9])
        cap = int(nb[0] + nu[0])
        recbuf = torch.empty(max(cap, 1) * ubt.TRI_REC_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        found = ctypes.c_int64(0)
    if args.only in ("edge-sampling", "vertex-sampling"):
        top = g.m if args.only == "edge-sampling" else g.n
        smp = torch.from_numpy(np.random.default_rng(1000).integers(0, top, size=10000).astype(np.int32)).cuda()
        lb = torch.empty(10000, dtype=torch.int64, device="cuda")
        lu = torch.empty(10000, dtype=torch.int64, device="cuda")
        le = torch.empty(2, dtype=torch.float64, device="cuda")
        lfn = ubt.lib().ubt_edge_local_counts if args.only == "edge-sampling" else ubt.lib().ubt_vertex_local_counts
        t08 = np.array([0.8])
    if args.only == "topk":
        nbytes = ctypes.c_size_t(0)
        ubt.lib().ubt_topk_workspace_size(1000, ctypes.byref(nbytes))
        twork = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        tout = torch.empty(1000 * ubt.TRI_REC_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        tn = ctypes.c_int64(0)
    cp = lambda t: ctypes.c_void_p(t.data_ptr())
    if args.only == "build":
        src_d = torch.from_numpy(g.src.view(np.int32)).cuda()
        dst_d = torch.from_numpy(g.dst.view(np.int32)).cuda()
        k_d = torch.from_numpy((g.k if g.k is not None else synth.quantise(g.p)).view(np.int32)).cuda()
        keep = []

        def build_once():  # the build kernels of ubt_create_graph (the graph itself is dropped)
            keep.clear()
            keep.append(ubt.Graph(g.n, src_d, dst_d, k=k_d))
    if args.only == "batch":
        # 500 ego nets (50..5,000 vertices, log-uniform) of the workload graph
        sel = synth.ego_select(g.n, g.src, g.dst, 500, 50, 5000, 1)
        eg = synth.ego_induce_torch(g.n, g.src, g.dst, sel, device="cuda")
        kp = torch.from_numpy(g.k.view(np.int32)).cuda()
        Gb = ubt.Graph(int(eg["v_off"][-1].item()), eg["src"], eg["dst"], k=kp[eg["eid"].long()], edge_key=eg["eid"],
                       vertex_offsets=eg["v_off"])
        ng = Gb.n_graphs
        bcounts = torch.empty(ng * 6, dtype=torch.int64, device="cuda")
        bexp = torch.empty(ng * 2, dtype=torch.float64, device="cuda")
        bworlds = torch.empty(ng * 64, dtype=torch.int64, device="cuda")
    fn = {
        "build": lambda: build_once() if args.only == "build" else None,
        "batch": lambda: Gb.batch_query_([0.6, 0.75, 0.9], 11, bcounts, bexp, bworlds) if args.only == "batch" else None,
        "count": lambda: G.count_threshold_(taus, counts, prune=True),
        "count32": lambda: G.count_threshold_(taus, counts, prune=True),
        "count-unpruned": lambda: G.count_threshold_(taus, counts, prune=False),
        "worlds": lambda: G.sample_worlds_(7, W, wout, None, wws),
        "expected": lambda: G.expected_counts_(eo),
        "backward": lambda: G.expected_counts_backward_(gout, grad),
        "enumerate": lambda: ubt.lib().ubt_enumerate(G.handle, 0.9, 3, 1, cp(recbuf), cap, ctypes.byref(found),
                                                     None),
        "aeo": lambda: G.count_aeo_([0.8], counts),          # edge-index form (graph built with the index)
        "aeo-tables": lambda: G.count_aeo_([0.8], counts),   # owner-table form (no index)
        "edge-sampling": lambda: lfn(G.handle, cp(smp), 10000, t08.ctypes.data_as(ctypes.c_void_p), 1, cp(lb),
                                     cp(lu), cp(le), None),
        "vertex-sampling": lambda: lfn(G.handle, cp(smp), 10000, t08.ctypes.data_as(ctypes.c_void_p), 1, cp(lb),
                                       cp(lu), cp(le), None),
        "topk": lambda: ubt.lib().ubt_topk(G.handle, 1000, 1, cp(tout), ctypes.byref(tn), cp(twork), twork.numel(),
                                           None),
    }[args.only]
    times = time_steps(fn, args.steps, args.warmup)
    print(json.dumps({"only": args.only, "workload": args.workload, "ms": 1e3 * float(np.mean(times)),
                      "guard": G.guard(), "tuning": at.current(at.QUERY_KNOBS.get(q or "count", []))}))
    return 0


def extra_cl1m(ubt, args, flush):
    """Chung-Lu n = 1e6 (gamma 2.1, mean degree 20, cap 50,000), P+ ~
    Beta(0.5, 0.5): the 4-threshold query (t = 0.55, 0.70, 0.85, 0.95) pruned
    and unpruned, its roofline and end to end through ubt_count_host (the
    counts are checked against the oracle in tests/test_gpu_fullsize.py)."""
    import torch
    from paper_2602_14084_gb300 import autotune as at
    g = make_graph("cl1m")
    out = torch.empty(2 * len(CL1M_TAUS), dtype=torch.int64, device="cuda")
    tuning = tuned(ubt, "count", at.count_variant(len(CL1M_TAUS), True), lambda: ubt.Graph(g.n, g.src, g.dst, k=g.k),
                   lambda G_: G_.count_threshold_(CL1M_TAUS, out, prune=True), args)
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    _, _, T, _ = G.expected_counts(with_exact=True)
    steps = max(3, args.steps // 2)
    ms = _events_ms(lambda: G.count_threshold_(CL1M_TAUS, out, prune=True), steps, 3, flush)
    b, u = out.cpu().numpy()[:4], out.cpu().numpy()[4:]
    ms0 = _events_ms(lambda: G.count_threshold_(CL1M_TAUS, out, prune=False), steps, 1, flush)
    b0, u0 = out.cpu().numpy()[:4], out.cpu().numpy()[4:]
    assert np.array_equal(b, b0) and np.array_equal(u, u0), "pruned and unpruned counts differ"
    st = G.traversal_stats(CL1M_TAUS, prune=True)
    alg = alg_bytes_of(st)
    pk, pk_kind = peaks()
    del G
    _release()
    e2e_ms = []
    with no_gc():
        for i in range(4):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ubt.count_host(g.n, g.src, g.dst, g.k, CL1M_TAUS)
            if i:
                e2e_ms.append(1e3 * (time.perf_counter() - t1))
    res = {"workload": "Chung-Lu n=1,000,000 gamma=2.1 mean-deg 20 cap 50,000, P+ ~ Beta(0.5,0.5) -> k/65536, "
                       "4 thresholds in one traversal",
           "n": g.n, "m": g.m, "triangles": T, "ms": ms, "triangles_per_s": T / (ms / 1e3), "unpruned_ms": ms0,
           "alg_bytes": alg, "streamed_entries": st["streamed"], "achieved_gbs": alg / (ms / 1e3) / 1e9,
           "frac_hbm": alg / (ms / 1e3) / 1e9 / pk["hbm_gbs"], "peak_kind": pk_kind,
           "kernel": count_kernel_name(ubt, 4), "e2e_ms": float(np.mean(e2e_ms)),
           "e2e_note": "ubt_count_host from pageable numpy arrays (H2D, build, query, D2H), host wall time",
           "balanced": b.tolist(), "unbalanced": u.tolist(),
           "tuning": {k: tuning[k] for k in ("source", "config") if k in tuning}}
    return res


def extra_worlds(ubt, args, flush):
    """R-MAT scale 20 with k ~ U{0..65536}: W = 4096 bit-sliced sign worlds."""
    import torch
    g = make_graph("rmat20")
    W = 4096
    wout = torch.empty(W, dtype=torch.int64, device="cuda")
    wt = torch.empty(1, dtype=torch.int64, device="cuda")
    wbuf = {}

    def run(G_):
        # the workspace depends on the words per pass: sized per call
        need = G_.sample_worlds_workspace(W)
        if wbuf.get("n", -1) < need:
            wbuf["ws"] = torch.empty(need, dtype=torch.uint8, device="cuda")
            wbuf["n"] = need
        return G_.sample_worlds_(7, W, wout, wt, wbuf["ws"])

    tuning = tuned(ubt, "worlds", "W%d" % W, lambda: ubt.Graph(g.n, g.src, g.dst, k=g.k), run, args)
    wbuf.clear()
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    eb, eu, T, _ = G.expected_counts(with_exact=True)
    wws = torch.empty(G.sample_worlds_workspace(W), dtype=torch.uint8, device="cuda")
    ms = _events_ms(lambda: G.sample_worlds_(7, W, wout, wt, wws), max(3, args.steps // 4), 1, flush)
    c = wout.cpu().numpy().astype(np.float64)
    z = (c.mean() - eb) / (c.std(ddof=1) / np.sqrt(W))
    res = {"workload": "R-MAT scale 20, edge factor 16, k ~ U{0..65536}", "n": g.n, "m": g.m, "triangles": T,
           "W": W, "ms": ms, "world_triangles_per_s": T * W / (ms / 1e3),
           "words_per_pass": ubt.get_tuning("world_words_per_pass"),
           "mc_mean_minus_exact_in_standard_errors": float(z),
           "tuning": {k: tuning[k] for k in ("source", "config") if k in tuning}}
    del G, wws
    _release()
    return res


EGO_TAUS = [0.6, 0.75, 0.9]


def extra_ego(ubt, args, flush):
    """10,000 ego nets (50..5,000 vertices, log-uniform) of R-MAT scale 20,
    answered per graph -- counts at 3 thresholds, exact expected counts and
    the 64 worlds of world word 0 -- by one replay of a captured CUDA graph."""
    import torch
    import synth
    g = make_graph("rmat20")
    t0 = time.perf_counter()
    sel = synth.ego_select(g.n, g.src, g.dst, 10000, 50, 5000, 1)
    eg = synth.ego_induce_torch(g.n, g.src, g.dst, sel, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    kp = torch.from_numpy(g.k.view(np.int32)).cuda()
    kb = kp[eg["eid"].long()]
    nv = int(eg["v_off"][-1].item())

    def make():
        return ubt.Graph(nv, eg["src"], eg["dst"], k=kb, edge_key=eg["eid"], vertex_offsets=eg["v_off"])

    from paper_2602_14084_gb300 import autotune as at
    saved = at.current()
    ng = int(eg["v_off"].numel()) - 1
    counts = torch.empty(ng * 2 * len(EGO_TAUS), dtype=torch.int64, device="cuda")
    expect = torch.empty(ng * 2, dtype=torch.float64, device="cuda")
    worlds = torch.empty(ng * 64, dtype=torch.int64, device="cuda")
    def run(G_):  # returns the outputs, which the tuner compares across configurations
        G_.batch_query_(EGO_TAUS, 11, counts, expect, worlds)
        return counts, expect, worlds

    tuning = tuned(ubt, "batch", "ego10k", make, run, args)
    t0 = time.perf_counter()
    G = make()
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    assert G.n_graphs == ng
    m_total = G.m
    del kb, kp
    eg = {k: v for k, v in eg.items() if k in ("v_off",)}
    _release()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        G.batch_query_(EGO_TAUS, 11, counts, expect, worlds, stream=side)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(side)
    direct_ms = _events_ms(lambda: G.batch_query_(EGO_TAUS, 11, counts, expect, worlds), max(3, args.steps // 4), 1)
    ref = (counts.clone(), expect.clone(), worlds.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
        G.batch_query_(EGO_TAUS, 11, counts, expect, worlds, stream=side)
    counts.zero_(), expect.zero_(), worlds.zero_()
    replay_ms = _events_ms(graph.replay, max(3, args.steps // 4), 1)
    same = bool(torch.equal(counts, ref[0]) and torch.equal(expect, ref[1]) and torch.equal(worlds, ref[2]))
    tri = float((expect.view(ng, 2).sum(1)).sum().item())
    res = {"workload": "10,000 ego nets of R-MAT scale 20 (50..5,000 vertices, log-uniform), parent edge keys",
           "graphs": ng, "vertices": G.n, "edges": m_total, "triangles": int(round(tri)),
           "generate_s": gen_s, "build_s": build_s, "direct_ms": direct_ms, "graph_replay_ms": replay_ms,
           "replay_equals_direct": same, "triangles_per_s": tri / (replay_ms / 1e3),
           "outputs": "per graph: counts at %s, E_bal/E_unbal, 64 world counts" % EGO_TAUS,
           "tuning": {k: tuning[k] for k in ("source", "config") if k in tuning}}
    del G, graph, counts, expect, worlds
    _release()
    at.apply(saved)  # the later extras run with the knobs they had before
    return res


def extra_grad(ubt, args, flush):
    """Chung-Lu n = 4e6, gamma 2.3, p ~ U[0,1] float32: expected counts
    forward and the hand-written adjoint backward through autograd."""
    import torch
    g = make_graph("cl4m")
    pt = torch.from_numpy(g.p).cuda().requires_grad_(True)
    G = ubt.Graph(g.n, g.src, g.dst, p=pt.detach())
    steps = max(3, args.steps // 4)

    def fwd():
        with torch.no_grad():
            ubt.expected_counts(G, pt)

    def fwd_bwd():
        pt.grad = None
        eb, eu = ubt.expected_counts(G, pt)
        (eb - eu).backward()

    fms = _events_ms(fwd, steps, 1, flush)
    fbms = _events_ms(fwd_bwd, steps, 1, flush)
    eb, eu = ubt.expected_counts(G, pt)
    res = {"workload": "Chung-Lu n=4,000,000 gamma=2.3 mean-deg 20 cap 50,000, p ~ U[0,1] float32",
           "n": g.n, "m": g.m, "triangles": int(round(eb.item() + eu.item())), "fwd_ms": fms, "fwd_bwd_ms": fbms,
           "via": "torch.autograd.Function -> ubt_set_edge_values + ubt_expected_counts / "
                  "ubt_expected_counts_backward"}
    del G, pt
    _release()
    res["subgraph_gradient_check"] = grad_check_subgraph(ubt, g)
    return res


def grad_check_subgraph(ubt, g):
    """The adjoint's gradient on the subgraph induced by a BFS from a seeded
    vertex (>= 1,000 edges) against float64 difference quotients of the GPU
    forward: E is affine in each p_e, so E(p_e = 1) - E(p_e = 0) is dE/dp_e
    exactly up to the forward's rounding.  Tolerance per edge 1e-5 max(|g|,
    1e-3 A_e) with A_e = sum over the edge's triangles of |(1-2p_f)(1-2p_g)|,
    which is the gradient at p' = min(p, 1 - p) (there every factor is |1-2p|)."""
    import torch
    import synth
    deg = np.bincount(np.concatenate([g.src, g.dst]).astype(np.int64), minlength=g.n)
    start = int(synth.rng(61).choice(np.nonzero(deg >= 10)[0]))
    verts, ls, ld, eid = synth.bfs_induced(g.n, g.src, g.dst, start, 1000)
    p = np.ascontiguousarray(g.p[eid])
    base = torch.from_numpy(p.copy()).cuda()
    G = ubt.Graph(verts.size, ls, ld, p=base)
    gout = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda")
    grad = torch.empty(ls.size, dtype=torch.float32, device="cuda")

    def backward_at(q):
        G.set_edge_values_(q)
        G.expected_counts_backward_(gout, grad)
        return grad.double().cpu().numpy()

    got = backward_at(base)
    A = backward_at(torch.minimum(base, 1.0 - base).contiguous())
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    fd = np.zeros(ls.size)
    for e in range(ls.size):
        vals = []
        for x in (1.0, 0.0):
            q = base.clone()
            q[e] = x
            G.set_edge_values_(q)
            G.expected_counts_(out)
            vals.append(out[0].item())
        fd[e] = vals[0] - vals[1]
    floor = 1e-3 * A
    tol = 1e-5 * np.maximum(np.abs(fd), floor)
    nz = np.abs(fd) > 0
    rel = np.abs(got - fd)[nz] / np.abs(fd)[nz]
    res = {"vertices": int(verts.size), "edges": int(ls.size), "max_plain_relative_error": float(rel.max()),
           "median_plain_relative_error": float(np.median(rel)),
           "edges_using_the_floor": int(np.count_nonzero(floor > np.abs(fd))),
           "edges_outside_tolerance": int(np.count_nonzero(np.abs(got - fd) > tol + 1e-12)),
           "guard": G.guard()}
    del G
    _release()
    return res


AEO_TAUS = [0.55, 0.6, 0.7, 0.8, 0.9, 0.95]


def extra_aeo(ubt, args, flush, name):
    """Absolute-Edge-Order iteration (Alg. 2) against the degree-ordered
    pruned traversal, one threshold at a time (the paper's Fig. 6 axis)."""
    import torch
    g = make_graph(name)
    k = g.k if g.k is not None else __import__("synth").quantise(g.p)
    t0 = time.perf_counter()
    G = ubt.Graph(g.n, g.src, g.dst, k=k, undirected=True, edge_index=True)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    out = torch.empty(2, dtype=torch.int64, device="cuda")
    steps = max(3, args.steps // 4)
    rows = []
    old = ubt.get_tuning("edge_index")
    try:
        for t in AEO_TAUS:
            ms_deg = _events_ms(lambda: G.count_threshold_([t], out, prune=True), steps, 1, flush)
            a = out.cpu().numpy().copy()
            ubt.set_tuning("edge_index", 1)
            ms_aeo = _events_ms(lambda: G.count_aeo_([t], out), steps, 1, flush)
            b = out.cpu().numpy().copy()
            ubt.set_tuning("edge_index", 0)
            ms_tab = _events_ms(lambda: G.count_aeo_([t], out), steps, 1, flush)
            c = out.cpu().numpy().copy()
            assert np.array_equal(a, b) and np.array_equal(a, c), "AEO and degree-ordered counts differ"
            rows.append({"t": t, "degree_ms": ms_deg, "aeo_ms": ms_aeo, "aeo_tables_ms": ms_tab,
                         "balanced": int(a[0]), "unbalanced": int(a[1])})
    finally:
        ubt.set_tuning("edge_index", old)
    res = {"workload": name, "n": g.n, "m": g.m, "build_with_undirected_and_index_s": build_s, "per_t": rows,
           "note": "aeo_ms: edge-index form (each edge streams the shorter Lemma 3 window); "
                   "aeo_tables_ms: owner tables in shared memory"}
    del G
    _release()
    return res


def extra_sampling(ubt, args, flush):
    """Edge (eImpr) and vertex (vImpr) sampling on the Chung-Lu n=1e6 graph:
    10,000 uniform samples per estimate, t = 0.8; time per estimate and the
    mean absolute percentage error over 10 seeds against the exact counts."""
    import torch
    g = make_graph("cl1m")
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k, undirected=True, edge_index=True)
    tau = [0.8]
    exact_b, exact_u = G.count_threshold(tau)
    K = 10000
    res = {"workload": "cl1m, t = 0.8, 10,000 samples per estimate", "exact_balanced": int(exact_b[0]),
           "exact_unbalanced": int(exact_u[0])}
    for kind in ("edge", "vertex"):
        fn = G.edge_local_counts if kind == "edge" else G.vertex_local_counts
        top = g.m if kind == "edge" else g.n
        ests, times = [], []
        for seed in range(10):
            smp = torch.from_numpy(np.random.default_rng(1000 + seed).integers(0, top, size=K).astype(np.int32)).cuda()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            _, _, est = fn(smp, tau)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
            ests.append(est[:, 0])
        ests = np.array(ests)
        ape_b = np.abs(ests[:, 0] - exact_b[0]) / max(1, exact_b[0])
        ape_u = np.abs(ests[:, 1] - exact_u[0]) / max(1, exact_u[0])
        res[kind] = {"ms_per_estimate_median": float(np.median(times)), "mape_balanced": float(ape_b.mean()),
                     "mape_unbalanced": float(ape_u.mean()),
                     "note": "time includes the D2H of the per-sample counts"}
    # vertex sampling without the edge index (every neighbour's row streamed)
    old = ubt.get_tuning("edge_index")
    ubt.set_tuning("edge_index", 0)
    try:
        smp = torch.from_numpy(np.random.default_rng(1000).integers(0, g.n, size=K).astype(np.int32)).cuda()
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            G.vertex_local_counts(smp, tau)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        res["vertex"]["ms_per_estimate_without_edge_index"] = float(np.median(times))
    finally:
        ubt.set_tuning("edge_index", old)
    del G
    _release()
    return res


DIST_TAUS = [0.55, 0.6, 0.7, 0.8, 0.9, 0.95]


def dist_p(name, m, seed):
    import synth
    return {"uniform": lambda: synth.rng(seed).random(m),
            "normal": lambda: synth.p_normal(m, seed),
            "beta_0.5_0.5": lambda: synth.p_beta(m, 0.5, 0.5, seed),
            "beta_3_1": lambda: synth.p_beta(m, 3.0, 1.0, seed),
            "beta_1_3": lambda: synth.p_beta(m, 1.0, 3.0, seed)}[name]()


def extra_dist(ubt, args, flush):
    """Pruned counting time against t for five P+ distributions on the same
    Chung-Lu n=1e6 structure (the paper's Fig. 7 study on one graph)."""
    import torch
    import synth
    g = make_graph("cl1m")
    out = torch.empty(2, dtype=torch.int64, device="cuda")
    steps = max(3, args.steps // 4)
    res = {"workload": "cl1m structure, P+ redrawn per distribution, one threshold per launch"}
    for i, name in enumerate(("uniform", "normal", "beta_0.5_0.5", "beta_3_1", "beta_1_3")):
        k = synth.quantise(dist_p(name, g.m, 300 + i))
        G = ubt.Graph(g.n, g.src, g.dst, k=k)
        rows = []
        for t in DIST_TAUS:
            ms = _events_ms(lambda: G.count_threshold_([t], out, prune=True), steps, 1, flush)
            c = out.cpu().numpy()
            rows.append({"t": t, "ms": ms, "balanced": int(c[0]), "unbalanced": int(c[1])})
        res[name] = rows
        del G
        _release()
    return res


def extra_topk(ubt, args, flush):
    """Top-k most balanced / most unbalanced triangles of the Chung-Lu n=1e6
    graph (Sec. 5's top-k adaptation; the whole search, enumeration and sort)."""
    import torch
    g = make_graph("cl1m")
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    res = {"workload": "cl1m"}
    for K in (1000, 100000):
        for which in (1, 2):
            G.topk(K, which)  # warm-up
            times = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rec = G.topk(K, which)
                times.append(1e3 * (time.perf_counter() - t0))
            res["K%d_%s" % (K, "bal" if which == 1 else "unbal")] = {
                "ms_median": float(np.median(times)), "kth_p_bal": float(rec["p_bal"][-1]),
                "note": "host wall time of the synchronous call, D2H of the K records included"}
    del G
    _release()
    # per-vertex top-10 of 100,000 uniformly drawn vertices, with and without
    # the edge index
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k, undirected=True, edge_index=True)
    verts = torch.from_numpy(np.random.default_rng(5).integers(0, g.n, size=100000).astype(np.int32)).cuda()
    G.vertex_topk(verts[:1000], 10, 1)
    old = ubt.get_tuning("edge_index")
    out = {}
    try:
        for mode in (old, 0):
            ubt.set_tuning("edge_index", mode)
            times = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                G.vertex_topk(verts, 10, 1)
                times.append(1e3 * (time.perf_counter() - t0))
            out["ms_median" if mode else "ms_median_without_edge_index"] = float(np.median(times))
    finally:
        ubt.set_tuning("edge_index", old)
    res["vertex_top10_of_100k_vertices"] = dict(out, note="host wall time, D2H of 1M records included")
    del G
    _release()
    return res


def extras(ubt, G, g, T, args, flush):
    """The other workloads of the path, each on its own graph."""
    from paper_2602_14084_gb300 import autotune as at
    out = {}
    for name, fn in (("c2_cl1m", extra_cl1m), ("c4_rmat20_worlds", extra_worlds), ("c4_ego10k", extra_ego),
                     ("c5_cl4m_grad", extra_grad),
                     ("aeo_vs_degree_cl1m", lambda u, a, f: extra_aeo(u, a, f, "cl1m")),
                     ("aeo_vs_degree_rmat22", lambda u, a, f: extra_aeo(u, a, f, "rmat22")),
                     ("sampling_cl1m", extra_sampling), ("topk_cl1m", extra_topk),
                     ("distributions_cl1m", extra_dist)):
        try:
            with at.tuning_scope(args.lib_defaults):  # each workload starts from the library defaults
                out[name] = fn(ubt, args, flush)
        except Exception as e:  # report, do not hide: the line says what failed
            out[name] = {"error": repr(e)[:300]}
    return out


if __name__ == "__main__":
    sys.exit(main())
