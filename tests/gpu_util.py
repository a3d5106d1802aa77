"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14084_gb300 import _build
    _build.build()
    import paper_2602_14084_gb300 as ubt
    return ubt


def sort_records(rec):
    """GPU records (structured array) sorted by (u, v, w) as plain arrays."""
    uvw = np.stack([rec["u"], rec["v"], rec["w"]], axis=1).astype(np.uint32)
    order = np.lexsort((uvw[:, 2], uvw[:, 1], uvw[:, 0]))
    return uvw[order], rec["cls"][order].astype(np.uint32), rec["p_bal"][order]


def mixed_graph(n, m, seed):
    """Random graph with a clique and a star planted (long forward lists)."""
    import synth
    s, d = synth.er_graph(n, m, seed)
    g = synth.rng(seed + 7)
    clique = g.choice(n, size=min(n, 70), replace=False)
    extra = [(int(a), int(b)) for i, a in enumerate(clique) for b in clique[i + 1:]]
    hub = int(g.integers(0, n))
    extra += [(hub, int(x)) for x in g.choice(n, size=min(n - 1, 400), replace=False) if int(x) != hub]
    a = np.concatenate([s, np.array([e[0] for e in extra], dtype=np.uint32)])
    b = np.concatenate([d, np.array([e[1] for e in extra], dtype=np.uint32)])
    lo, hi = np.minimum(a, b).astype(np.int64), np.maximum(a, b).astype(np.int64)
    key = np.unique(lo * n + hi)
    src, dst = (key // n).astype(np.uint32), (key % n).astype(np.uint32)
    return synth.random_orientation(src, dst, seed + 9)


def core_graph(n, m, core, seed):
    """Random graph plus a clique on `core` seeded vertices (deduplicated,
    randomly oriented)."""
    import synth
    s, d = synth.er_graph(n, m, seed)
    c = np.sort(synth.rng(seed + 3).choice(n, size=core, replace=False)).astype(np.int64)
    iu = np.triu_indices(core, 1)
    a = np.concatenate([s.astype(np.int64), c[iu[0]]])
    b = np.concatenate([d.astype(np.int64), c[iu[1]]])
    key = np.unique(np.minimum(a, b) * n + np.maximum(a, b))
    return synth.random_orientation((key // n).astype(np.uint32), (key % n).astype(np.uint32), seed + 5)


def grad_report(got, want, gabs):
    """(ok mask, plain relative error per edge, edges where the floor applied)."""
    floor = 1e-3 * gabs
    tol = 1e-5 * np.maximum(np.abs(want), floor)
    ok = np.abs(got - want) <= tol + 1e-12
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    return ok, rel, int(np.count_nonzero(floor > np.abs(want)))


def difference_quotients(ubt, G, p, edges):
    """(E_bal(p_e = 1) - E_bal(p_e = 0)) for each listed edge, from the GPU
    forward, in float64."""
    import torch
    base = torch.from_numpy(p.copy()).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    fd = np.zeros(len(edges))
    for i, e in enumerate(edges):
        vals = []
        for x in (1.0, 0.0):
            q = base.clone()
            q[int(e)] = x
            G.set_edge_values_(q)
            G.expected_counts_(out)
            vals.append(out[0].item())
        fd[i] = vals[0] - vals[1]
    G.set_edge_values_(base)
    return fd
