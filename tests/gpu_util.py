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
