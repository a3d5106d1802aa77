"""The graph the GPU builds (forward CSR under Node Order, list order, work
lists) checked entry by entry against a numpy construction of the same
definitions."""
import numpy as np
import pytest

import synth
from gpu_util import mixed_graph, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ubt():
    return require_gpu()


def expected_forward(n, s, d):
    """Node Order (degree, then id): each edge goes from its earlier endpoint."""
    deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=n)
    a, b = s.astype(np.int64), d.astype(np.int64)
    before = (deg[a] < deg[b]) | ((deg[a] == deg[b]) & (a < b))
    return np.where(before, a, b), np.where(before, b, a)


def check_export(ubt, G, n, s, d, k=None, p=None):
    ex = G.export()
    m = s.size
    lo, hi = expected_forward(n, s, d)
    cnt = np.bincount(lo, minlength=n)
    rp = ex["row_ptr"].astype(np.int64)
    assert rp[0] == 0 and np.array_equal(np.diff(rp), cnt)
    col, val, eid = ex["col"].astype(np.int64), ex["val"].astype(np.int64), ex["eid"].astype(np.int64)
    assert np.array_equal(np.sort(eid), np.arange(m))
    assert np.array_equal(hi[eid], col)
    assert np.array_equal(lo[eid], np.repeat(np.arange(n), cnt))
    owner = np.repeat(np.arange(n), cnt)
    same = owner[1:] == owner[:-1]
    if k is not None:
        q = 32768 - k.astype(np.int64)
        assert np.array_equal(q[eid], val)
        key = (32768 - np.abs(val)) * (1 << 32) + col
    else:
        want = np.rint((1.0 - 2.0 * p.astype(np.float64)) * 2.0 ** 30).astype(np.int64)
        assert np.array_equal(want[eid], val)
        key = col
    assert np.all(key[1:][same] > key[:-1][same])
    lists = ex["lists"].astype(np.int64)
    assert np.array_equal(np.sort(lists), np.nonzero(cnt >= 2)[0])
    ng, nh, nm, ns = [int(x) for x in ex["list_sizes"]]
    thr = ubt.get_tuning("hub_threshold")
    smax = ubt.get_tuning("short_max")
    block, med, short = lists[:ng + nh], lists[ng + nh:ng + nh + nm], lists[ng + nh + nm:]
    assert np.all(cnt[block] > thr)
    assert np.all((cnt[med] > smax) & (cnt[med] <= thr))
    assert np.all(cnt[short] <= smax) and np.all(np.diff(short) > 0)


@pytest.mark.parametrize("seed,n,m", [(1, 2000, 20000), (2, 5000, 100000), (3, 50, 1225)])
def test_fixed_graph_layout(ubt, seed, n, m):
    s, d = synth.er_graph(n, m, seed)
    k = synth.k_uniform(m, seed + 1)
    check_export(ubt, ubt.Graph(n, s, d, k=k), n, s, d, k=k)


def test_mixed_and_rmat_layout(ubt):
    s, d = mixed_graph(3000, 30000, 5)
    k = synth.k_uniform(s.size, 6)
    check_export(ubt, ubt.Graph(3000, s, d, k=k), 3000, s, d, k=k)
    s, d = synth.rmat(14, 16, 0.57, 0.19, 0.19, 3)
    k = synth.quantise(synth.p_beta(s.size, 0.5, 0.5, 4))
    check_export(ubt, ubt.Graph(1 << 14, s, d, k=k), 1 << 14, s, d, k=k)


def test_real_graph_layout(ubt):
    s, d = synth.er_graph(3000, 40000, 9)
    p = synth.p_uniform_f32(s.size, 10)
    p[:5] = [0.0, 1.0, 0.5, 1e-30, 2.0 ** -24]
    check_export(ubt, ubt.Graph(3000, s, d, p=p), 3000, s, d, p=p)


def test_long_lists_sorted_in_global_memory(ubt):
    """Lists longer than the shared-memory sort limit take the global-memory path."""
    old = ubt.get_tuning("sort_smem_max")
    try:
        ubt.set_tuning("sort_smem_max", 64)
        s, d = mixed_graph(3000, 30000, 5)
        k = synth.k_uniform(s.size, 6)
        G = ubt.Graph(3000, s, d, k=k)
        assert G.info()["max_out_degree"] > 64
        check_export(ubt, G, 3000, s, d, k=k)
        p = synth.p_uniform_f32(s.size, 7)
        check_export(ubt, ubt.Graph(3000, s, d, p=p), 3000, s, d, p=p)
    finally:
        ubt.set_tuning("sort_smem_max", old)
