"""The graph the GPU builds (forward CSR under Node Order, list order, pair
partition, work lists) checked entry by entry against a numpy construction
of the same definitions."""
import numpy as np
import pytest

import synth
from gpu_util import core_graph, mixed_graph, require_gpu

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
    # pair partition: every forward edge is one pair, owned by the endpoint
    # whose list is the table (the later one when pull is on and its list is
    # longer), streaming the other endpoint's list
    pull = ubt.get_tuning("pull")
    du, dv = cnt[lo], cnt[hi]
    own = np.where((pull == 1) & (dv > du), hi, lo)
    streamed = np.where(own == hi, lo, hi)
    pp = ex["pair_ptr"].astype(np.int64)
    assert pp[0] == 0 and np.array_equal(np.diff(pp), np.bincount(own, minlength=n))
    ppos = ex["pair_pos"].astype(np.int64)
    assert np.array_equal(np.sort(ppos), np.arange(m))
    e_of_pair = eid[ppos]  # input edge of every pair
    pair_owner = np.repeat(np.arange(n), np.diff(pp))
    assert np.array_equal(own[e_of_pair], pair_owner)
    assert np.array_equal(streamed[e_of_pair], ex["pair_streamed"].astype(np.int64))
    # work lists: owners with a table of >= 2 entries and at least one pair
    work = np.bincount(pair_owner, weights=cnt[ex["pair_streamed"].astype(np.int64)], minlength=n)
    lists = ex["lists"].astype(np.int64)
    npairs = np.diff(pp)
    assert np.array_equal(np.sort(lists), np.nonzero((cnt >= 2) & (npairs >= 1))[0])
    ng, nh, nm, ns = [int(x) for x in ex["list_sizes"]]
    assert ns == 0 and ng + nh + nm == lists.size
    thr = ubt.get_tuning("hub_threshold")
    bw = ubt.get_tuning("block_work")
    gthr = max(thr, ubt.get_tuning("smem_table_max") // 4)
    giant, block, med = lists[:ng], lists[ng:ng + nh], lists[ng + nh:]
    assert np.all(cnt[giant] > gthr)
    assert np.all((cnt[block] <= gthr) & ((cnt[block] > thr) | (work[block] > bw)))
    assert np.all((cnt[med] <= thr) & (work[med] <= bw))


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


@pytest.mark.parametrize("knobs", [{"warp_sort_max": 128}, {"warp_sort_max": 256},
                                   {"warp_sort_max": 512, "sort_smem_max": 256},
                                   {"warp_sort_max": 128, "sort_smem_max": 512}])
def test_layout_under_other_row_sorts(ubt, knobs):
    """Rows of 129..512 entries sorted by one warp or by one block (and, past
    sort_smem_max, in global memory) give the same layout.  The graph plants
    a 600-clique, so its forward rows reach every length class up to 599."""
    old = {k: ubt.get_tuning(k) for k in knobs}
    try:
        for k, v in knobs.items():
            ubt.set_tuning(k, v)
        s, d = core_graph(3000, 20000, 600, 15)
        k = synth.k_uniform(s.size, 16)
        G = ubt.Graph(3000, s, d, k=k)
        assert G.info()["max_out_degree"] > 512
        check_export(ubt, G, 3000, s, d, k=k)
        p = synth.p_uniform_f32(s.size, 17)
        check_export(ubt, ubt.Graph(3000, s, d, p=p), 3000, s, d, p=p)
    finally:
        for k, v in old.items():
            ubt.set_tuning(k, v)


def forward_rows(n, s, d):
    """Owner of every edge under Node Order (the endpoint with the smaller
    (degree, id)) and the length of each vertex's forward list."""
    deg = np.bincount(s, minlength=n) + np.bincount(d, minlength=n)
    a, b = s.astype(np.int64), d.astype(np.int64)
    ab = (deg[a] < deg[b]) | ((deg[a] == deg[b]) & (a < b))
    lo = np.where(ab, a, b)
    return lo, np.bincount(lo, minlength=n)


@pytest.mark.parametrize("lo,hi", [(2, 7), (10, 30), (40, 120), (140, 250), (270, 500), (520, 590)])
@pytest.mark.parametrize("kind", ["fixed", "real"])
def test_duplicate_edge_in_every_row_class(ubt, lo, hi, kind):
    """A repeated edge (reversed, another probability) in a forward row of
    each length class is refused with UBT_ERR_DUPLICATE_EDGE: lane groups,
    warp sorts, block sorts; FIXED rows check with a set before their one
    sort, REAL rows compare neighbours after theirs."""
    n = 3000
    s, d = core_graph(n, 20000, 600, 15)
    owner, length = forward_rows(n, s, d)
    cand = np.nonzero((length[owner] >= lo) & (length[owner] <= hi))[0]
    assert cand.size > 0
    e = int(cand[len(cand) // 2])
    s2 = np.concatenate([s, d[e:e + 1]])
    d2 = np.concatenate([d, s[e:e + 1]])
    if kind == "fixed":
        k = synth.k_uniform(s2.size, 18)
        k[-1] = (int(k[e]) + 12345) % 65537
        with pytest.raises(ubt.UbtError) as err:
            ubt.Graph(n, s2, d2, k=k)
    else:
        p = synth.p_uniform_f32(s2.size, 19)
        with pytest.raises(ubt.UbtError) as err:
            ubt.Graph(n, s2, d2, p=p)
    assert err.value.status == -3
    k0 = synth.k_uniform(s.size, 18)
    assert ubt.Graph(n, s, d, k=k0).guard() == 0  # the same graph without the copy builds


@pytest.mark.parametrize("knobs", [{"pull": 0}, {"block_work": 1}, {"hub_threshold": 2, "block_work": 1 << 30}])
def test_layout_under_other_partitions(ubt, knobs):
    old = {k: ubt.get_tuning(k) for k in knobs}
    try:
        for k, v in knobs.items():
            ubt.set_tuning(k, v)
        s, d = mixed_graph(3000, 30000, 5)
        k = synth.k_uniform(s.size, 6)
        check_export(ubt, ubt.Graph(3000, s, d, k=k), 3000, s, d, k=k)
    finally:
        for k, v in old.items():
            ubt.set_tuning(k, v)
