"""Top-k query (Sec. 5): the K triangles of highest balance (unbalance)
probability against the oracle's full enumeration sorted by the same order
(P_bal descending / ascending, ties by (u, v, w)) -- identical whenever the
tied triangles at the K-th value fit the candidate buffer; otherwise the
records above the K-th value are identical and the rest are valid ties."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import mixed_graph, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ubt():
    return require_gpu()


def oracle_topk(n, s, d, k, K, which):
    uvw, cls, pb = oracle.enumerate_records(n, s, d, k, 0.5, 3)  # every triangle once, exact P_bal
    key = -pb if which == 1 else pb
    order = np.lexsort((uvw[:, 2], uvw[:, 1], uvw[:, 0], key))
    return uvw[order][:K], pb[order][:K]


def graphs():
    g = synth.config_graph("er2k")
    yield "er2k", g.n, g.src, g.dst, g.k
    s, d = synth.rmat(12, 16, 0.57, 0.19, 0.19, 3)
    yield "rmat12", 1 << 12, s, d, synth.quantise(synth.p_beta(s.size, 0.5, 0.5, 4))
    s, d = mixed_graph(3000, 30000, 5)
    k = synth.k_uniform(s.size, 6)
    r = synth.rng(8).random(s.size)
    k[r < 0.2] = 0          # many certain edges: many exact ties
    k[(r >= 0.2) & (r < 0.3)] = 65536
    yield "mixed_ties", 3000, s, d, k


@pytest.mark.parametrize("which", [1, 2])
def test_topk_matches_oracle(ubt, which):
    for name, n, s, d, k in graphs():
        G = ubt.Graph(n, s, d, k=k)
        T = oracle.num_triangles(n, s, d)
        for K in sorted({1, 7, 100, 1000, max(1, T - 1), T, T + 5}):
            want_uvw, want_pb = oracle_topk(n, s, d, k, K, which)
            rec = G.topk(K, which)
            assert rec.shape[0] == min(K, T), (name, K)
            got_uvw = np.stack([rec["u"], rec["v"], rec["w"]], axis=1).astype(np.uint32)
            assert np.array_equal(rec["p_bal"], want_pb), (name, K, which)
            assert np.array_equal(got_uvw, want_uvw), (name, K, which)
            assert np.all(rec["cls"] == which)
        assert G.guard() == 0


def test_topk_ties_beyond_the_buffer(ubt):
    """K_40 with one probability: 9,880 triangles share one value, more than
    the candidate buffer for K = 10 holds; any 10 distinct triangles answer."""
    n = 40
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    s = np.array([a for a, _ in pairs], dtype=np.uint32)
    d = np.array([b for _, b in pairs], dtype=np.uint32)
    k = np.full(len(pairs), 50000, dtype=np.uint32)
    G = ubt.Graph(n, s, d, k=k)
    _, _, pb = oracle.enumerate_records(n, s, d, k, 0.5, 3)
    for which in (1, 2):
        rec = G.topk(10, which)
        assert rec.shape[0] == 10
        assert np.all(rec["p_bal"] == pb[0])
        uvw = np.stack([rec["u"], rec["v"], rec["w"]], axis=1)
        assert np.unique(uvw, axis=0).shape[0] == 10
        assert np.all((uvw[:, 0] < uvw[:, 1]) & (uvw[:, 1] < uvw[:, 2]) & (uvw[:, 2] < n))
    assert math.comb(n, 3) == 9880


def test_topk_invalid(ubt):
    s, d = synth.er_graph(100, 500, 3)
    G = ubt.Graph(100, s, d, k=synth.k_uniform(500, 4))
    for K, which in [(0, 1), (5, 3)]:
        with pytest.raises(ubt.UbtError):
            G.topk(K, which)
    E = ubt.Graph(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32), k=np.zeros(0, np.uint32))
    assert E.topk(3, 1).shape[0] == 0


def oracle_vertex_topk(n, s, d, k, K, which, vertices):
    uvw, cls, pb = oracle.enumerate_records(n, s, d, k, 0.5, 3)
    out = []
    for v in vertices:
        sel = np.any(uvw == v, axis=1)
        u, p = uvw[sel], pb[sel]
        key = -p if which == 1 else p
        order = np.lexsort((u[:, 2], u[:, 1], u[:, 0], key))
        out.append((u[order][:K], p[order][:K]))
    return out


@pytest.mark.parametrize("which", [1, 2])
def test_vertex_topk_matches_oracle(ubt, which):
    for name, n, s, d, k in graphs():
        G = ubt.Graph(n, s, d, k=k, undirected=True)
        verts = np.unique(np.concatenate([synth.rng(3).integers(0, n, size=60), [0, n - 1]])).astype(np.uint32)
        deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=n)
        verts = np.unique(np.concatenate([verts, [int(np.argmax(deg))]])).astype(np.uint32)  # the largest hub too
        for K in (1, 5, 64):
            got = G.vertex_topk(verts, K, which)
            want = oracle_vertex_topk(n, s, d, k, K, which, verts)
            for v, g_rec, (w_uvw, w_pb) in zip(verts, got, want):
                assert g_rec.shape[0] == w_uvw.shape[0], (name, v, K)
                assert np.array_equal(g_rec["p_bal"], w_pb), (name, v, K, which)
                g_uvw = np.stack([g_rec["u"], g_rec["v"], g_rec["w"]], axis=1).astype(np.uint32)
                assert np.array_equal(g_uvw, w_uvw), (name, v, K, which)
        assert G.guard() == 0


def test_vertex_topk_chunked_tables(ubt):
    s, d = mixed_graph(3000, 30000, 21)
    k = synth.k_uniform(s.size, 22)
    old = ubt.get_tuning("smem_table_max")
    try:
        ubt.set_tuning("smem_table_max", 64)
        G = ubt.Graph(3000, s, d, k=k, undirected=True)
        deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=3000)
        verts = np.argsort(-deg)[:8].astype(np.uint32)   # rows far longer than one table
        got = G.vertex_topk(verts, 16, 1)
        want = oracle_vertex_topk(3000, s, d, k, 16, 1, verts)
        for g_rec, (w_uvw, w_pb) in zip(got, want):
            assert np.array_equal(g_rec["p_bal"], w_pb)
            assert np.array_equal(np.stack([g_rec["u"], g_rec["v"], g_rec["w"]], axis=1).astype(np.uint32), w_uvw)
    finally:
        ubt.set_tuning("smem_table_max", old)


@pytest.mark.parametrize("mode", [1, 2])
def test_vertex_topk_with_edge_index(ubt, mode):
    """Neighbour pairs looked up in the edge index (where cheaper: mode 1;
    for every neighbour: mode 2) give the same answers."""
    old = ubt.get_tuning("edge_index")
    try:
        ubt.set_tuning("edge_index", mode)
        for name, n, s, d, k in graphs():
            G = ubt.Graph(n, s, d, k=k, undirected=True, edge_index=True)
            deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=n)
            verts = np.unique(np.concatenate([synth.rng(4).integers(0, n, size=40), np.argsort(-deg)[:4],
                                              [0, n - 1]])).astype(np.uint32)
            for which in (1, 2):
                for K in (1, 64):
                    got = G.vertex_topk(verts, K, which)
                    want = oracle_vertex_topk(n, s, d, k, K, which, verts)
                    for v, g_rec, (w_uvw, w_pb) in zip(verts, got, want):
                        assert np.array_equal(g_rec["p_bal"], w_pb), (name, v, K, which)
                        g_uvw = np.stack([g_rec["u"], g_rec["v"], g_rec["w"]], axis=1).astype(np.uint32)
                        assert np.array_equal(g_uvw, w_uvw), (name, v, K, which)
            assert G.guard() == 0
    finally:
        ubt.set_tuning("edge_index", old)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_vertex_topk_chunked_tables_with_edge_index(ubt, mode):
    """Rows longer than one table: with the index every pair is looked up in
    it (modes 1, 2), without (mode 0) the table is built chunk by chunk."""
    s, d = mixed_graph(3000, 30000, 21)
    k = synth.k_uniform(s.size, 22)
    old = {x: ubt.get_tuning(x) for x in ("smem_table_max", "edge_index")}
    try:
        ubt.set_tuning("smem_table_max", 64)
        ubt.set_tuning("edge_index", mode)
        G = ubt.Graph(3000, s, d, k=k, undirected=True, edge_index=True)
        deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=3000)
        verts = np.concatenate([np.argsort(-deg)[:8], synth.rng(6).integers(0, 3000, size=24)]).astype(np.uint32)
        for which in (1, 2):
            got = G.vertex_topk(verts, 16, which)
            want = oracle_vertex_topk(3000, s, d, k, 16, which, verts)
            for g_rec, (w_uvw, w_pb) in zip(got, want):
                assert np.array_equal(g_rec["p_bal"], w_pb)
                assert np.array_equal(np.stack([g_rec["u"], g_rec["v"], g_rec["w"]], axis=1).astype(np.uint32),
                                      w_uvw)
        assert G.guard() == 0
    finally:
        for x, v in old.items():
            ubt.set_tuning(x, v)


@pytest.mark.parametrize("table_max, n_list", [(64, 3000), (4096, 3000), (64, 200)])
def test_vertex_topk_every_vertex(ubt, table_max, n_list):
    """Every vertex of the graph (or 200 drawn with repeats), with tables of
    64 slots (most rows longer than one table, pairs from the edge index) and
    of 4,096: the answers equal the oracle's for each vertex."""
    s, d = mixed_graph(3000, 30000, 21)
    k = synth.k_uniform(s.size, 22)
    old = ubt.get_tuning("smem_table_max")
    try:
        ubt.set_tuning("smem_table_max", table_max)
        G = ubt.Graph(3000, s, d, k=k, undirected=True, edge_index=True)
        verts = np.arange(3000, dtype=np.uint32) if n_list == 3000 else \
            synth.rng(9).integers(0, 3000, size=n_list).astype(np.uint32)
        got = G.vertex_topk(verts, 8, 1)
        want = oracle_vertex_topk(3000, s, d, k, 8, 1, verts)
        for v, g_rec, (w_uvw, w_pb) in zip(verts, got, want):
            assert np.array_equal(g_rec["p_bal"], w_pb), v
            assert np.array_equal(np.stack([g_rec["u"], g_rec["v"], g_rec["w"]], axis=1).astype(np.uint32), w_uvw), v
        assert G.guard() == 0
    finally:
        ubt.set_tuning("smem_table_max", old)
