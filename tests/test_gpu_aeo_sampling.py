"""The Absolute-Edge-Order iteration (Alg. 2) and the local counts of the
samplers (Algs. 3-6) against the oracle: counts and records bit-exact, local
counts of every sampled edge / vertex bit-exact, and the undirected layout
entry by entry against numpy."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import core_graph, mixed_graph, require_gpu, sort_records

pytestmark = pytest.mark.gpu

TAUS = [0.5, 0.6, 0.75, 0.9, 0.99, 1.0]
SWEEP32 = [0.51 + i * (0.48 / 31) for i in range(32)]


@pytest.fixture(scope="module")
def ubt():
    return require_gpu()


def cases():
    out = []
    g = synth.config_graph("er2k")
    out.append(("er2k", g.n, g.src, g.dst, g.k))
    s, d = synth.er_graph(300, 6000, 100)
    out.append(("er300", 300, s, d, synth.k_uniform(6000, 200)))
    s, d = mixed_graph(3000, 30000, 5)
    out.append(("mixed3000", 3000, s, d, synth.k_uniform(s.size, 6)))
    s, d = synth.rmat(12, 16, 0.57, 0.19, 0.19, 3)
    out.append(("rmat12", 1 << 12, s, d, synth.quantise(synth.p_beta(s.size, 0.5, 0.5, 4))))
    s, d = synth.chung_lu(20000, 2.1, 20.0, 2000.0, 3)
    k = synth.quantise(synth.p_beta_mixture(s.size, 4))
    out.append(("cl20k", 20000, s, d, k))
    return out


CASES = cases()


def with_knobs(ubt, knobs):
    class Scope:
        def __enter__(self):
            self.old = {k: ubt.get_tuning(k) for k in knobs}
            for k, v in knobs.items():
                ubt.set_tuning(k, v)

        def __exit__(self, *e):
            for k, v in self.old.items():
                ubt.set_tuning(k, v)
    return Scope()


@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_undirected_layout(ubt, case):
    name, n, s, d, k = case
    G = ubt.Graph(n, s, d, k=k, undirected=True)
    ex = G.export_undirected()
    m = s.size
    deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=n)
    up = ex["uptr"].astype(np.int64)
    assert up[0] == 0 and np.array_equal(np.diff(up), deg)
    row = np.repeat(np.arange(n), deg)
    col, val, eid, mir = (ex[x].astype(np.int64) for x in ("col", "val", "eid", "mirror"))
    # every input edge twice, once in each endpoint's row
    assert np.array_equal(np.bincount(eid, minlength=m), np.full(m, 2))
    a, b = s.astype(np.int64)[eid], d.astype(np.int64)[eid]
    assert np.all(((row == a) & (col == b)) | ((row == b) & (col == a)))
    assert np.array_equal(val, 32768 - k.astype(np.int64)[eid])
    # rows in Absolute Edge Order: |q| descending, then neighbour id
    key = (32768 - np.abs(val)) * (1 << 32) + col
    same = row[1:] == row[:-1]
    assert np.all(key[1:][same] > key[:-1][same])
    # mirrors
    assert np.array_equal(mir[mir], np.arange(2 * m))
    assert np.array_equal(eid[mir], eid) and np.array_equal(row[mir], col)
    # AEO owners: the endpoint with the longer row (ties: larger id)
    ap = ex["apair_ptr"].astype(np.int64)
    pos = ex["apair_pos"].astype(np.int64)
    other = ex["apair_other"].astype(np.int64)
    owner = np.repeat(np.arange(n), np.diff(ap))
    assert np.array_equal(np.sort(eid[pos]), np.arange(m))
    assert np.array_equal(row[pos], owner) and np.array_equal(col[pos], other)
    du, dv = deg[owner], deg[other]
    assert np.all((du > dv) | ((du == dv) & (owner > other)))


@pytest.mark.parametrize("knobs", [{"warp_sort_max": 128}, {"warp_sort_max": 512}, {"sort_smem_max": 256}])
def test_undirected_layout_under_other_row_sorts(ubt, knobs):
    """Undirected rows of every length up to ~620 (a planted 600-clique)
    sorted by warps, by blocks of each class and in global memory give the
    same layout, and Alg. 2 still counts as the oracle does."""
    s, d = core_graph(3000, 20000, 600, 25)
    k = synth.k_uniform(s.size, 26)
    with with_knobs(ubt, knobs):
        test_undirected_layout(ubt, ("core600", 3000, s, d, k))
        G = ubt.Graph(3000, s, d, k=k, undirected=True)
        ob, ou = oracle.count_threshold(3000, s, d, k, [0.6, 0.9])
        gb, gu = G.count_aeo([0.6, 0.9])
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_aeo_counts_bit_exact(ubt, case):
    name, n, s, d, k = case
    G = ubt.Graph(n, s, d, k=k, undirected=True)
    for taus in (TAUS, SWEEP32, [0.7]):
        ob, ou = oracle.count_threshold(n, s, d, k, taus)
        for vis in (0, 1):
            with with_knobs(ubt, {"count_visitor": vis}):
                gb, gu = G.count_aeo(taus)
            assert np.array_equal(gb, ob) and np.array_equal(gu, ou), (name, len(taus), vis)
    # the degree-ordered traversal of the same graph agrees
    gb, gu = G.count_threshold(TAUS)
    ob, ou = oracle.count_threshold(n, s, d, k, TAUS)
    assert np.array_equal(gb, ob) and np.array_equal(gu, ou)
    assert G.guard() == 0


@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_aeo_enumeration_bit_exact(ubt, case):
    name, n, s, d, k = case
    G = ubt.Graph(n, s, d, k=k, undirected=True)
    for tau, which in [(0.5, 3), (0.75, 3), (0.9, 1), (0.9, 2)]:
        ouvw, ocls, opb = oracle.enumerate_records(n, s, d, k, tau, which)
        uvw, cls, pb = sort_records(G.enumerate_aeo(tau, which))
        assert np.array_equal(uvw, ouvw) and np.array_equal(cls, ocls) and np.array_equal(pb, opb), (name, tau)
    assert G.guard() == 0


def test_aeo_chunked_tables(ubt):
    """Rows longer than one table are processed chunk by chunk."""
    s, d = mixed_graph(3000, 30000, 21)
    k = synth.k_uniform(s.size, 22)
    with with_knobs(ubt, {"smem_table_max": 64}):
        G = ubt.Graph(3000, s, d, k=k, undirected=True)
        ob, ou = oracle.count_threshold(3000, s, d, k, TAUS)
        gb, gu = G.count_aeo(TAUS)
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou)
        eb, eu, vb, vu = oracle.local_counts(3000, s, d, k, TAUS)
        edges = np.arange(s.size, dtype=np.uint32)
        gb, gu, _ = G.edge_local_counts(edges, TAUS)
        assert np.array_equal(gb, eb) and np.array_equal(gu, eu)
        verts = np.arange(3000, dtype=np.uint32)
        gb, gu, _ = G.vertex_local_counts(verts, TAUS)
        assert np.array_equal(gb, vb) and np.array_equal(gu, vu)
    assert G.guard() == 0


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_edge_and_vertex_local_counts(ubt, case):
    name, n, s, d, k = case
    m = s.size
    G = ubt.Graph(n, s, d, k=k, undirected=True)
    taus = [0.5, 0.6, 0.8, 0.95]
    eb, eu, vb, vu = oracle.local_counts(n, s, d, k, taus)
    ob, ou = oracle.count_threshold(n, s, d, k, taus)
    # uniform samples with repeats
    rng = synth.rng(7)
    es = rng.integers(0, m, size=700).astype(np.uint32)
    gb, gu, est = G.edge_local_counts(es, taus)
    assert np.array_equal(gb, eb[es]) and np.array_equal(gu, eu[es]), name
    assert np.allclose(est[0], m / 3.0 * eb[es].mean(0), rtol=1e-12)
    vs = rng.integers(0, n, size=700).astype(np.uint32)
    gb, gu, est = G.vertex_local_counts(vs, taus)
    assert np.array_equal(gb, vb[vs]) and np.array_equal(gu, vu[vs]), name
    assert np.allclose(est[1], n / 3.0 * vu[vs].mean(0), rtol=1e-12)
    # every edge (vertex) once: the estimator is the exact count
    _, _, est = G.edge_local_counts(np.arange(m, dtype=np.uint32), taus)
    assert np.allclose(est[0], ob, rtol=1e-12) and np.allclose(est[1], ou, rtol=1e-12)
    _, _, est = G.vertex_local_counts(np.arange(n, dtype=np.uint32), taus)
    assert np.allclose(est[0], ob, rtol=1e-12) and np.allclose(est[1], ou, rtol=1e-12)
    assert G.guard() == 0


def test_sampling_degenerate_and_invalid(ubt):
    s, d = synth.er_graph(200, 2000, 9)
    k = synth.k_uniform(s.size, 10)
    G = ubt.Graph(200, s, d, k=k, undirected=True)
    gb, gu, est = G.edge_local_counts(np.zeros(0, dtype=np.uint32), [0.6])
    assert gb.shape == (0, 1) and np.all(est == 0)
    gb, gu, _ = G.edge_local_counts(np.array([5, s.size, 7], dtype=np.uint32), [0.6])
    assert G.guard() != 0          # the out-of-range index is reported ...
    assert gb[1, 0] == 0 and gu[1, 0] == 0   # ... and counts nothing
    eb, eu, _, _ = oracle.local_counts(200, s, d, k, [0.6])
    assert gb[0, 0] == eb[5, 0] and gb[2, 0] == eb[7, 0]
    # a graph built without the undirected rows cannot answer
    H = ubt.Graph(200, s, d, k=k)
    with pytest.raises(ubt.UbtError) as e:
        H.count_aeo([0.6])
    assert e.value.status == -11
    with pytest.raises(ubt.UbtError):
        H.edge_local_counts(np.array([1], dtype=np.uint32), [0.6])
    # REAL graphs have no undirected option
    with pytest.raises(ubt.UbtError):
        ubt.Graph(200, s, d, p=synth.p_uniform_f32(s.size, 3), undirected=True)
    # empty graph
    E = ubt.Graph(10, np.zeros(0, np.uint32), np.zeros(0, np.uint32), k=np.zeros(0, np.uint32), undirected=True)
    b, u = E.count_aeo([0.6, 0.9])
    assert np.all(b == 0) and np.all(u == 0)
    gb, gu, _ = E.vertex_local_counts(np.arange(10, dtype=np.uint32), [0.6])
    assert np.all(gb == 0) and np.all(gu == 0)


def test_undirected_rows_sorted_in_global_memory(ubt):
    """Rows longer than the shared-memory sort limit are sorted in place in
    global memory; the layout and the counts stay the same."""
    s, d = mixed_graph(3000, 30000, 5)
    k = synth.k_uniform(s.size, 6)
    with with_knobs(ubt, {"sort_smem_max": 64}):
        test_undirected_layout(ubt, ("mixed-sort64", 3000, s, d, k))
        G = ubt.Graph(3000, s, d, k=k, undirected=True)
        ob, ou = oracle.count_threshold(3000, s, d, k, TAUS)
        gb, gu = G.count_aeo(TAUS)
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_vertex_local_counts_with_edge_index(ubt, case, mode):
    """Vertex local counts on a graph with the edge index: neighbour pairs
    looked up in it (mode 1 where cheaper, mode 2 always, mode 0 never) give
    the oracle's counts bit for bit; so do edge local counts and the AEO
    count on the same graph."""
    name, n, s, d, k = case
    taus = [0.5, 0.6, 0.8, 0.95]
    eb, eu, vb, vu = oracle.local_counts(n, s, d, k, taus)
    with with_knobs(ubt, {"edge_index": mode}):
        G = ubt.Graph(n, s, d, k=k, undirected=True, edge_index=True)
        vs = synth.rng(17).integers(0, n, size=500).astype(np.uint32)
        gb, gu, _ = G.vertex_local_counts(vs, taus)
        assert np.array_equal(gb, vb[vs]) and np.array_equal(gu, vu[vs]), (name, mode)
        gb, gu, _ = G.vertex_local_counts(np.arange(n, dtype=np.uint32), taus)
        assert np.array_equal(gb, vb) and np.array_equal(gu, vu), (name, mode)
        es = synth.rng(18).integers(0, s.size, size=300).astype(np.uint32)
        gb, gu, _ = G.edge_local_counts(es, taus)
        assert np.array_equal(gb, eb[es]) and np.array_equal(gu, eu[es]), (name, mode)
        ob, ou = oracle.count_threshold(n, s, d, k, taus)
        gb, gu = G.count_aeo(taus)
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou)
        assert G.guard() == 0


def test_edge_index_chunked_tables_and_options(ubt):
    s, d = mixed_graph(3000, 30000, 21)
    k = synth.k_uniform(s.size, 22)
    taus = [0.5, 0.7, 0.9]
    _, _, vb, vu = oracle.local_counts(3000, s, d, k, taus)
    for mode in (1, 2):
        with with_knobs(ubt, {"smem_table_max": 64, "edge_index": mode}):
            G = ubt.Graph(3000, s, d, k=k, undirected=True, edge_index=True)
            gb, gu, _ = G.vertex_local_counts(np.arange(3000, dtype=np.uint32), taus)
            assert np.array_equal(gb, vb) and np.array_equal(gu, vu), mode
            assert G.guard() == 0
    # the index needs the undirected rows
    with pytest.raises(ubt.UbtError):
        ubt.Graph(3000, s, d, k=k, edge_index=True)
    # empty graph
    z = np.zeros(0, np.uint32)
    E = ubt.Graph(10, z, z, k=z, undirected=True, edge_index=True)
    gb, gu, _ = E.vertex_local_counts(np.arange(10, dtype=np.uint32), [0.6])
    assert np.all(gb == 0) and np.all(gu == 0)


@pytest.mark.parametrize("split", [1, 8, 200])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_vertex_samples_split_across_blocks(ubt, case, split):
    """Vertex samples with long rows are queued (64 per call) and their
    neighbours spread over all blocks by a second launch; the rest of the
    long ones are counted in place.  Repeats of one long vertex each get its
    full counts."""
    name, n, s, d, k = case
    taus = [0.5, 0.65, 0.8, 0.95]
    _, _, vb, vu = oracle.local_counts(n, s, d, k, taus)
    deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=n)
    hubs = np.argsort(-deg)[:5]
    vs = np.concatenate([np.repeat(hubs, 3), synth.rng(23).integers(0, n, size=400)]).astype(np.uint32)
    with with_knobs(ubt, {"vertex_split": split, "edge_index": 1}):
        G = ubt.Graph(n, s, d, k=k, undirected=True, edge_index=True)
        gb, gu, est = G.vertex_local_counts(vs, taus)
        assert np.array_equal(gb, vb[vs]) and np.array_equal(gu, vu[vs]), (name, split)
        assert np.allclose(est[0], n / 3.0 * vb[vs].mean(0), rtol=1e-12)
        gb, gu, _ = G.vertex_local_counts(np.arange(n, dtype=np.uint32), taus)
        assert np.array_equal(gb, vb) and np.array_equal(gu, vu), (name, split)
        assert G.guard() == 0


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_aeo_edge_index_form(ubt, case):
    """The Alg. 2 iteration on a graph with the edge index (each edge streams
    the shorter of its two Lemma 3 windows and looks the closing edge up):
    counts for 1 / 6 / 32 thresholds with both counting visitors and records
    bit-exact against the oracle, and equal to the table form's."""
    name, n, s, d, k = case
    G = ubt.Graph(n, s, d, k=k, undirected=True, edge_index=True)
    for taus in (TAUS, SWEEP32, [0.7], [0.5]):
        ob, ou = oracle.count_threshold(n, s, d, k, taus)
        for vis in (0, 1):
            with with_knobs(ubt, {"count_visitor": vis}):
                gb, gu = G.count_aeo(taus)
            assert np.array_equal(gb, ob) and np.array_equal(gu, ou), (name, len(taus), vis)
        with with_knobs(ubt, {"edge_index": 0}):  # the table form on the same graph
            gb, gu = G.count_aeo(taus)
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou), (name, len(taus), "tables")
    for tau, which in [(0.5, 3), (0.75, 3), (0.9, 1), (0.9, 2)]:
        ouvw, ocls, opb = oracle.enumerate_records(n, s, d, k, tau, which)
        uvw, cls, pb = sort_records(G.enumerate_aeo(tau, which))
        assert np.array_equal(uvw, ouvw) and np.array_equal(cls, ocls) and np.array_equal(pb, opb), (name, tau)
    assert G.guard() == 0
