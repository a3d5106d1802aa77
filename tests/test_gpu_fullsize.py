"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (the package's shipped tunings applied the same way).

Where the oracle finishes in seconds it runs on the whole graph (Chung-Lu
n=1e6: counts, exact expected-count sums, enumeration; Chung-Lu n=4e6:
expected counts and the whole gradient).  Where it needs minutes (R-MAT
scale 22 and 20, tens of millions of edges), its values were written once by
tests/golden/make_fullsize_golden.py (which calls only the oracle) and are
compared exactly: R-MAT 22's triangle count and 32-threshold counts, R-MAT
20's balanced counts in every world of four seeded world words and their sum
over all 4,096 worlds.  Each stored file carries a digest of its input, which
the test checks first.  On top: every enumeration record is a triangle of
the input with the class and P_bal of the paper's four-term sum, and for
sampled vertices the records through that vertex equal the oracle's
enumeration of its ego net; properties that hold at any size (pruned ==
unpruned, both pair directions agree, monotonicity in t, the t = 0.5
partition, words-per-pass invariance of the sign worlds, the Monte-Carlo
mean against the exact expectation).  Counts and records are compared
exactly; floating-point values within the tolerances of the other parity
tests.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import difference_quotients, grad_report, require_gpu, sort_records

pytestmark = pytest.mark.gpu

TAUS = [0.55, 0.70, 0.85, 0.95]
SWEEP32 = [0.51 + i * (0.48 / 31) for i in range(32)]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def stored(name, g):
    """The oracle's stored values for graph g, after checking they were made
    from the same input arrays."""
    with open(os.path.join(GOLDEN, name)) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for a in (g.src, g.dst, g.k):
        h.update(np.ascontiguousarray(a, dtype=np.uint32).tobytes())
    assert rec["input_digest"] == h.hexdigest()[:24], "the generator produced another graph than the stored one"
    assert rec["n"] == g.n and rec["m"] == g.m
    return rec


@pytest.fixture(scope="module")
def ubt():
    return require_gpu()


def bench_graph(ubt, g, query, variant, **kw):
    """The graph built under the knobs the benchmark uses for this query."""
    from paper_2602_14084_gb300 import autotune as at
    saved = at.current()
    G = ubt.Graph(g.n, g.src, g.dst, **kw)
    rec = at.lookup(query, G.info(), variant)
    if rec:
        at.apply(rec["config"])
        G.close()
        G = ubt.Graph(g.n, g.src, g.dst, **kw)
    return G, saved


def edge_k_lookup(n, src, dst, k):
    """Sorted undirected edge keys and their k, for looking records up."""
    a, b = np.minimum(src, dst).astype(np.int64), np.maximum(src, dst).astype(np.int64)
    key = a * n + b
    order = np.argsort(key)
    return key[order], k[order].astype(np.int64)


def k_of(n, keys, ks, a, b):
    lo, hi = np.minimum(a, b).astype(np.int64), np.maximum(a, b).astype(np.int64)
    q = lo * n + hi
    i = np.searchsorted(keys, q)
    i = np.minimum(i, keys.size - 1)
    assert np.all(keys[i] == q), "record edge not in the input"
    return ks[i]


def test_cl1m_full_counts_expected_and_enumeration(ubt):
    """Chung-Lu n=1e6 (9.1M edges): the whole graph against the oracle."""
    from paper_2602_14084_gb300 import autotune as at
    g = synth.config_graph("cl1m")
    G, saved = bench_graph(ubt, g, "count", at.count_variant(len(TAUS), True), k=g.k)
    try:
        ob, ou = oracle.count_threshold(g.n, g.src, g.dst, g.k, TAUS)
        for prune in (1, 0):
            gb, gu = G.count_threshold(TAUS, prune=prune)
            assert np.array_equal(gb, ob) and np.array_equal(gu, ou), prune
        oT, oS = oracle.expected_fixed(g.n, g.src, g.dst, g.k)
        _, _, T, sumP = G.expected_counts(with_exact=True)
        assert T == oT and oS == T * (1 << 47) - 4 * sumP
        ouvw, ocls, opb = oracle.enumerate_records(g.n, g.src, g.dst, g.k, 0.95, 3)
        uvw, cls, pb = sort_records(G.enumerate(0.95, 3, prune=1))
        assert np.array_equal(uvw, ouvw) and np.array_equal(cls, ocls) and np.array_equal(pb, opb)
        assert G.guard() == 0
    finally:
        G.close()
        at.apply(saved)


def test_rmat22_full_sweep_and_enumeration(ubt):
    """R-MAT scale 22 (64.2M edges): the 32-threshold sweep against the
    oracle's stored counts, and the t = 0.9 enumeration by the four-term sum
    per record and sampled oracle enumerations."""
    from paper_2602_14084_gb300 import autotune as at
    g = synth.config_graph("rmat22")
    want = stored("rmat22_sweep32.json", g)
    assert want["taus"] == SWEEP32
    G, saved = bench_graph(ubt, g, "count", at.count_variant(32, True), k=g.k)
    try:
        b, u = G.count_threshold(SWEEP32, prune=1)
        assert np.array_equal(b, want["balanced"]) and np.array_equal(u, want["unbalanced"])
        b0, u0 = G.count_threshold(SWEEP32, prune=0)
        assert np.array_equal(b, b0) and np.array_equal(u, u0)
        assert np.all(np.diff(b) <= 0) and np.all(np.diff(u) <= 0)
        _, _, T, _ = G.expected_counts(with_exact=True)
        assert T == want["triangles"]
        hb, hu = G.count_threshold([0.5], prune=1)
        assert int(hb[0]) + int(hu[0]) == T  # at t = 0.5 every triangle is classified once
        assert b[0] + u[0] <= T
        nb9, nu9 = G.count_threshold([0.9], prune=1)
        rec = G.enumerate(0.9, 3, prune=1)
        assert rec.shape[0] == int(nb9[0]) + int(nu9[0])
        assert G.guard() == 0
        # the other pair direction (Alg. 1 as written) gives the same sweep
        pull = ubt.get_tuning("pull")
        ubt.set_tuning("pull", 1 - pull)
        G2 = ubt.Graph(g.n, g.src, g.dst, k=g.k)
        ubt.set_tuning("pull", pull)
        b2, u2 = G2.count_threshold(SWEEP32, prune=1)
        assert np.array_equal(b, b2) and np.array_equal(u, u2)
        assert G2.guard() == 0
        G2.close()
        G.close()
    finally:
        at.apply(saved)
    # every record: a triangle of the input, classified and valued by the
    # paper's four-term sum (Sec. 3) in exact integers, as the oracle does:
    # N = 2^48 P_bal = k1 k2 k3 + k1 k2' k3' + k1' k2 k3' + k1' k2' k3, k' = 2^16 - k
    keys, ks = edge_k_lookup(g.n, g.src, g.dst, g.k)
    uvw, cls, pb = sort_records(rec)
    assert np.all((uvw[:, 0] < uvw[:, 1]) & (uvw[:, 1] < uvw[:, 2]))
    assert np.unique(uvw, axis=0).shape[0] == uvw.shape[0]
    k1, k2, k3 = [k_of(g.n, keys, ks, uvw[:, i], uvw[:, j]) for i, j in ((0, 1), (0, 2), (1, 2))]
    c1, c2, c3 = 65536 - k1, 65536 - k2, 65536 - k3
    N = k1 * k2 * k3 + k1 * c2 * c3 + c1 * k2 * c3 + c1 * c2 * k3
    assert np.array_equal(pb, N.astype(np.float64) * 2.0 ** -48)
    tb, tu = int(np.ceil(0.9 * 2.0 ** 48)), int(np.floor(0.9 * 2.0 ** 48))
    want_cls = np.where(N >= tb, 1, np.where((1 << 48) - N > tu, 2, 0))
    assert np.array_equal(cls, want_cls)
    # completeness on sampled vertices: all records through v = the oracle's
    # enumeration of v's ego net (v and all its neighbours) restricted to v
    off, nbr, _ = synth.csr_undirected(g.n, g.src, g.dst)
    deg = np.diff(off)
    cand = np.nonzero((deg >= 20) & (deg <= 3000))[0]
    picks = synth.rng(5).choice(cand, size=24, replace=False)
    sets = [np.unique(np.concatenate([[v], nbr[off[v]:off[v + 1]]])).astype(np.uint32) for v in picks]
    v_off = np.zeros(len(sets) + 1, dtype=np.int64)
    v_off[1:] = np.cumsum([x.size for x in sets])
    sub = synth.ego_induce(g.n, g.src, g.dst, {"v_off": v_off, "vid": np.concatenate(sets)})
    for i, v in enumerate(picks):
        v0, v1 = int(sub["v_off"][i]), int(sub["v_off"][i + 1])
        e0, e1 = int(sub["e_off"][i]), int(sub["e_off"][i + 1])
        ouvw, ocls, opb = oracle.enumerate_records(v1 - v0, sub["src"][e0:e1] - v0, sub["dst"][e0:e1] - v0,
                                                   g.k[sub["eid"][e0:e1]], 0.9, 3)
        vid = sub["vid"][v0:v1]
        gl = vid[ouvw.astype(np.int64)] if ouvw.size else np.zeros((0, 3), np.uint32)
        mine = np.any(gl == v, axis=1)
        want = gl[mine]
        order = np.lexsort((want[:, 2], want[:, 1], want[:, 0])) if want.size else np.zeros(0, np.int64)
        want, wcls, wpb = want[order], ocls[mine][order], opb[mine][order]
        got = np.any(uvw == v, axis=1)
        assert np.array_equal(uvw[got], want), v
        assert np.array_equal(cls[got], wcls) and np.array_equal(pb[got], wpb), v


def test_rmat20_worlds_full(ubt):
    """R-MAT scale 20 (15.7M edges), W = 4096 sign worlds: the oracle's counts
    of four seeded world words and its sum over all worlds; words per pass do
    not change a count, totals agree, and the Monte-Carlo mean of the
    balanced count lies within 5 standard errors of its exact expectation."""
    import torch
    from paper_2602_14084_gb300 import autotune as at
    g = synth.config_graph("rmat20")
    want = stored("rmat20_worlds.json", g)
    G, saved = bench_graph(ubt, g, "worlds", "W4096", k=g.k)
    try:
        W = 4096
        assert want["W"] == W and want["world_seed"] == 7
        eb, _, T, _ = G.expected_counts(with_exact=True)
        out = torch.empty(W, dtype=torch.int64, device="cuda")
        tot = torch.empty(1, dtype=torch.int64, device="cuda")
        G.sample_worlds_(7, W, out, tot)
        a = out.cpu().numpy()
        # the oracle's per-world counts of the stored words, and their sum over all worlds
        for w, counts in want["per_world"].items():
            w = int(w)
            assert np.array_equal(a[64 * w:64 * (w + 1)], counts), w
        assert int(a.sum()) == want["balanced_sum_over_all_worlds"]
        wpp = ubt.get_tuning("world_words_per_pass")
        ubt.set_tuning("world_words_per_pass", 8 if wpp != 8 else 64)
        G.sample_worlds_(7, W, out, tot)
        ubt.set_tuning("world_words_per_pass", wpp)
        assert np.array_equal(out.cpu().numpy(), a)
        assert int(tot.item()) == int(a.sum())
        assert np.all((a >= 0) & (a <= T))
        z = (a.mean() - eb) / (a.std(ddof=1) / np.sqrt(W))
        assert abs(z) < 5.0, z
        assert G.guard() == 0
    finally:
        G.close()
        at.apply(saved)


def test_ego10k_full_batch_sampled_graphs(ubt):
    """The 10,000-ego-net batch of R-MAT scale 20: sampled graphs' counts,
    expected counts and world word 0 (parent edge keys) against the oracle."""
    import torch
    g = synth.config_graph("rmat20")
    sel = synth.ego_select(g.n, g.src, g.dst, 10000, 50, 5000, 1)
    eg = synth.ego_induce_torch(g.n, g.src, g.dst, sel, device="cuda")
    kb = torch.from_numpy(g.k.view(np.int32)).cuda()[eg["eid"].long()]
    G = ubt.Graph(int(eg["v_off"][-1].item()), eg["src"], eg["dst"], k=kb, edge_key=eg["eid"],
                  vertex_offsets=eg["v_off"])
    taus = [0.6, 0.75, 0.9]
    counts, expect, worlds = G.batch_query(taus, seed=11)
    assert G.guard() == 0
    v_off = eg["v_off"].cpu().numpy()
    e_off = eg["e_off"].cpu().numpy()
    picks = sorted(set(synth.rng(9).choice(10000, size=20, replace=False).tolist()) | {0, 9999})
    src = eg["src"].cpu().numpy().view(np.uint32)
    dst = eg["dst"].cpu().numpy().view(np.uint32)
    eid = eg["eid"].cpu().numpy().view(np.uint32)
    for gi in picks:
        v0, v1 = int(v_off[gi]), int(v_off[gi + 1])
        e0, e1 = int(e_off[gi]), int(e_off[gi + 1])
        ls, ld, lk = src[e0:e1] - v0, dst[e0:e1] - v0, g.k[eid[e0:e1]]
        ob, ou = oracle.count_threshold(v1 - v0, ls, ld, lk, taus)
        assert np.array_equal(counts[gi, 0], ob) and np.array_equal(counts[gi, 1], ou), gi
        oT, oS = oracle.expected_fixed(v1 - v0, ls, ld, lk)
        assert abs(expect[gi, 0] - oS / float(1 << 48)) <= 1e-12 * max(1.0, oT), gi
        ow = oracle.world_counts(v1 - v0, ls, ld, lk, 11, [0], ekey=eid[e0:e1])
        assert np.array_equal(worlds[gi], ow), gi


def test_cl4m_full_expected_counts_and_gradient(ubt):
    """Chung-Lu n=4e6 (39.6M edges), p ~ U[0,1] float32: expected counts and
    the whole gradient through autograd against the oracle."""
    import torch
    g = synth.config_graph("cl4m")
    pt = torch.from_numpy(g.p).cuda().requires_grad_(True)
    G = ubt.Graph(g.n, g.src, g.dst, p=pt.detach())
    eb, eu = ubt.expected_counts(G, pt)
    ob, ou, T = oracle.expected_real(g.n, g.src, g.dst, g.p)
    assert abs(eb.item() - ob) <= 1e-9 * max(1.0, abs(ob))
    assert abs(eu.item() - ou) <= 1e-9 * max(1.0, abs(ou))
    (eb - eu).backward()
    got = pt.grad.double().cpu().numpy()
    og, ga = oracle.grad_real(g.n, g.src, g.dst, g.p, with_abs=True)
    want = 2.0 * og  # d(E_bal - E_unbal)/dp = 2 dE_bal/dp
    tol = 1e-5 * np.maximum(np.abs(want), 1e-3 * 2.0 * ga)
    bad = np.abs(got - want) > tol + 1e-12
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - want) / (tol + 1e-30))))
    assert G.guard() == 0


def test_cl1m_full_aeo_sampling_and_topk(ubt):
    """Chung-Lu n=1e6 with the undirected rows and the edge index, as the
    benchmark builds it for the Alg. 2 iteration, the samplers and top-k:
    AEO counts on the whole graph; local counts of 5,000 sampled edges and of
    5,000 sampled vertices plus the 16 largest hubs (repeated, so the split
    launch's queue overflows and both of its paths run), with the index in
    every mode; the top 1,000 most balanced / unbalanced triangles against
    the oracle's enumeration above t = 0.999."""
    g = synth.config_graph("cl1m")
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k, undirected=True, edge_index=True)
    try:
        ob, ou = oracle.count_threshold(g.n, g.src, g.dst, g.k, TAUS)
        gb, gu = G.count_aeo(TAUS)
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou)
        eb, eu, vb, vu = oracle.local_counts(g.n, g.src, g.dst, g.k, TAUS)
        es = synth.rng(31).integers(0, g.m, size=5000).astype(np.uint32)
        gb, gu, _ = G.edge_local_counts(es, TAUS)
        assert np.array_equal(gb, eb[es]) and np.array_equal(gu, eu[es])
        deg = np.bincount(np.concatenate([g.src, g.dst]).astype(np.int64), minlength=g.n)
        hubs = np.argsort(-deg)[:16]
        vs = np.concatenate([synth.rng(32).integers(0, g.n, size=5000), np.repeat(hubs, 5)]).astype(np.uint32)
        old = ubt.get_tuning("edge_index")
        try:
            for mode in (1, 0, 2):
                ubt.set_tuning("edge_index", mode)
                gb, gu, est = G.vertex_local_counts(vs, TAUS)
                assert np.array_equal(gb, vb[vs]) and np.array_equal(gu, vu[vs]), mode
                assert np.allclose(est[0], g.n / 3.0 * vb[vs].mean(0), rtol=1e-12)
        finally:
            ubt.set_tuning("edge_index", old)
        for which in (1, 2):
            ouvw, _, opb = oracle.enumerate_records(g.n, g.src, g.dst, g.k, 0.999, which)
            key = -opb if which == 1 else opb
            order = np.lexsort((ouvw[:, 2], ouvw[:, 1], ouvw[:, 0], key))
            assert order.size > 1000
            rec = G.topk(1000, which)
            assert np.array_equal(rec["p_bal"], opb[order][:1000]), which
            got = np.stack([rec["u"], rec["v"], rec["w"]], axis=1).astype(np.uint32)
            assert np.array_equal(got, ouvw[order][:1000]), which
        assert G.guard() == 0
    finally:
        G.close()


def test_cl4m_subgraph_gradient_against_difference_quotients(ubt):
    """Chung-Lu n=4e6, p ~ U[0,1] float32: on the subgraph induced by a BFS
    from a seeded vertex, grown until it holds >= 1,000 edges, the adjoint's
    gradient of every edge against float64 difference quotients of the GPU
    forward and against the oracle's analytic gradient.  E is affine in each
    p_e, so the central difference at p_e = 1/2 with h = 1/2, E(p_e = 1) -
    E(p_e = 0), is exact up to the forward's rounding (endpoints stored
    exactly).  Tolerance per edge: 1e-5 max(|g|, 1e-3 sum |terms|); the plain
    relative error and the number of edges where the floor applied are
    printed."""
    import torch
    g = synth.config_graph("cl4m")
    deg = np.bincount(np.concatenate([g.src, g.dst]).astype(np.int64), minlength=g.n)
    start = int(synth.rng(61).choice(np.nonzero(deg >= 10)[0]))
    verts, ls, ld, eid = synth.bfs_induced(g.n, g.src, g.dst, start, 1000)
    assert ls.size >= 1000
    p = np.ascontiguousarray(g.p[eid])
    pt = torch.from_numpy(p.copy()).cuda().requires_grad_(True)
    G = ubt.Graph(verts.size, ls, ld, p=pt.detach())
    eb, _ = ubt.expected_counts(G, pt)
    eb.backward()
    got = pt.grad.double().cpu().numpy()
    fd = difference_quotients(ubt, G, p, np.arange(ls.size))
    og, ga = oracle.grad_real(verts.size, ls, ld, p, with_abs=True)
    for name, ref in (("difference quotients", fd), ("oracle analytic", og)):
        ok, rel, floored = grad_report(got, ref, ga)
        nz = np.abs(ref) > 0
        print("C5 subgraph (%d vertices, %d edges) vs %s: max plain relative error %.3e over %d edges with "
              "a nonzero gradient, floor used on %d edges, %d outside tolerance"
              % (verts.size, ls.size, name, float(rel[nz].max()) if nz.any() else 0.0, int(nz.sum()), floored,
                 int((~ok).sum())))
        assert ok.all(), name
    # the two references agree with each other as well
    assert np.allclose(fd, og, rtol=1e-6, atol=1e-8)
    assert G.guard() == 0
