"""GPU path vs the CPU oracle, element by element, on seeded inputs.

Counts, enumeration records and per-world counts are bit-exact; expected
counts of FIXED graphs are compared through their exact integer sums; REAL
(float32) expected counts within 1e-9 relative and gradients within 1e-5
relative per edge (floored at 1e-3 of the edge's sum of |terms|, where
cancellation makes a relative bound meaningless).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import mixed_graph, require_gpu, sort_records

pytestmark = pytest.mark.gpu

TAUS = [0.5, 0.6, 0.75, 0.9, 0.99, 1.0]


@pytest.fixture(scope="module")
def ubt():
    return require_gpu()


@pytest.fixture(scope="module")
def er2k():
    return synth.config_graph("er2k")


def graphs_for_parity():
    out = []
    g = synth.config_graph("er2k")
    out.append(("er2k", g.n, g.src, g.dst, g.k))
    for seed, (n, m) in enumerate([(300, 6000), (1500, 40000), (64, 2016)]):
        s, d = synth.er_graph(n, m, 100 + seed)
        out.append(("er%d_%d" % (n, m), n, s, d, synth.k_uniform(m, 200 + seed)))
    s, d = mixed_graph(3000, 30000, 5)
    out.append(("mixed3000", 3000, s, d, synth.k_uniform(s.size, 6)))
    s, d = synth.rmat(12, 16, 0.57, 0.19, 0.19, 3)
    out.append(("rmat12", 1 << 12, s, d, synth.quantise(synth.p_beta(s.size, 0.5, 0.5, 4))))
    return out


PARITY = graphs_for_parity()


@pytest.mark.parametrize("case", PARITY, ids=[c[0] for c in PARITY])
@pytest.mark.parametrize("prune", [0, 1])
def test_counts_bit_exact(ubt, case, prune):
    name, n, s, d, k = case
    G = ubt.Graph(n, s, d, k=k)
    ob, ou = oracle.count_threshold(n, s, d, k, TAUS)
    gb, gu = G.count_threshold(TAUS, prune=prune)
    assert G.guard() == 0
    assert np.array_equal(gb, ob) and np.array_equal(gu, ou), (name, gb, ob, gu, ou)
    for i, t in enumerate(TAUS):  # single-threshold launches
        b1, u1 = G.count_threshold([t], prune=prune)
        assert (int(b1[0]), int(u1[0])) == (int(ob[i]), int(ou[i])), (name, t)
    assert G.guard() == 0


SWEEP32 = [0.51 + i * (0.48 / 31) for i in range(32)]
MANY = {
    "sweep32": SWEEP32,
    "nine": [0.9, 0.5, 0.55, 0.6, 0.65, 0.7, 0.8, 0.95, 1.0],
    # 64 thresholds, unsorted, with repeats and both ends of [0.5, 1]
    "sixty_four": [float(x) for x in np.random.default_rng(7).permutation(
        np.concatenate([np.linspace(0.5, 1.0, 48), [0.5, 1.0, 0.75, 0.75], np.linspace(0.52, 0.98, 12)]))],
}


@pytest.mark.parametrize("case", PARITY, ids=[c[0] for c in PARITY])
@pytest.mark.parametrize("which", sorted(MANY))
def test_counts_many_thresholds_bit_exact(ubt, case, which):
    """More than 8 thresholds: one traversal bins every product among all levels."""
    name, n, s, d, k = case
    taus = MANY[which]
    G = ubt.Graph(n, s, d, k=k)
    ob, ou = oracle.count_threshold(n, s, d, k, taus)
    old = ubt.get_tuning("count_visitor")
    try:
        for vis in (0, 1):
            ubt.set_tuning("count_visitor", vis)
            for prune in (0, 1):
                gb, gu = G.count_threshold(taus, prune=prune)
                assert np.array_equal(gb, ob) and np.array_equal(gu, ou), (name, which, vis, prune)
    finally:
        ubt.set_tuning("count_visitor", old)
    assert G.guard() == 0


DISTS = {"uniform": lambda m, sd: synth.rng(sd).random(m),
         "normal": lambda m, sd: synth.p_normal(m, sd),
         "beta_0.5_0.5": lambda m, sd: synth.p_beta(m, 0.5, 0.5, sd),
         "beta_3_1": lambda m, sd: synth.p_beta(m, 3.0, 1.0, sd),
         "beta_1_3": lambda m, sd: synth.p_beta(m, 1.0, 3.0, sd)}


@pytest.mark.parametrize("dist", sorted(DISTS))
def test_counts_across_p_distributions(ubt, dist):
    """The five P+ distributions of the Sec. 6 distribution study on one
    structure: pruned counts bit-exact for both counting visitors."""
    s, d = mixed_graph(3000, 30000, 41)
    k = synth.quantise(DISTS[dist](s.size, 42))
    G = ubt.Graph(3000, s, d, k=k)
    taus = TAUS + SWEEP32
    ob, ou = oracle.count_threshold(3000, s, d, k, taus)
    old = ubt.get_tuning("count_visitor")
    try:
        for vis in (0, 1):
            ubt.set_tuning("count_visitor", vis)
            gb, gu = G.count_threshold(taus, prune=1)
            assert np.array_equal(gb, ob) and np.array_equal(gu, ou), (dist, vis)
            for i, t in enumerate(TAUS):
                b1, u1 = G.count_threshold([t], prune=1)
                assert (int(b1[0]), int(u1[0])) == (int(ob[i]), int(ou[i])), (dist, vis, t)
    finally:
        ubt.set_tuning("count_visitor", old)
    assert G.guard() == 0


@pytest.mark.parametrize("case", PARITY, ids=[c[0] for c in PARITY])
def test_enumeration_bit_exact(ubt, case):
    name, n, s, d, k = case
    G = ubt.Graph(n, s, d, k=k)
    for tau, which in [(0.5, 3), (0.75, 3), (0.9, 1), (0.9, 2), (0.6, 3)]:
        ouvw, ocls, opb = oracle.enumerate_records(n, s, d, k, tau, which)
        for prune in (0, 1):
            rec = G.enumerate(tau, which, prune=prune)
            uvw, cls, pb = sort_records(rec)
            assert np.array_equal(uvw, ouvw), (name, tau, which, prune)
            assert np.array_equal(cls, ocls)
            assert np.array_equal(pb, opb)
    assert G.guard() == 0


def test_enumeration_capacity(ubt, er2k):
    g = er2k
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    ouvw, _, _ = oracle.enumerate_records(g.n, g.src, g.dst, g.k, 0.6, 3)
    assert ouvw.shape[0] > 10
    with pytest.raises(ubt.UbtError) as e:
        G.enumerate(0.6, 3, capacity=5)
    assert e.value.status == -7 and str(ouvw.shape[0]) in str(e.value)


@pytest.mark.parametrize("case", PARITY, ids=[c[0] for c in PARITY])
def test_expected_counts_fixed_exact(ubt, case):
    name, n, s, d, k = case
    G = ubt.Graph(n, s, d, k=k)
    eb, eu, T, sumP = G.expected_counts(with_exact=True)
    oT, oS = oracle.expected_fixed(n, s, d, k)
    assert T == oT
    # oracle: sum of 2^48 P_bal = sum (2^47 - 4 P) = T 2^47 - 4 sum P
    assert oS == T * (1 << 47) - 4 * sumP
    e_exact = oS / float(1 << 48)
    assert abs(eb - e_exact) <= 1e-12 * max(1.0, e_exact)
    assert abs(eu - (oT - e_exact)) <= 1e-12 * max(1.0, oT - e_exact)


@pytest.mark.parametrize("seed,n,m", [(1, 2000, 20000), (2, 3000, 60000)])
def test_expected_counts_and_gradient_real(ubt, seed, n, m):
    import torch
    s, d = synth.er_graph(n, m, seed)
    if seed == 2:
        s, d = mixed_graph(n, m, seed)
    p = synth.p_uniform_f32(s.size, seed + 50)
    pt = torch.from_numpy(p).cuda().requires_grad_(True)
    G = ubt.Graph(n, s, d, p=pt.detach())
    eb, eu = ubt.expected_counts(G, pt)
    ob, ou, T = oracle.expected_real(n, s, d, p)
    assert abs(eb.item() - ob) <= 1e-9 * max(1.0, abs(ob))
    assert abs(eu.item() - ou) <= 1e-9 * max(1.0, abs(ou))
    (0.7 * eb - 1.3 * eu).backward()
    g = pt.grad.double().cpu().numpy()
    og, ga = oracle.grad_real(n, s, d, p, with_abs=True)
    want = 0.7 * og + 1.3 * og  # dE_unbal/dp = -dE_bal/dp
    tol = 1e-5 * np.maximum(np.abs(want), 1e-3 * 2.0 * ga)
    assert np.all(np.abs(g - want) <= tol + 1e-12), np.max(np.abs(g - want) / (tol + 1e-30))


def test_gradient_fixed_graph_exact(ubt, er2k):
    import torch
    g = er2k
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    gout = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda")
    grad = torch.empty(g.m, dtype=torch.float32, device="cuda")
    G.expected_counts_backward_(gout, grad)
    p = (g.k.astype(np.float64) / 65536.0).astype(np.float32)
    og = oracle.grad_real(g.n, g.src, g.dst, p)
    assert np.allclose(grad.cpu().numpy(), og, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("W", [64, 256, 4096])
def test_worlds_bit_exact(ubt, er2k, W):
    g = er2k
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    for wpp in (1, 4, 64):
        ubt.set_tuning("world_words_per_pass", wpp)
        got, tot = G.sample_worlds(seed=1234, W=W)
        want = oracle.world_counts(g.n, g.src, g.dst, g.k, 1234, list(range(W // 64)))
        assert np.array_equal(got, want), wpp
        assert tot == int(want.sum())
    ubt.set_tuning("world_words_per_pass", 8)


def test_worlds_64_words_per_pass_with_long_lists(ubt):
    """One pass of 64 words (two words per lane, rows staged in shared
    memory) on a graph with block tasks (a planted clique and star)."""
    s, d = mixed_graph(3000, 30000, 5)
    k = synth.k_uniform(s.size, 6)
    G = ubt.Graph(3000, s, d, k=k)
    old = ubt.get_tuning("world_words_per_pass")
    try:
        ubt.set_tuning("world_words_per_pass", 64)
        got, tot = G.sample_worlds(seed=4321, W=4096)
    finally:
        ubt.set_tuning("world_words_per_pass", old)
    want = oracle.world_counts(3000, s, d, k, 4321, list(range(64)))
    assert np.array_equal(got, want)
    assert tot == int(want.sum())
    assert G.guard() == 0


def test_worlds_with_edge_keys(ubt):
    n, m = 500, 6000
    s, d = synth.er_graph(n, m, 77)
    k = synth.k_uniform(m, 78)
    key = (np.arange(m, dtype=np.uint64) * 2654435761 % (1 << 32)).astype(np.uint32)
    G = ubt.Graph(n, s, d, k=k, edge_key=key)
    got, _ = G.sample_worlds(seed=9, W=128)
    want = oracle.world_counts(n, s, d, k, 9, [0, 1], ekey=key)
    assert np.array_equal(got, want)


def test_batch_of_ego_nets(ubt):
    n = 1 << 12
    ps, pd = synth.rmat(12, 16, 0.57, 0.19, 0.19, 11)
    pk = synth.k_uniform(ps.size, 12)
    eg = synth.ego_nets(n, ps, pd, 40, 10, 300, 13)
    taus = [0.6, 0.75, 0.9]
    k = pk[eg["eid"]]
    G = ubt.Graph(int(eg["v_off"][-1]), eg["src"], eg["dst"], k=k, edge_key=eg["eid"],
                  vertex_offsets=eg["v_off"])
    counts, expect, worlds = G.batch_query(taus, seed=5)
    for gi in range(40):
        v0, v1 = int(eg["v_off"][gi]), int(eg["v_off"][gi + 1])
        e0, e1 = int(eg["e_off"][gi]), int(eg["e_off"][gi + 1])
        ls = eg["src"][e0:e1] - v0
        ld = eg["dst"][e0:e1] - v0
        lk = k[e0:e1]
        ob, ou = oracle.count_threshold(v1 - v0, ls, ld, lk, taus)
        assert np.array_equal(counts[gi, 0], ob) and np.array_equal(counts[gi, 1], ou), gi
        T, S = oracle.expected_fixed(v1 - v0, ls, ld, lk)
        e_exact = S / float(1 << 48)
        assert abs(expect[gi, 0] - e_exact) <= 1e-12 * max(1.0, e_exact)
        assert abs(expect[gi, 1] - (T - e_exact)) <= 1e-12 * max(1.0, T)
        ow = oracle.world_counts(v1 - v0, ls, ld, lk, 5, [0], ekey=eg["eid"][e0:e1])
        assert np.array_equal(worlds[gi], ow), gi


def test_batch_from_torch_extraction_and_cuda_graph_capture(ubt):
    """The batch built from the GPU ego-net extraction equals the CPU one, and
    a batch query captured in a CUDA graph and replayed gives the same answers
    as a direct call (and as the oracle on sampled ego nets)."""
    import torch
    n = 1 << 14
    ps, pd = synth.rmat(14, 16, 0.57, 0.19, 0.19, 21)
    pk = synth.k_uniform(ps.size, 22)
    sel = synth.ego_select(n, ps, pd, 120, 20, 1500, 23)
    cpu = synth.ego_induce(n, ps, pd, sel)
    gpu = synth.ego_induce_torch(n, ps, pd, sel, device="cuda", chunk=1 << 18)
    for key in ("v_off", "e_off", "src", "dst", "eid", "vid"):
        assert np.array_equal(gpu[key].cpu().numpy().astype(np.int64), cpu[key].astype(np.int64)), key
    k = torch.from_numpy(pk.view(np.int32)).cuda()[gpu["eid"].long()]
    G = ubt.Graph(int(cpu["v_off"][-1]), gpu["src"], gpu["dst"], k=k, edge_key=gpu["eid"], vertex_offsets=gpu["v_off"])
    taus = [0.6, 0.75, 0.9]
    ng = G.n_graphs
    c = torch.empty(ng * 6, dtype=torch.int64, device="cuda")
    e = torch.empty(ng * 2, dtype=torch.float64, device="cuda")
    w = torch.empty(ng * 64, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        G.batch_query_(taus, 3, c, e, w, stream=side)
    torch.cuda.synchronize()
    ref = (c.clone(), e.clone(), w.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
        G.batch_query_(taus, 3, c, e, w, stream=side)
    for x in (c, e, w):
        x.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(c, ref[0]) and torch.equal(e, ref[1]) and torch.equal(w, ref[2])
    cn, en, wn = c.cpu().numpy().reshape(ng, 2, 3), e.cpu().numpy().reshape(ng, 2), w.cpu().numpy().reshape(ng, 64)
    kk = pk[cpu["eid"]]
    for gi in [0, 1, 17, 60, ng - 1]:
        v0, v1 = int(cpu["v_off"][gi]), int(cpu["v_off"][gi + 1])
        e0, e1 = int(cpu["e_off"][gi]), int(cpu["e_off"][gi + 1])
        ls, ld, lk = cpu["src"][e0:e1] - v0, cpu["dst"][e0:e1] - v0, kk[e0:e1]
        ob, ou = oracle.count_threshold(v1 - v0, ls, ld, lk, taus)
        assert np.array_equal(cn[gi, 0], ob) and np.array_equal(cn[gi, 1], ou), gi
        T, S = oracle.expected_fixed(v1 - v0, ls, ld, lk)
        assert abs(en[gi, 0] - S / float(1 << 48)) <= 1e-12 * max(1.0, T)
        ow = oracle.world_counts(v1 - v0, ls, ld, lk, 3, [0], ekey=cpu["eid"][e0:e1])
        assert np.array_equal(wn[gi], ow), gi
    assert G.guard() == 0


def test_giant_lists_use_global_tables(ubt):
    """Lists longer than the shared-memory table go through the global-table path."""
    old = ubt.get_tuning("smem_table_max")
    try:
        ubt.set_tuning("smem_table_max", 64)
        s, d = mixed_graph(3000, 30000, 21)
        k = synth.k_uniform(s.size, 22)
        G = ubt.Graph(3000, s, d, k=k)
        ob, ou = oracle.count_threshold(3000, s, d, k, TAUS)
        gb, gu = G.count_threshold(TAUS, prune=1)
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou)
        gb, gu = G.count_threshold(TAUS, prune=0)
        assert np.array_equal(gb, ob) and np.array_equal(gu, ou)
        T, S = oracle.expected_fixed(3000, s, d, k)
        _, _, T2, sumP = G.expected_counts(with_exact=True)
        assert T2 == T and S == T * (1 << 47) - 4 * sumP
    finally:
        ubt.set_tuning("smem_table_max", old)


@pytest.mark.parametrize("knobs", [{"hub_threshold": 2}, {"hub_threshold": 200}, {"pull": 0},
                                   {"block_work": 1}, {"block_work": 1 << 30, "hub_threshold": 32},
                                   {"block_unit": 1}, {"block_unit": 32}, {"count_visitor": 1},
                                   {"small_batch": 1, "warp_threads": 64, "block_threads": 64}, {"warp_threads": 512, "block_threads": 128},
                                   {"long_min": 1}, {"long_min": 1 << 20}, {"long_tail": 1},
                                   {"long_tail": 1, "long_min": 1}, {"long_tail": 1, "long_min": 64, "count_visitor": 1},
                                   {"long_tail": 1, "long_min": 130, "pull": 0}])
def test_task_split_variants(ubt, knobs):
    """Every way of partitioning the pairs and splitting the work into block /
    warp tasks gives the same bit-exact counts and expected-count sums."""
    old = {k: ubt.get_tuning(k) for k in knobs}
    try:
        for k, v in knobs.items():
            ubt.set_tuning(k, v)
        s, d = mixed_graph(2000, 25000, 31)
        k = synth.k_uniform(s.size, 32)
        G = ubt.Graph(2000, s, d, k=k)
        ob, ou = oracle.count_threshold(2000, s, d, k, TAUS)
        for prune in (0, 1):
            gb, gu = G.count_threshold(TAUS, prune=prune)
            assert np.array_equal(gb, ob) and np.array_equal(gu, ou), prune
        T, S = oracle.expected_fixed(2000, s, d, k)
        _, _, T2, sumP = G.expected_counts(with_exact=True)
        assert T2 == T and S == T * (1 << 47) - 4 * sumP
        ouvw, ocls, opb = oracle.enumerate_records(2000, s, d, k, 0.75, 3)
        uvw, cls, pb = sort_records(G.enumerate(0.75, 3))
        assert np.array_equal(uvw, ouvw) and np.array_equal(cls, ocls) and np.array_equal(pb, opb)
        assert G.guard() == 0
    finally:
        for k, v in old.items():
            ubt.set_tuning(k, v)


def test_degenerate_graphs(ubt):
    z = np.zeros(0, dtype=np.uint32)
    for n in (0, 1, 5):
        G = ubt.Graph(n, z, z, k=z)
        b, u = G.count_threshold([0.6, 0.9])
        assert b.tolist() == [0, 0] and u.tolist() == [0, 0]
        assert G.expected_counts(with_exact=True)[2] == 0
        assert G.enumerate(0.5).size == 0
    # a single triangle, each boundary case of the paper's text
    s = np.array([0, 0, 1], dtype=np.uint32)
    d = np.array([1, 2, 2], dtype=np.uint32)
    for kk in ([32768, 65536, 65536], [65536, 65536, 49152], [65536, 65536, 16384], [65536, 65536, 0],
               [0, 0, 0], [65536] * 3):
        k = np.array(kk, dtype=np.uint32)
        G = ubt.Graph(3, s, d, k=k)
        ob, ou = oracle.count_threshold(3, s, d, k, TAUS)
        for prune in (0, 1):
            gb, gu = G.count_threshold(TAUS, prune=prune)
            assert np.array_equal(gb, ob) and np.array_equal(gu, ou), kk


def test_invalid_inputs_rejected(ubt):
    s = np.array([0, 1, 2], dtype=np.uint32)
    d = np.array([1, 2, 0], dtype=np.uint32)
    k = np.array([1, 2, 3], dtype=np.uint32)
    cases = [
        (dict(n=3, src=s, dst=np.array([1, 2, 2], np.uint32), k=k), -2),      # self-loop
        (dict(n=3, src=s, dst=np.array([1, 0, 0], np.uint32), k=k), -3),      # duplicate {0,1}
        (dict(n=2, src=s, dst=d, k=k), -4),                                    # vertex 2 >= n
        (dict(n=3, src=s, dst=d, k=np.array([1, 65537, 3], np.uint32)), -5),   # k out of range
    ]
    for kw, code in cases:
        with pytest.raises(ubt.UbtError) as e:
            ubt.Graph(kw["n"], kw["src"], kw["dst"], k=kw["k"])
        assert e.value.status == code
    with pytest.raises(ubt.UbtError) as e:
        ubt.Graph(3, s, d, p=np.array([0.1, 1.5, 0.2], np.float32))
    assert e.value.status == -5
    with pytest.raises(ubt.UbtError) as e:
        ubt.Graph(3, s, d, p=np.array([0.1, np.nan, 0.2], np.float32))
    assert e.value.status == -5
    G = ubt.Graph(3, s, d, k=k)
    for bad in (0.49, 1.01, float("nan")):
        with pytest.raises(ubt.UbtError) as e:
            G.count_threshold([bad])
        assert e.value.status == -6
    Gp = ubt.Graph(3, s, d, p=np.array([0.1, 0.5, 0.2], np.float32))
    with pytest.raises(ubt.UbtError) as e:
        Gp.count_threshold([0.6])
    assert e.value.status == -11


def test_count_host_end_to_end(ubt, er2k):
    g = er2k
    b, u = ubt.count_host(g.n, g.src, g.dst, g.k, [0.6, 0.75, 0.9])
    ob, ou = oracle.count_threshold(g.n, g.src, g.dst, g.k, [0.6, 0.75, 0.9])
    assert np.array_equal(b, ob) and np.array_equal(u, ou)


def test_workspace_one_byte_short_is_refused_before_any_kernel(ubt, er2k):
    """A workspace one byte below the queried size: ubt_create_graph,
    ubt_sample_worlds, ubt_topk and ubt_count_host return
    UBT_ERR_WORKSPACE_TOO_SMALL and leave their outputs untouched."""
    import ctypes
    import torch
    g = er2k
    L = ubt.lib()
    cp = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    src = torch.from_numpy(g.src.view(np.int32)).cuda()
    dst = torch.from_numpy(g.dst.view(np.int32)).cuda()
    kk = torch.from_numpy(g.k.view(np.int32)).cuda()
    nb = ctypes.c_size_t(0)
    assert L.ubt_graph_workspace_size(g.n, g.m, 0, None, ctypes.byref(nb)) == 0
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p(0)
    st = L.ubt_create_graph(g.n, g.m, cp(src), cp(dst), cp(kk), None, 0, None, cp(ws), int(nb.value) - 1, stream,
                            ctypes.byref(h))
    assert st == -8 and not h.value
    G = ubt.Graph(g.n, g.src, g.dst, k=g.k)
    W = 128
    need = G.sample_worlds_workspace(W)
    wws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.full((W,), -1, dtype=torch.int64, device="cuda")
    st = L.ubt_sample_worlds(G.handle, ctypes.c_uint64(7), W, cp(out), None, cp(wws), need - 1, stream)
    assert st == -8
    torch.cuda.synchronize()
    assert bool((out == -1).all())
    K = 100
    L.ubt_topk_workspace_size(K, ctypes.byref(nb))
    tw = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    tout = torch.full((K * ubt.TRI_REC_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device="cuda")
    nout = ctypes.c_int64(-1)
    st = L.ubt_topk(G.handle, K, 1, cp(tout), ctypes.byref(nout), cp(tw), int(nb.value) - 1, stream)
    assert st == -8 and nout.value == -1
    torch.cuda.synchronize()
    assert bool((tout == 0xAB).all())
    L.ubt_count_host_workspace_size(g.n, g.m, ctypes.byref(nb))
    hws = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    taus = np.array([0.6, 0.9])
    hout = np.full(4, -1, dtype=np.int64)
    st = L.ubt_count_host(g.n, g.m, g.src.ctypes.data_as(ctypes.c_void_p), g.dst.ctypes.data_as(ctypes.c_void_p),
                          g.k.ctypes.data_as(ctypes.c_void_p), taus.ctypes.data_as(ctypes.c_void_p), 2, 1,
                          hout.ctypes.data_as(ctypes.c_void_p), cp(hws), int(nb.value) - 1, stream)
    assert st == -8 and (hout == -1).all()
    assert G.guard() == 0
