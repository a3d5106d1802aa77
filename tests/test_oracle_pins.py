"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something fixed independently of its
code: brute force over every sign world in exact rational arithmetic, O(n^3)
listing, closed forms on complete graphs, the single-triangle cases the paper
fixes in words (tests/golden/boundary_cases.json), the paper's lemmas as
invariants, finite differences, and numpy's Philox generator.  None of these
needs a GPU.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ONE = 65536


# ---------------------------------------------------------------- helpers

def brute_triangles(n, src, dst):
    """O(n^3) triangle listing over the adjacency matrix: sorted (a<b<c) rows
    with the input edge index of (ab, ac, bc)."""
    A = np.full((n, n), -1, dtype=np.int64)
    for i, (a, b) in enumerate(zip(src.tolist(), dst.tolist())):
        A[a, b] = i
        A[b, a] = i
    out_v, out_e = [], []
    for a in range(n):
        for b in range(a + 1, n):
            if A[a, b] < 0:
                continue
            for c in range(b + 1, n):
                if A[a, c] >= 0 and A[b, c] >= 0:
                    out_v.append((a, b, c))
                    out_e.append((A[a, b], A[a, c], A[b, c]))
    return (np.asarray(out_v, dtype=np.int64).reshape(-1, 3),
            np.asarray(out_e, dtype=np.int64).reshape(-1, 3))


def world_prob_table(probs):
    """All 2^m sign worlds: returns list of (signs tuple, probability Fraction).
    Edge signs independent, P(+) = probs[e] (Fractions)."""
    m = len(probs)
    out = []
    for signs in itertools.product((0, 1), repeat=m):
        pr = Fraction(1)
        for e, s in enumerate(signs):
            pr *= probs[e] if s else (1 - probs[e])
        out.append((signs, pr))
    return out


def small_graph(seed, n, m):
    s, d = synth.er_graph(n, m, seed)
    return s, d


def special_k(m, seed):
    """k values mixing certain edges, coin flips and uniform draws."""
    g = synth.rng(seed)
    k = synth.k_uniform(m, seed).astype(np.int64)
    pick = g.random(m)
    k[pick < 0.15] = 0
    k[(pick >= 0.15) & (pick < 0.3)] = ONE
    k[(pick >= 0.3) & (pick < 0.4)] = ONE // 2
    return k.astype(np.uint32)


# ---------------------------------------------------------------- listing

@pytest.mark.parametrize("seed,n,m", [(1, 30, 120), (2, 60, 500), (3, 90, 1500), (4, 12, 66)])
def test_listing_matches_bruteforce(seed, n, m):
    s, d = small_graph(seed, n, m)
    v, e = oracle.list_triangles(n, s, d)
    bv, be = brute_triangles(n, s, d)
    assert v.shape == bv.shape
    assert np.array_equal(v.astype(np.int64), bv)
    assert np.array_equal(e.astype(np.int64), be)
    assert oracle.num_triangles(n, s, d) == bv.shape[0]


def test_triangle_count_trace_formula():
    g = synth.config_graph("er2k")
    A = np.zeros((g.n, g.n), dtype=np.float64)
    A[g.src, g.dst] = 1
    A[g.dst, g.src] = 1
    tr = np.trace(A @ A @ A) / 6.0
    assert oracle.num_triangles(g.n, g.src, g.dst) == int(round(tr))


def test_rejects_invalid_graphs():
    with pytest.raises(oracle.OracleError, match="self-loop"):
        oracle.num_triangles(4, np.array([0, 1]), np.array([1, 1]))
    with pytest.raises(oracle.OracleError, match="duplicate"):
        oracle.num_triangles(4, np.array([0, 1]), np.array([1, 0]))
    with pytest.raises(oracle.OracleError, match="vertex"):
        oracle.num_triangles(4, np.array([0, 1]), np.array([4, 2]))
    with pytest.raises(oracle.OracleError, match="probability"):
        oracle.count_threshold(4, np.array([0]), np.array([1]), np.array([65537]), [0.6])
    with pytest.raises(oracle.OracleError, match="tau"):
        oracle.count_threshold(4, np.array([0]), np.array([1]), np.array([5]), [0.4])


def test_empty_graphs():
    z = np.zeros(0, dtype=np.uint32)
    assert oracle.num_triangles(0, z, z) == 0
    assert oracle.num_triangles(5, z, z) == 0
    b, u = oracle.count_threshold(5, z, z, z, [0.6, 0.9])
    assert b.tolist() == [0, 0] and u.tolist() == [0, 0]
    assert oracle.expected_fixed(5, z, z, z) == (0, 0)


# ---------------------------------------------------------------- brute force over sign worlds

@pytest.mark.parametrize("seed,n,m", [(11, 7, 12), (12, 6, 13), (13, 8, 13), (14, 5, 10)])
def test_pbal_counts_and_expected_match_all_sign_worlds(seed, n, m):
    """Sec. 3: P_bal is the probability that the triangle has an odd number of
    positive edges under independent signs.  Sum that over every one of the
    2^m sign worlds in exact rationals and compare every oracle output."""
    s, d = small_graph(seed, n, m)
    k = special_k(m, seed)
    probs = [Fraction(int(x), ONE) for x in k]
    worlds = world_prob_table(probs)
    bv, be = brute_triangles(n, s, d)
    assert bv.shape[0] > 0
    # exact P_bal per triangle by brute force
    pbal = []
    for tri in be:
        acc = Fraction(0)
        for signs, pr in worlds:
            if (signs[tri[0]] + signs[tri[1]] + signs[tri[2]]) % 2 == 1:
                acc += pr
        pbal.append(acc)
    # enumeration at t = 0.5 lists every triangle exactly once, with exact P_bal
    uvw, cls, pb = oracle.enumerate_records(n, s, d, k, 0.5, 3)
    assert np.array_equal(uvw.astype(np.int64), bv)
    for i, ex in enumerate(pbal):
        assert Fraction(float(pb[i])) == ex
        assert cls[i] == (1 if ex >= Fraction(1, 2) else 2)
    # counts at several thresholds, straight from the definitions
    taus = [0.5, 0.55, 0.6, 0.75, 0.8, 0.9, 0.99, 1.0]
    bal, unbal = oracle.count_threshold(n, s, d, k, taus)
    for i, t in enumerate(taus):
        ft = Fraction(t)
        assert bal[i] == sum(1 for x in pbal if x >= ft)
        assert unbal[i] == sum(1 for x in pbal if 1 - x > ft)
    # expected number of balanced triangles = sum over worlds of P(world) * #balanced
    e_bal = Fraction(0)
    for signs, pr in worlds:
        nb = sum(1 for tri in be if (signs[tri[0]] + signs[tri[1]] + signs[tri[2]]) % 2 == 1)
        e_bal += pr * nb
    T, S = oracle.expected_fixed(n, s, d, k)
    assert T == bv.shape[0]
    assert Fraction(S, 1 << 48) == e_bal


@pytest.mark.parametrize("seed", [21, 22])
def test_expected_real_matches_all_sign_worlds(seed):
    n, m = 7, 13
    s, d = small_graph(seed, n, m)
    p = synth.p_uniform_f32(m, seed)
    p[0] = 0.0
    p[1] = 1.0
    probs = [Fraction(float(x)) for x in p]
    worlds = world_prob_table(probs)
    _, be = brute_triangles(n, s, d)
    e_bal = Fraction(0)
    for signs, pr in worlds:
        nb = sum(1 for tri in be if (signs[tri[0]] + signs[tri[1]] + signs[tri[2]]) % 2 == 1)
        e_bal += pr * nb
    eb, eu, T = oracle.expected_real(n, s, d, p)
    assert T == be.shape[0]
    assert abs(eb - float(e_bal)) <= 1e-14 * max(1.0, float(e_bal))
    assert abs(eu - float(T - e_bal)) <= 1e-14 * max(1.0, float(T - e_bal))


# ---------------------------------------------------------------- closed forms on K_n

@pytest.mark.parametrize("n,k", [(6, 49152), (9, 1000), (10, 65536), (8, 32768), (7, 0), (12, 60000)])
def test_complete_graph_closed_forms(n, k):
    """On K_n with one P+ for every edge, E[(-1)^{#positive}] = s^3 with
    s = 1 - 2p (product of independent factors), hence P_bal = (1 - s^3)/2 for
    each of the C(n,3) triangles, and d P_bal / d p_e = s^2 for each of the
    n - 2 triangles through an edge."""
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    s = np.array([a for a, _ in pairs], dtype=np.uint32)
    d = np.array([b for _, b in pairs], dtype=np.uint32)
    kk = np.full(len(pairs), k, dtype=np.uint32)
    T = math.comb(n, 3)
    p = Fraction(k, ONE)
    sg = 1 - 2 * p
    pbal = (1 - sg ** 3) / 2
    taus = [0.5, 0.6, 0.75, 0.9, 1.0]
    bal, unbal = oracle.count_threshold(n, s, d, kk, taus)
    for i, t in enumerate(taus):
        assert bal[i] == (T if pbal >= Fraction(t) else 0)
        assert unbal[i] == (T if 1 - pbal > Fraction(t) else 0)
    T2, S = oracle.expected_fixed(n, s, d, kk)
    assert T2 == T and Fraction(S, 1 << 48) == T * pbal
    pf = np.full(len(pairs), k / ONE, dtype=np.float32)
    g = oracle.grad_real(n, s, d, pf)
    assert np.allclose(g, float((n - 2) * sg ** 2), rtol=0, atol=1e-12)
    eb, eu, T3 = oracle.expected_real(n, s, d, pf)
    assert T3 == T
    assert abs(eb - float(T * pbal)) <= 1e-12 * T


# ---------------------------------------------------------------- boundary cases from the paper's text

def _golden_cases():
    with open(os.path.join(GOLDEN, "boundary_cases.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_boundary_cases(case):
    s = np.array([0, 0, 1], dtype=np.uint32)
    d = np.array([1, 2, 2], dtype=np.uint32)
    k = np.array(case["k"], dtype=np.uint32)
    uvw, cls, pb = oracle.enumerate_records(3, s, d, k, 0.5, 3)
    assert uvw.tolist() == [[0, 1, 2]]
    assert pb[0] == case["p_bal"]
    for t, eb, eu in case["counts"]:
        bal, unbal = oracle.count_threshold(3, s, d, k, [t])
        assert (int(bal[0]), int(unbal[0])) == (eb, eu), (t, case["name"])


# ---------------------------------------------------------------- invariants from the lemmas

@pytest.mark.parametrize("seed", [31, 32, 33])
def test_partition_at_half(seed):
    """At t = 0.5 the unclassified range [1-t, t) is empty (Def. 6): every
    triangle is balanced or unbalanced, never both."""
    s, d = small_graph(seed, 200, 3000)
    k = special_k(s.size, seed)
    bal, unbal = oracle.count_threshold(200, s, d, k, [0.5])
    assert bal[0] + unbal[0] == oracle.num_triangles(200, s, d)


@pytest.mark.parametrize("seed", [41, 42])
def test_lemma1_reversal(seed):
    """Lemma 1: with every P+ replaced by 1 - P+, a triangle's balance
    probability becomes its old unbalance probability.  Counts therefore swap,
    up to ties at exactly t (balanced uses >=, unbalanced uses >)."""
    n = 150
    s, d = small_graph(seed, n, 2500)
    k = special_k(s.size, seed)
    kr = (ONE - k.astype(np.int64)).astype(np.uint32)
    uvw, _, pb = oracle.enumerate_records(n, s, d, k, 0.5, 3)
    uvw_r, _, pb_r = oracle.enumerate_records(n, s, d, kr, 0.5, 3)
    assert np.array_equal(uvw, uvw_r)
    assert np.array_equal(pb_r, 1.0 - pb)
    taus = [0.5, 0.6, 0.75, 0.875, 0.9, 1.0]
    bal, unbal = oracle.count_threshold(n, s, d, k, taus)
    bal_r, unbal_r = oracle.count_threshold(n, s, d, kr, taus)
    for i, t in enumerate(taus):
        ties_unbal = int(np.sum((1.0 - pb) == t))
        ties_bal = int(np.sum(pb == t))
        assert bal_r[i] == unbal[i] + ties_unbal
        assert unbal_r[i] == bal[i] - ties_bal


@pytest.mark.parametrize("seed", [51, 52])
def test_lemma2_edge_bounds(seed):
    """Lemma 2: a triangle's balance (and unbalance) probability lies within
    [min(p, 1-p), max(p, 1-p)] for each of its edges."""
    n = 120
    s, d = small_graph(seed, n, 2000)
    k = special_k(s.size, seed)
    vtx, eid = oracle.list_triangles(n, s, d)
    uvw, _, pb = oracle.enumerate_records(n, s, d, k, 0.5, 3)
    assert np.array_equal(vtx, uvw)
    p = k.astype(np.float64) / ONE
    for j in range(3):
        pe = p[eid[:, j]]
        lo = np.minimum(pe, 1 - pe)
        hi = np.maximum(pe, 1 - pe)
        assert np.all(pb >= lo) and np.all(pb <= hi)
        assert np.all(1 - pb >= lo) and np.all(1 - pb <= hi)


def test_monotone_in_tau():
    g = synth.config_graph("er2k")
    taus = np.linspace(0.5, 1.0, 41)
    bal, unbal = oracle.count_threshold(g.n, g.src, g.dst, g.k, taus)
    assert np.all(np.diff(bal) <= 0) and np.all(np.diff(unbal) <= 0)


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("seed", [61, 62])
def test_gradient_matches_central_differences(seed):
    """E_bal is affine in each p_e (a triangle holds three distinct edges), so a
    central difference is exact up to rounding."""
    n = 40
    s, d = small_graph(seed, n, 300)
    p = synth.p_uniform_f32(s.size, seed)
    g = oracle.grad_real(n, s, d, p)
    h = np.float32(2.0 ** -6)
    for e in range(0, s.size, 7):
        pp = p.copy(); pp[e] = p[e] + h
        pm = p.copy(); pm[e] = p[e] - h
        # the oracle rejects p outside [0, 1]; shift the stencil inside when needed
        if pp[e] > 1.0:
            pp[e], pm[e] = p[e], p[e] - 2 * h
        if pm[e] < 0.0:
            pp[e], pm[e] = p[e] + 2 * h, p[e]
        fp = oracle.expected_real(n, s, d, pp)[0]
        fm = oracle.expected_real(n, s, d, pm)[0]
        fd = (fp - fm) / (float(pp[e]) - float(pm[e]))
        assert abs(fd - g[e]) <= 1e-9 * max(1.0, abs(g[e])), e


# ---------------------------------------------------------------- Philox and sign worlds

def numpy_philox_block(ctr, key):
    """Philox4x64-10 of one counter through numpy (which increments the
    counter before producing each block)."""
    c = int(ctr[0]) | (int(ctr[1]) << 64) | (int(ctr[2]) << 128) | (int(ctr[3]) << 192)
    c = (c - 1) % (1 << 256)
    words = [(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(words, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 2, 3, 4], [5, 6]),
    ([2**64 - 1, 2**64 - 1, 7, 9], [2**63 + 11, 12345]),
    ([123456789, 42, 3, 0], [987654321, 0]),
])
def test_philox_matches_numpy(ctr, key):
    assert np.array_equal(oracle.philox4x64_10(ctr, key), numpy_philox_block(ctr, key))


def world_word_numpy(seed, ekey, w, k):
    r = np.concatenate([numpy_philox_block([ekey, w, c, 0], [seed, 0]) for c in range(4)])
    word = 0
    for j in range(64):
        u = 0
        for b in range(16):
            u |= ((int(r[b]) >> j) & 1) << b
        if u < k:
            word |= 1 << j
    return word


def test_world_word_matches_numpy_draws():
    for (seed, ekey, w, k) in [(1, 0, 0, 32768), (7, 123, 5, 1), (99, 4000000, 63, 65535),
                               (3, 17, 2, 65536), (3, 17, 2, 0), (2**40 + 5, 9, 1, 40000)]:
        assert oracle.world_word(seed, ekey, w, k) == world_word_numpy(seed, ekey, w, k)


def test_world_sign_frequencies():
    """P(+) = k / 65536: each world bit is a Bernoulli(k/65536) draw."""
    words = 400
    for k in [0, 1, 6553, 32768, 50000, 65535, 65536]:
        ones = sum(bin(oracle.world_word(5, e, w, k)).count("1") for e in range(5) for w in range(words // 5))
        trials = 64 * words
        p = k / ONE
        sd = math.sqrt(max(trials * p * (1 - p), 1e-12))
        assert abs(ones - trials * p) <= 6 * sd + 1e-9, k


def test_world_counts_match_independent_recount():
    n, m = 9, 22
    s, d = small_graph(71, n, m)
    k = special_k(m, 71)
    ekey = (np.arange(m, dtype=np.uint32) * 7 + 3).astype(np.uint32)
    words = [0, 3]
    seed = 1234
    got = oracle.world_counts(n, s, d, k, seed, words, ekey=ekey)
    _, be = brute_triangles(n, s, d)
    bits = {(e, w): world_word_numpy(seed, int(ekey[e]), w, int(k[e])) for e in range(m) for w in words}
    want = np.zeros(len(words) * 64, dtype=np.int64)
    for i, w in enumerate(words):
        for j in range(64):
            for tri in be:
                pos = sum((bits[(int(e), w)] >> j) & 1 for e in tri)
                want[i * 64 + j] += pos % 2
    assert np.array_equal(got, want)


def test_world_mean_estimates_expected_count():
    g = synth.config_graph("er2k")
    words = list(range(16))  # 1024 worlds
    c = oracle.world_counts(g.n, g.src, g.dst, g.k, 77, words).astype(np.float64)
    T, S = oracle.expected_fixed(g.n, g.src, g.dst, g.k)
    e_bal = S / float(1 << 48)
    sd = c.std(ddof=1) / math.sqrt(c.size)
    assert abs(c.mean() - e_bal) <= 6 * sd


# ---------------------------------------------------------------- local counts (Sec. 6 samplers)

@pytest.mark.parametrize("seed,n,m", [(41, 8, 14), (42, 7, 13)])
def test_local_counts_match_all_sign_worlds(seed, n, m):
    """|B_t(e)| and |B_t(v)|: classified triangles through an edge or a vertex,
    from exact rational P_bal over every sign world and O(n^3) listing."""
    s, d = small_graph(seed, n, m)
    k = special_k(m, seed)
    probs = [Fraction(int(x), ONE) for x in k]
    worlds = world_prob_table(probs)
    bv, be = brute_triangles(n, s, d)
    taus = [0.5, 0.6, 0.8, 0.95]
    want_eb = np.zeros((m, len(taus)), dtype=np.int64)
    want_eu = np.zeros((m, len(taus)), dtype=np.int64)
    want_vb = np.zeros((n, len(taus)), dtype=np.int64)
    want_vu = np.zeros((n, len(taus)), dtype=np.int64)
    for tri_v, tri_e in zip(bv, be):
        pb = sum((pr for signs, pr in worlds if (signs[tri_e[0]] + signs[tri_e[1]] + signs[tri_e[2]]) % 2 == 1),
                 Fraction(0))
        for i, t in enumerate(taus):
            if pb >= Fraction(t):
                want_eb[tri_e, i] += 1
                want_vb[tri_v, i] += 1
            if 1 - pb > Fraction(t):
                want_eu[tri_e, i] += 1
                want_vu[tri_v, i] += 1
    eb, eu, vb, vu = oracle.local_counts(n, s, d, k, taus)
    assert np.array_equal(eb, want_eb) and np.array_equal(eu, want_eu)
    assert np.array_equal(vb, want_vb) and np.array_equal(vu, want_vu)


@pytest.mark.parametrize("seed", [43, 44])
def test_local_counts_sum_to_three_times_the_counts(seed):
    """Every triangle has three edges and three vertices."""
    s, d = synth.er_graph(300, 6000, seed)
    k = special_k(s.size, seed)
    taus = [0.5, 0.55, 0.7, 0.9, 1.0]
    bal, unbal = oracle.count_threshold(300, s, d, k, taus)
    eb, eu, vb, vu = oracle.local_counts(300, s, d, k, taus)
    assert np.array_equal(eb.sum(0), 3 * bal) and np.array_equal(eu.sum(0), 3 * unbal)
    assert np.array_equal(vb.sum(0), 3 * bal) and np.array_equal(vu.sum(0), 3 * unbal)


@pytest.mark.parametrize("n,k", [(7, 49152), (9, 1000), (6, 32768)])
def test_local_counts_complete_graph(n, k):
    """K_n with one P+: every edge is in n - 2 triangles, every vertex in
    C(n-1, 2), all with P_bal = (1 - s^3)/2."""
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    s = np.array([a for a, _ in pairs], dtype=np.uint32)
    d = np.array([b for _, b in pairs], dtype=np.uint32)
    kk = np.full(len(pairs), k, dtype=np.uint32)
    sg = 1 - 2 * Fraction(k, ONE)
    pbal = (1 - sg ** 3) / 2
    taus = [0.5, 0.6, 0.9]
    eb, eu, vb, vu = oracle.local_counts(n, s, d, kk, taus)
    for i, t in enumerate(taus):
        isb, isu = pbal >= Fraction(t), 1 - pbal > Fraction(t)
        assert np.all(eb[:, i] == (n - 2) * isb) and np.all(eu[:, i] == (n - 2) * isu)
        assert np.all(vb[:, i] == math.comb(n - 1, 2) * isb) and np.all(vu[:, i] == math.comb(n - 1, 2) * isu)


# ------------------------------------------- the multi-threaded resident count

@pytest.mark.parametrize("name", ["er2k", "mixed", "rmat12", "cl"])
def test_resident_count_equals_serial_pass(name):
    """ResidentGraph.count (Alg. 1's outer loop split over threads) gives the
    serial oracle's counts for every thread count, and its samples partition
    them."""
    if name == "er2k":
        g = synth.config_graph("er2k")
        n, s, d, k = g.n, g.src, g.dst, g.k
    elif name == "mixed":
        n = 400
        s, d = synth.er_graph(n, 6000, 71)
        k = special_k(s.size, 72)
    elif name == "rmat12":
        g = synth.config_graph("rmat12")
        n, s, d, k = g.n, g.src, g.dst, g.k
    else:
        n = 20000
        s, d = synth.chung_lu(n, 2.1, 20.0, 2000.0, 73)
        k = synth.quantise(synth.p_beta_mixture(s.size, 74))
    taus = [0.51 + i * (0.48 / 31) for i in range(32)]
    b, u = oracle.count_threshold(n, s, d, k, taus)
    T = oracle.num_triangles(n, s, d)
    R = oracle.ResidentGraph(n, s, d)
    for th in (1, 2, 7):
        b2, u2, t2 = R.count(k, taus, threads=th)
        assert np.array_equal(b2, b) and np.array_equal(u2, u) and t2 == T, th
    sb, su, st = np.zeros(32, np.int64), np.zeros(32, np.int64), 0
    for r in range(3):
        b3, u3, t3 = R.count(k, taus, threads=3, sample_mod=3, sample_rem=r)
        sb, su, st = sb + b3, su + u3, st + t3
    assert np.array_equal(sb, b) and np.array_equal(su, u) and st == T
    R.close()


def test_resident_count_sample_is_the_triangles_of_the_sampled_earliest_vertices():
    """A sample (class(u) == rem) counts exactly the triangles whose earliest
    vertex in Node Order (degree, then id) is such a u: checked against the
    O(n^3) listing with Node Order computed here."""
    n = 70
    s, d = synth.er_graph(n, 900, 81)
    k = special_k(s.size, 82)
    tri, _ = brute_triangles(n, s, d)
    deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=n)
    rank = np.lexsort((np.arange(n), deg))  # vertices in Node Order
    pos = np.empty(n, np.int64)
    pos[rank] = np.arange(n)
    first = tri[np.arange(tri.shape[0]), np.argmin(pos[tri], axis=1)]
    R = oracle.ResidentGraph(n, s, d)
    for mod in (2, 5):
        cls = np.array([oracle.sample_class(x, mod) for x in range(n)])
        assert np.all((cls >= 0) & (cls < mod))
        for rem in range(mod):
            _, _, t = R.count(k, [0.5], threads=2, sample_mod=mod, sample_rem=rem)
            assert t == int(np.count_nonzero(cls[first] == rem)), (mod, rem)
