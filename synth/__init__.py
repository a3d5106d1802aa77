"""Seeded synthetic inputs for the uncertain-signed-triangle path.

This module is shared by the CUDA path's tests and benchmark and by the
CPU oracle's tests.  It only draws graphs and edge-sign probabilities; it
contains none of the method's arithmetic (no balance probabilities, no
thresholds, no triangle listing).

The paper's datasets (SNAP/Konect graphs with synthetic sign probabilities,
Sec. 7.1, Table 2) are not available, so these generators stand in for them:

* ``er_graph``     -- Erdos-Renyi G(n, m): m distinct unordered pairs.
* ``chung_lu``     -- power-law expected-degree graph (Chung-Lu).
* ``rmat``         -- R-MAT / Kronecker edge draws, symmetrised, deduplicated.
* ``k_uniform``    -- 16-bit fixed-point probabilities k ~ U{0..65536}.
* ``quantise``     -- real p in [0,1] -> k = round-half-even(p * 65536).
* ``p_beta`` / ``p_beta_mixture`` / ``p_uniform_f32`` -- the P+ distributions
  the paper uses (uniform, Beta(0.5,0.5), sign-biased Betas; Sec. 7.1).
* ``ego_select`` / ``ego_induce`` / ``ego_induce_torch`` / ``ego_nets`` --
  batches of induced ego-net subgraphs of a parent graph (member sets on the
  CPU; induced edges on the CPU or, for large batches, with torch on a GPU).
* ``bfs_induced``  -- induced subgraph grown in BFS order to a target size.

Every graph is returned as ``(src, dst)`` uint32 arrays of an undirected
simple graph (no self-loops, no duplicate pairs); the edge index in these
arrays is the edge id ``eid`` used everywhere else.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import threading

import numpy as np

__all__ = [
    "rng", "er_graph", "chung_lu", "rmat", "k_uniform", "quantise",
    "p_beta", "p_beta_mixture", "p_uniform_f32", "ego_nets", "bfs_induced",
    "csr_undirected", "random_orientation", "Graph", "config_graph",
]

K_ONE = 65536  # fixed-point denominator: p = k / 65536, k in [0, 65536]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _map(fn, items):
    """Thread-pool map (numpy releases the GIL in the heavy loops); the result
    does not depend on the number of workers."""
    items = list(items)
    if len(items) <= 1 or _workers() == 1:
        return [fn(x) for x in items]
    with cf.ThreadPoolExecutor(_workers()) as ex:
        return list(ex.map(fn, items))


def _chunk_rng(seed: int, chunk: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, chunk])))


def _merge_unique(parts) -> np.ndarray:
    """Sorted distinct values of the union of sorted int64 arrays, computed in
    key ranges in parallel."""
    parts = [p for p in parts if p.size]
    if not parts:
        return np.zeros(0, dtype=np.int64)
    total = sum(p.size for p in parts)
    nr = max(1, min(4 * _workers(), total // (1 << 20)))
    sample = np.sort(np.concatenate([p[:: max(1, p.size // 256)] for p in parts]))
    splits = [None] + [int(sample[(i * sample.size) // nr]) for i in range(1, nr)] + [None]

    def one(i):
        lo, hi = splits[i], splits[i + 1]
        seg = []
        for p in parts:
            a = 0 if lo is None else np.searchsorted(p, lo, side="left")
            b = p.size if hi is None else np.searchsorted(p, hi, side="left")
            seg.append(p[a:b])
        return _sorted_unique(np.concatenate(seg))

    return np.concatenate(_map(one, range(nr)))


def _sorted_unique(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent compare; faster than np.unique here)."""
    keys = np.sort(keys, kind="stable")
    if keys.size == 0:
        return keys
    keep = np.empty(keys.size, dtype=bool)
    keep[0] = True
    np.not_equal(keys[1:], keys[:-1], out=keep[1:])
    return keys[keep]


def _dedup_pairs(a: np.ndarray, b: np.ndarray, n: int):
    """Canonicalise to (min, max), drop self-loops and duplicate pairs.

    Keeps the first draw of each pair and returns pairs sorted by (min, max).
    """
    a = a.astype(np.int64)
    b = b.astype(np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = _sorted_unique(lo * np.int64(n) + hi)
    return (key // n).astype(np.uint32), (key % n).astype(np.uint32)


def er_graph(n: int, m: int, seed: int, shuffle_endpoints: bool = True):
    """G(n, m): m distinct unordered pairs drawn uniformly, no self-loops.

    The edges come out in a random order and, with ``shuffle_endpoints``,
    with a random endpoint first, so consumers must canonicalise.
    """
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the number of vertex pairs")
    g = rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = int((m - keys.size) * 1.3) + 16
        a = g.integers(0, n, size=need, dtype=np.int64)
        b = g.integers(0, n, size=need, dtype=np.int64)
        ok = a != b
        lo = np.minimum(a[ok], b[ok])
        hi = np.maximum(a[ok], b[ok])
        new = lo * n + hi
        allk = np.concatenate([keys, new])
        _, first = np.unique(allk, return_index=True)
        keys = allk[np.sort(first)]
    keys = keys[:m]
    src = (keys // n).astype(np.uint32)
    dst = (keys % n).astype(np.uint32)
    if shuffle_endpoints:
        flip = g.random(m) < 0.5
        src, dst = np.where(flip, dst, src), np.where(flip, src, dst)
    return src, dst


def chung_lu(n: int, gamma: float, mean_deg: float, max_deg: float, seed: int):
    """Chung-Lu power-law graph.

    Expected-degree weights w_i = c * (i + 1)^(-1/(gamma-1)), scaled so the
    mean is ``mean_deg`` after capping every weight at ``max_deg`` (the scale
    is solved by bisection).  n * mean_deg / 2 endpoint pairs are drawn with
    probability proportional to w (inverse-CDF sampling); self-loops and
    repeated pairs are dropped, so the realised edge count is a little below
    the nominal one and is whatever the returned arrays hold.
    """
    base = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    lo, hi = 0.0, mean_deg * n / base.sum() * 1e4
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.minimum(base * mid, max_deg).mean() < mean_deg:
            lo = mid
        else:
            hi = mid
    w = np.minimum(base * hi, max_deg)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    draws = int(round(n * mean_deg / 2.0))
    chunk = 1 << 21

    def one(c):
        cnt = min(chunk, draws - c * chunk)
        r = _chunk_rng(seed, c)
        a = np.minimum(np.searchsorted(cdf, r.random(cnt), side="right"), n - 1).astype(np.int64)
        b = np.minimum(np.searchsorted(cdf, r.random(cnt), side="right"), n - 1).astype(np.int64)
        keep = a != b
        a, b = a[keep], b[keep]
        return _sorted_unique(np.minimum(a, b) * n + np.maximum(a, b))

    key = _merge_unique(_map(one, range((draws + chunk - 1) // chunk)))
    return (key // n).astype(np.uint32), (key % n).astype(np.uint32)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         chunk: int = 1 << 21):
    """R-MAT edge draws on 2^scale vertices, symmetrised and deduplicated.

    Each of the 2^scale * edge_factor draws picks one quadrant per level
    with probabilities (a, b, c, 1-a-b-c).  Draws come in chunks of 2^21, each
    from its own seed (seed, chunk).  Vertex labels are not permuted.
    """
    n = 1 << scale
    total = n * edge_factor
    ab, abc = a + b, a + b + c

    def one(ci):
        cnt = min(chunk, total - ci * chunk)
        g = _chunk_rng(seed, ci)
        u = np.zeros(cnt, dtype=np.int64)
        v = np.zeros(cnt, dtype=np.int64)
        for _ in range(scale):
            r = g.random(cnt, dtype=np.float32)
            u = (u << 1) | (r >= ab)                       # quadrants c, d
            v = (v << 1) | (((r >= a) & (r < ab)) | (r >= abc))  # quadrants b, d
        keep = u != v
        u, v = u[keep], v[keep]
        return _sorted_unique(np.minimum(u, v) * n + np.maximum(u, v))

    key = _merge_unique(_map(one, range((total + chunk - 1) // chunk)))
    return (key // n).astype(np.uint32), (key % n).astype(np.uint32)


def k_uniform(m: int, seed: int) -> np.ndarray:
    """k ~ Uniform{0, ..., 65536} (all 65,537 fixed-point values)."""
    return rng(seed).integers(0, K_ONE + 1, size=m, dtype=np.int64).astype(np.uint32)


def quantise(p: np.ndarray) -> np.ndarray:
    """k = round-half-even(p * 65536), clamped to [0, 65536]."""
    k = np.rint(np.asarray(p, dtype=np.float64) * K_ONE)
    return np.clip(k, 0, K_ONE).astype(np.uint32)


def p_beta(m: int, alpha: float, beta: float, seed: int) -> np.ndarray:
    return rng(seed).beta(alpha, beta, size=m)


def p_normal(m: int, seed: int, mean: float = 0.5, sd: float = 0.15) -> np.ndarray:
    """Normal(mean, sd) clipped to [0, 1] (the paper's Sec. 6 distribution
    study names a Normal without its parameters)."""
    return np.clip(rng(seed).normal(mean, sd, size=m), 0.0, 1.0)


def p_beta_mixture(m: int, seed: int, w: float = 0.5,
                   ab1=(8.0, 2.0), ab2=(2.0, 8.0)) -> np.ndarray:
    """w * Beta(ab1) + (1 - w) * Beta(ab2): sign-confident bimodal P+."""
    g = rng(seed)
    pick = g.random(m) < w
    x1 = g.beta(ab1[0], ab1[1], size=m)
    x2 = g.beta(ab2[0], ab2[1], size=m)
    return np.where(pick, x1, x2)


def p_uniform_f32(m: int, seed: int) -> np.ndarray:
    return rng(seed).random(m, dtype=np.float32)


def random_orientation(src, dst, seed: int):
    """Swap the endpoints of a random half of the edges (same graph)."""
    flip = rng(seed).random(len(src)) < 0.5
    return np.where(flip, dst, src).astype(np.uint32), np.where(flip, src, dst).astype(np.uint32)


def csr_undirected(n: int, src, dst):
    """Undirected adjacency (both directions) as (offsets int64, nbr uint32, eid int64)."""
    m = len(src)
    a = np.concatenate([src, dst]).astype(np.int64)
    b = np.concatenate([dst, src]).astype(np.int64)
    e = np.concatenate([np.arange(m), np.arange(m)]).astype(np.int64)
    order = np.lexsort((b, a))
    a, b, e = a[order], b[order], e[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, a + 1, 1)
    off = np.cumsum(off)
    return off, b.astype(np.uint32), e


def ego_select(n: int, src, dst, count: int, smin: int, smax: int, seed: int):
    """Seeded member sets of a batch of ego nets.

    For ego net i (drawn from its own seed (seed, i)): the size s is
    log-uniform in [smin, smax]; the centre is a uniformly chosen vertex with
    degree >= s - 1 (if none exists, the highest-degree vertex and
    s = deg + 1); the members are the centre plus s - 1 of its neighbours
    chosen uniformly without replacement.

    Returns {"v_off": int64 [count + 1], "vid": uint32 [members]} with every
    ego net's members sorted by parent id.
    """
    off, nbr, _ = csr_undirected(n, src, dst)
    deg = np.diff(off)
    order_by_deg = np.argsort(deg, kind="stable")
    sorted_deg = deg[order_by_deg]

    def one(i):
        g = _chunk_rng(seed, i)
        s = int(round(np.exp(g.uniform(np.log(smin), np.log(smax)))))
        first = np.searchsorted(sorted_deg, s - 1, side="left")
        if first >= n:
            centre = int(order_by_deg[-1])
            s = int(deg[centre]) + 1
        else:
            centre = int(order_by_deg[g.integers(first, n)])
        nb = nbr[off[centre]:off[centre + 1]].astype(np.int64)
        pick = g.choice(nb.size, size=min(s - 1, nb.size), replace=False)
        return np.unique(np.concatenate([[centre], nb[pick]]))

    sets = _map(one, range(count))
    v_off = np.zeros(count + 1, dtype=np.int64)
    v_off[1:] = np.cumsum([x.size for x in sets])
    vid = np.concatenate(sets).astype(np.uint32) if sets else np.zeros(0, np.uint32)
    return {"v_off": v_off, "vid": vid}


def ego_induce(n: int, src, dst, sel, which=None):
    """Subgraphs the parent induces on the member sets of `sel` (all of them,
    or the ego nets listed in `which`), as one batch.

    Returns a dict of concatenated arrays:
      v_off (count+1, int64): vertex offsets; graph i owns global ids
          [v_off[i], v_off[i+1]), in the order of its sorted member list.
      e_off (count+1, int64): edge offsets into src/dst/eid.
      src, dst (uint32): GLOBAL vertex ids, src < dst; edges of a graph come
          in member order, then in the parent's adjacency order.
      eid (uint32): the parent edge id of each subgraph edge.
      vid (uint32): parent vertex id of each global vertex.
    """
    off, nbr, eidx = csr_undirected(n, src, dst)
    deg = np.diff(off)
    idxs = range(sel["v_off"].size - 1) if which is None else list(which)
    local = threading.local()

    def one(i):
        verts = sel["vid"][sel["v_off"][i]:sel["v_off"][i + 1]].astype(np.int64)
        mark = getattr(local, "mark", None)
        if mark is None:
            mark = local.mark = np.full(n, -1, dtype=np.int32)
        mark[verts] = np.arange(verts.size, dtype=np.int32)
        starts, lens = off[verts], deg[verts]
        tot = int(lens.sum())
        rep = np.repeat(np.arange(verts.size, dtype=np.int32), lens)
        idx = np.arange(tot, dtype=np.int64) + np.repeat(starts - (np.cumsum(lens) - lens), lens)
        lw = mark[nbr[idx]]
        keep = lw > rep
        mark[verts] = -1
        return verts, rep[keep].astype(np.int64), lw[keep].astype(np.int64), eidx[idx[keep]]

    parts = _map(one, idxs)
    count = len(parts)
    v_off = np.zeros(count + 1, dtype=np.int64)
    e_off = np.zeros(count + 1, dtype=np.int64)
    v_off[1:] = np.cumsum([p[0].size for p in parts])
    e_off[1:] = np.cumsum([p[1].size for p in parts])
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return {
        "v_off": v_off,
        "e_off": e_off,
        "src": cat([p[1] + v_off[i] for i, p in enumerate(parts)], np.uint32),
        "dst": cat([p[2] + v_off[i] for i, p in enumerate(parts)], np.uint32),
        "eid": cat([p[3] for p in parts], np.uint32),
        "vid": cat([p[0] for p in parts], np.uint32),
    }


def ego_induce_torch(n: int, src, dst, sel, device="cuda", chunk=1 << 27):
    """ego_induce for all ego nets of `sel`, computed with torch on `device`;
    the same arrays as ego_induce, as torch tensors (int64 offsets, int32
    vertex / edge ids holding the uint32 values).

    Membership is a bitmap per ego net (count x n bits); the members'
    adjacency lists are expanded in chunks of about `chunk` entries.
    """
    import torch
    dev = torch.device(device)
    s = torch.from_numpy(np.asarray(src, dtype=np.int64)).to(dev)
    d = torch.from_numpy(np.asarray(dst, dtype=np.int64)).to(dev)
    m = s.numel()
    a = torch.cat([s, d])
    b = torch.cat([d, s])
    e = torch.cat([torch.arange(m, device=dev), torch.arange(m, device=dev)])
    order = torch.argsort(a * n + b)
    a, b, e = a[order], b[order], e[order]
    deg = torch.bincount(a, minlength=n)
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(deg, 0)
    del a, order
    v_off = torch.from_numpy(np.asarray(sel["v_off"], dtype=np.int64)).to(dev)
    vid = torch.from_numpy(np.asarray(sel["vid"], dtype=np.int64)).to(dev)
    G = v_off.numel() - 1
    N = vid.numel()
    gid = torch.repeat_interleave(torch.arange(G, device=dev), v_off[1:] - v_off[:-1])
    words = (n + 63) // 64
    bitmap = torch.zeros(G * words, dtype=torch.int64, device=dev)
    one = torch.ones(1, dtype=torch.int64, device=dev)
    bitmap.scatter_reduce_(0, gid * words + (vid >> 6), torch.bitwise_left_shift(one, vid & 63), reduce="sum")
    key = gid * n + vid  # sorted: members sorted within each ego net, nets in order
    lens = deg[vid]
    ends = torch.cumsum(lens, 0)
    out_src, out_dst, out_eid = [], [], []
    lo = 0
    total = int(ends[-1].item()) if N else 0
    while lo < N:
        start_e = int(ends[lo - 1].item()) if lo else 0
        hi = int(torch.searchsorted(ends, torch.tensor([start_e + chunk], device=dev)).item())
        hi = max(hi, lo + 1)
        hi = min(hi, N)
        ln = lens[lo:hi]
        rep = torch.repeat_interleave(torch.arange(lo, hi, device=dev), ln)
        excl = torch.cumsum(ln, 0) - ln
        pos = torch.arange(rep.numel(), device=dev) - torch.repeat_interleave(excl, ln) + off[vid[rep]]
        w = b[pos]
        g = gid[rep]
        bit = torch.bitwise_right_shift(bitmap[g * words + (w >> 6)], w & 63) & 1
        keep = (bit == 1) & (w > vid[rep])
        rk, wk, gk = rep[keep], w[keep], g[keep]
        out_src.append(rk)
        out_dst.append(torch.searchsorted(key, gk * n + wk))
        out_eid.append(e[pos[keep]])
        lo = hi
        del rep, excl, pos, w, g, bit, keep
    src_g = torch.cat(out_src) if out_src else torch.zeros(0, dtype=torch.int64, device=dev)
    dst_g = torch.cat(out_dst) if out_dst else torch.zeros(0, dtype=torch.int64, device=dev)
    eid_g = torch.cat(out_eid) if out_eid else torch.zeros(0, dtype=torch.int64, device=dev)
    e_cnt = torch.bincount(gid[src_g], minlength=G) if src_g.numel() else torch.zeros(G, dtype=torch.int64, device=dev)
    e_off = torch.zeros(G + 1, dtype=torch.int64, device=dev)
    e_off[1:] = torch.cumsum(e_cnt, 0)
    del bitmap
    return {"v_off": v_off, "e_off": e_off, "src": src_g.to(torch.int32), "dst": dst_g.to(torch.int32),
            "eid": eid_g.to(torch.int32), "vid": vid.to(torch.int32), "total_adjacency": total}


def ego_nets(n: int, src, dst, count: int, smin: int, smax: int, seed: int):
    """ego_select followed by ego_induce (all ego nets, on the CPU)."""
    return ego_induce(n, src, dst, ego_select(n, src, dst, count, smin, smax, seed))


def bfs_induced(n: int, src, dst, start: int, min_edges: int):
    """Add vertices in BFS order from ``start`` until the induced edge count
    reaches ``min_edges``; return (vertex ids, local src, local dst, parent eid).
    """
    off, nbr, _ = csr_undirected(n, src, dst)
    inset = np.zeros(n, dtype=bool)
    order = []
    seen = np.zeros(n, dtype=bool)
    seen[start] = True
    edges = 0
    head = 0
    queue = [start]
    while head < len(queue) and edges < min_edges:
        x = queue[head]
        head += 1
        nb = nbr[off[x]:off[x + 1]]
        edges += int(inset[nb].sum())
        inset[x] = True
        order.append(x)
        for y in nb:
            if not seen[y]:
                seen[y] = True
                queue.append(int(y))
    verts = np.asarray(sorted(order), dtype=np.int64)
    local = np.full(n, -1, dtype=np.int64)
    local[verts] = np.arange(verts.size)
    s64 = np.asarray(src, dtype=np.int64)
    d64 = np.asarray(dst, dtype=np.int64)
    keep = inset[s64] & inset[d64]
    eid = np.nonzero(keep)[0]
    return (verts.astype(np.uint32), local[s64[keep]].astype(np.uint32),
            local[d64[keep]].astype(np.uint32), eid.astype(np.uint32))


class Graph:
    """A generated uncertain signed graph: n, src, dst and k (or p)."""

    def __init__(self, name, n, src, dst, k=None, p=None, meta=None):
        self.name = name
        self.n = int(n)
        self.src = np.ascontiguousarray(src, dtype=np.uint32)
        self.dst = np.ascontiguousarray(dst, dtype=np.uint32)
        self.k = None if k is None else np.ascontiguousarray(k, dtype=np.uint32)
        self.p = None if p is None else np.ascontiguousarray(p, dtype=np.float32)
        self.meta = dict(meta or {})

    @property
    def m(self):
        return int(self.src.size)


def config_graph(name: str, seed: int = 1) -> Graph:
    """The five workload graphs, by the name they are known by elsewhere.

    er2k      -- G(n=2,000, m=20,000), k ~ U{0..65536}.
    cl1m      -- Chung-Lu n=1e6, gamma=2.1, mean degree 20, max 50,000,
                 P+ ~ Beta(0.5, 0.5) quantised to 16 bits.
    rmat22    -- R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05),
                 P+ ~ 0.5 Beta(8,2) + 0.5 Beta(2,8) quantised.
    rmat20    -- R-MAT scale 20, edge factor 16, k ~ U{0..65536}.
    cl4m      -- Chung-Lu n=4e6, gamma=2.3, mean degree 20, max 50,000,
                 p ~ U[0,1] float32.
    Small variants for tests and profiling: ``rmat<s>`` for any scale s
    (k ~ U{0..65536}, as rmat20), ``rmat<s>m`` with rmat22's Beta mixture;
    ``cl<n>`` is not provided (use chung_lu directly).
    """
    if name == "er2k":
        n = 2000
        s, d = er_graph(n, 20000, seed)
        return Graph(name, n, s, d, k=k_uniform(20000, seed + 1000))
    if name == "cl1m":
        n = 1_000_000
        s, d = chung_lu(n, 2.1, 20.0, 50_000.0, seed)
        k = quantise(p_beta(s.size, 0.5, 0.5, seed + 1000))
        return Graph(name, n, s, d, k=k)
    if name == "cl4m":
        n = 4_000_000
        s, d = chung_lu(n, 2.3, 20.0, 50_000.0, seed)
        return Graph(name, n, s, d, p=p_uniform_f32(s.size, seed + 1000))
    if name.startswith("rmat"):
        mixture = name.endswith("m")
        scale = int(name[4:-1] if mixture else name[4:])
        s, d = rmat(scale, 16, 0.57, 0.19, 0.19, seed)
        if scale == 22 or mixture:
            k = quantise(p_beta_mixture(s.size, seed + 1000))
        else:
            k = k_uniform(s.size, seed + 1000)
        return Graph(name, 1 << scale, s, d, k=k)
    raise KeyError(name)
