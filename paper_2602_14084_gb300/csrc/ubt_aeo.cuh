// ubt_aeo.cuh -- the edge iteration of Alg. 2 in Absolute Edge Order.
//
// Alg. 2 visits the edges in Absolute Edge Order (Def. AEO: a(e) = |P+ - 0.5|
// descending, ties by (min id, max id)), stops at the first edge with
// a(e) < a(t) (Lemma 2) and, for edge e = (u, v), intersects the neighbours
// of u and of v reached through edges after e in the order whose value passes
// Lemma 3's cutoff.  Each triangle is found once, from its first edge in the
// order (the edge with the largest |q|).  In the fixed-point form
// (|q| = |32768 - k| = 65536 a(e), L = ceil((2t - 1) 2^45)):
//   Lemma 2   edge e can be in a classified triangle only if |q_e| 2^30 >= L
//   Lemma 3   a partner edge f of e (after e) only if |q_f| |q_e|^2 >= L: the
//             third edge is after e too, so |q| <= |q_e| for both partners
//             and |P| <= |q_f| |q_e|^2.
//
// GPU layout.  The undirected rows hold every edge at x sorted by |q|
// descending then neighbour id -- for one row this is exactly Absolute Edge
// Order -- so "after e" is "at a later position of the row" and both cutoffs
// are prefixes.  Edge e = x-y is handled by x (the endpoint with the longer
// row), whose row prefix is a hash table (kept in shared memory, in chunks if
// it is longer than one table); y's row is streamed from the position after
// e (its mirror position + 1) to the Lemma 3 cutoff, and a hit w counts only
// if x-w lies after e in x's row and passes the cutoff.  All edges are
// processed in parallel: the order only decides which edge finds a triangle.
#pragma once

#include "ubt_traverse.cuh"

namespace ubt {

struct AeoArgs {
  const uint32_t* uptr;       // undirected rows
  const uint64_t* uadj;
  const uint32_t* umir;       // mirror position of every entry
  const uint32_t* apair_ptr;  // edges owned by x: [apair_ptr[x], apair_ptr[x + 1])
  const uint64_t* apairs;     // streamed endpoint | position of the edge in x's row << 32
  const uint32_t* alist;      // owners: block tasks first, then warp tasks
  uint32_t n_owners;
  uint32_t n_block;           // owners handled by a whole block
  uint32_t wcap;              // per-warp table slots
  uint32_t n;
  uint32_t m2;                // 2m, the number of row entries
  Scratch* sc;
  uint32_t cap;               // table slots (power of two)
  uint32_t unit;              // edges a warp takes at a time
  int64_t L;                  // pruning level (0: none)
};

// One lane's edge e = x-y: its row-x position and value, the Lemma 3
// multiplier q_e^2, and the streamed range [vs, vs + dv) of y's row.
struct AeoPair {
  uint32_t x, y, pe, qe, vs, dv;
  int64_t cut;
  bool ok;
};

__device__ __forceinline__ AeoPair aeo_pair(const AeoArgs& a, uint32_t x, uint32_t idx, bool in, uint32_t tab_begin,
                                            uint32_t tab_end, uint32_t rs, uint32_t tlen) {
  AeoPair pr;
  pr.x = x;
  pr.ok = in;
  pr.vs = 0;
  pr.dv = 0;
  pr.cut = 0;
  const uint64_t d = in ? a.apairs[idx] : 0ull;
  pr.y = (uint32_t)d;
  pr.pe = (uint32_t)(d >> 32);
  if (pr.ok && (pr.pe >= a.m2 || pr.y >= a.n)) {
    guard_fail(a.sc, kGuardList, x);
    pr.ok = false;
  }
  // no table entry after e in this chunk: nothing to find
  if (pr.pe + 1 >= tab_end) pr.ok = false;
  const uint64_t e = pr.ok ? a.uadj[pr.pe] : 0ull;
  pr.qe = adj_valbits(e);
  const int64_t aq = qabs(pr.qe);
  pr.cut = aq * aq;
  if (a.L > 0 && aq * (1ll << 30) < a.L) pr.ok = false;  // Lemma 2
  // the table entries that can pair with e lie in x's row after e and before
  // Lemma 3's cutoff: skip the chunk when it holds none of them
  if (pr.ok && a.L > 0 && rs + prune_prefix(a.uadj + rs, tlen, pr.cut, a.L) <= tab_begin) pr.ok = false;
  if (pr.ok) {
    const uint32_t ys = a.uptr[pr.y], ye = a.uptr[pr.y + 1];
    const uint32_t start = a.umir[pr.pe] + 1;
    if (ye < ys || ye > a.m2 || start < ys || start > ye) {
      guard_fail(a.sc, kGuardList, pr.y);
      pr.ok = false;
    } else {
      const uint32_t end = a.L > 0 ? ys + prune_prefix(a.uadj + ys, ye - ys, pr.cut, a.L) : ye;  // Lemma 3
      pr.vs = start;
      pr.dv = end > start ? end - start : 0u;
    }
  }
  return pr;
}

// A hit w of the table counts only if x-w lies after e in x's row and passes
// Lemma 3's cutoff.
__device__ __forceinline__ bool aeo_keep(const AeoArgs& a, uint32_t pw, uint32_t qxw, uint32_t pe, int64_t cut) {
  return pw > pe && (a.L == 0 || qabs(qxw) * cut >= a.L);
}

// One warp streams the ranges of up to 32 edges (one per lane).
template <class V>
__device__ __forceinline__ void aeo_probe(const AeoArgs& a, V& vis, const Table& t, const AeoPair& pr) {
  const int lane = (int)lane_id();
  const uint64_t* __restrict__ adj = a.uadj;
  Scratch* const sc = a.sc;
  const uint32_t dv = pr.ok ? pr.dv : 0u;
  constexpr uint32_t kLong = 48;
  unsigned longm = __ballot_sync(kFull, dv >= kLong);
  while (longm) {
    const int j = __ffs(longm) - 1;
    longm &= longm - 1;
    const uint32_t xj = __shfl_sync(kFull, pr.x, j);
    const uint32_t yj = __shfl_sync(kFull, pr.y, j);
    const uint32_t vsj = __shfl_sync(kFull, pr.vs, j);
    const uint32_t dvj = __shfl_sync(kFull, dv, j);
    const uint32_t qj = __shfl_sync(kFull, pr.qe, j);
    const uint32_t pj = __shfl_sync(kFull, pr.pe, j);
    const long long cj = __shfl_sync(kFull, (long long)pr.cut, j);
    for (uint32_t off = 0; off < dvj; off += 64) {
      uint64_t e[2];
#pragma unroll
      for (int s = 0; s < 2; s++) {
        const uint32_t i = off + 32 * s + lane;
        e[s] = i < dvj ? adj[vsj + i] : 0ull;
      }
#pragma unroll
      for (int s = 0; s < 2; s++) {
        const uint32_t i = off + 32 * s + lane;
        uint32_t qxw = 0, pxw = 0;
        bool hit = i < dvj && table_find<true>(t, adj_col(e[s]), qxw, pxw, sc);
        hit = hit && aeo_keep(a, pxw, qxw, pj, cj);
        if (off + 32 * s < dvj) vis.step(hit, xj, yj, adj_col(e[s]), qj, qxw, adj_valbits(e[s]), pj, pxw, vsj + i);
      }
    }
  }
  // short ranges: concatenated so that every lane probes one entry per step
  const uint32_t ds = dv >= kLong ? 0u : dv;
  uint32_t incl = ds;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t excl = incl - ds;
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t f = base + lane;
    const bool act = f < total;
    int j = 0;
#pragma unroll
    for (int b = 16; b > 0; b >>= 1) {
      const uint32_t tj = __shfl_sync(kFull, incl, j + b - 1);
      if (tj <= f) j += b;
    }
    j = j > 31 ? 31 : j;
    const uint32_t vsj = __shfl_sync(kFull, pr.vs, j);
    const uint32_t exj = __shfl_sync(kFull, excl, j);
    const uint32_t xj = __shfl_sync(kFull, pr.x, j);
    const uint32_t yj = __shfl_sync(kFull, pr.y, j);
    const uint32_t qj = __shfl_sync(kFull, pr.qe, j);
    const uint32_t pj = __shfl_sync(kFull, pr.pe, j);
    const long long cj = __shfl_sync(kFull, (long long)pr.cut, j);
    const uint32_t pos = vsj + (f - exj);
    const uint64_t e = act ? adj[pos] : 0ull;
    uint32_t qxw = 0, pxw = 0;
    bool hit = act && table_find<true>(t, adj_col(e), qxw, pxw, sc);
    hit = hit && aeo_keep(a, pxw, qxw, pj, cj);
    vis.step(hit, xj, yj, adj_col(e), qj, qxw, adj_valbits(e), pj, pxw, pos);
  }
}

// One block handles owner x: its row's Lemma 2 prefix goes into the table,
// chunk by chunk when it is longer than one table; for every chunk, every
// edge x owns streams its range.
template <class V>
__device__ void aeo_task(const AeoArgs& a, V& vis, uint32_t x, uint32_t* tab, uint32_t* s_misc) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (x >= a.n) {
    if (tid == 0) guard_fail(a.sc, kGuardVertex, x);
    return;
  }
  const uint32_t rs = a.uptr[x], re = a.uptr[x + 1];
  const uint32_t ps = a.apair_ptr[x], pend = a.apair_ptr[x + 1];
  if (re < rs || re > a.m2 || pend < ps || pend - ps > re - rs) {
    if (tid == 0) guard_fail(a.sc, kGuardList, x);
    return;
  }
  const uint32_t np = pend - ps;
  if (tid == 0) s_misc[0] = a.L > 0 ? prune_prefix(a.uadj + rs, re - rs, 1ll << 30, a.L) : re - rs;  // Lemma 2
  __syncthreads();
  const uint32_t tlen = s_misc[0];
  __syncthreads();
  if (tlen < 2 || np == 0) return;
  const uint32_t chunk = a.cap / 4;
  const uint32_t nw = blockDim.x >> 5;
  vis.task_begin(x);
  for (uint32_t c0 = 0; c0 < tlen; c0 += chunk) {
    const uint32_t c1 = min(tlen, c0 + chunk);
    const uint32_t slots = slots_for(c1 - c0);
    const Table t = make_table(tab, a.cap, slots);
    for (uint32_t i = tid; i < slots; i += blockDim.x) t.key[i] = kEmpty;
    if (tid == 0) s_misc[1] = 0;
    __syncthreads();
    for (uint32_t i = c0 + tid; i < c1; i += blockDim.x) {
      const uint64_t e = a.uadj[rs + i];
      table_insert(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
    }
    __syncthreads();
    while (true) {
      uint32_t c = 0, cnt = 0;
      if (lane == 0) {
        const uint32_t seen = *(volatile uint32_t*)&s_misc[1];
        const uint32_t rem = seen < np ? np - seen : 0u;
        const uint32_t want = max(1u, min(a.unit, rem / (2 * nw)));
        c = atomicAdd(&s_misc[1], want);
        cnt = c < np ? min(want, np - c) : 0u;
      }
      c = __shfl_sync(kFull, c, 0);
      cnt = __shfl_sync(kFull, cnt, 0);
      if (cnt == 0) break;
      aeo_probe<V>(a, vis, t, aeo_pair(a, x, ps + c + lane, (uint32_t)lane < cnt, rs + c0, rs + c1, rs, tlen));
    }
    __syncthreads();
  }
  vis.task_end(x);
  __syncthreads();
}

// One warp handles owner x (a row of at most 128 entries): one table.
template <class V>
__device__ void aeo_warp_task(const AeoArgs& a, V& vis, uint32_t x, uint32_t* wtab) {
  const int lane = (int)lane_id();
  if (x >= a.n) {
    if (lane == 0) guard_fail(a.sc, kGuardVertex, x);
    return;
  }
  const uint32_t rs = a.uptr[x], re = a.uptr[x + 1];
  const uint32_t ps = a.apair_ptr[x], pend = a.apair_ptr[x + 1];
  if (re < rs || re > a.m2 || pend < ps || pend - ps > re - rs) {
    if (lane == 0) guard_fail(a.sc, kGuardList, x);
    return;
  }
  const uint32_t np = pend - ps;
  const uint32_t tlen = a.L > 0 ? prune_prefix(a.uadj + rs, re - rs, 1ll << 30, a.L) : re - rs;  // Lemma 2
  if (tlen < 2 || np == 0) return;
  const uint32_t slots = slots_for(tlen);
  if (slots > a.wcap) {
    if (lane == 0) guard_fail(a.sc, kGuardTable, x);
    return;
  }
  const Table t = make_table(wtab, a.wcap, slots);
  for (uint32_t i = lane; i < slots; i += 32) t.key[i] = kEmpty;
  __syncwarp();
  for (uint32_t i = lane; i < tlen; i += 32) {
    const uint64_t e = a.uadj[rs + i];
    table_insert(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
  }
  __syncwarp();
  vis.task_begin(x);
  for (uint32_t cs = 0; cs < np; cs += 32)
    aeo_probe<V>(a, vis, t, aeo_pair(a, x, ps + cs + lane, (uint32_t)lane < np - cs, rs, rs + tlen, rs, tlen));
  vis.task_end(x);
  __syncwarp();
}

template <class V>
__global__ void __launch_bounds__(512, 2) k_aeo(AeoArgs a, typename V::P p) {
  extern __shared__ __align__(16) char smem[];
  __shared__ uint32_t s_misc[4];
  V vis(p, smem);
  vis.block_init();
  __syncthreads();
  uint32_t* tab = (uint32_t*)(smem + ((V::smem_bytes((int)blockDim.x) + 15) / 16) * 16);
  while (true) {
    if (threadIdx.x == 0) s_misc[2] = (uint32_t)atomicAdd(&a.sc->task[0], 1ull);
    __syncthreads();
    const uint32_t task = s_misc[2];
    __syncthreads();
    if (task >= a.n_block) break;
    aeo_task(a, vis, a.alist[task], tab, s_misc);
  }
  __syncthreads();  // the block tables are free: the region becomes per-warp tables
  const int lane = threadIdx.x & 31;
  uint32_t* wtab = tab + (size_t)(threadIdx.x >> 5) * a.wcap * 3;
  while (true) {
    unsigned long long t0 = 0;
    if (lane == 0) t0 = atomicAdd(&a.sc->task[1], 1ull);
    t0 = __shfl_sync(kFull, t0, 0);
    if (t0 >= (unsigned long long)(a.n_owners - a.n_block)) break;
    aeo_warp_task(a, vis, a.alist[a.n_block + (uint32_t)t0], wtab);
  }
  __syncthreads();
  vis.block_end();
}

// The same iteration on a graph with the edge index (UBT_OPT_EDGE_INDEX):
// no owner tables.  Edge e = u-v has two windows of candidate partners, u's
// row after e and v's row after e, each up to Lemma 3's cutoff; the shorter
// one is streamed and, for each entry s-w of it, the closing edge o-w (o the
// other endpoint) is looked up in the index.  It counts when o-w lies after
// e in o's row -- |q_ow| < |q_e|, or equal and w > s, the row order being
// Absolute Edge Order -- and passes the cutoff, exactly the conditions the
// table form tests through row positions.  Warps take 32 edges at a time;
// long windows are streamed by the whole warp, short ones concatenated.
// Visitors without CSR positions only (the positions of o-w are not known).
struct AeoIxArgs {
  const uint32_t* uptr;
  const uint64_t* uadj;
  const uint32_t* uepos;      // 2m: [2e + side] position of edge e in its endpoints' rows
  const uint4* eslots;        // edge index
  uint64_t emask;
  int eshift;
  uint32_t n, m, m2;
  Scratch* sc;
  int64_t L;
};

__device__ __forceinline__ bool aeo_ix_find(const AeoIxArgs& a, uint32_t o, uint32_t w, uint32_t& val) {
  const int r = edge_index_lookup(a.eslots, a.emask, a.eshift, o, w, val);
  if (r < 0) guard_fail(a.sc, kGuardFind, o);
  return r > 0;
}

// entry s-w of the streamed window: the closing edge o-w, if it exists, lies
// after e in o's row and passes Lemma 3
__device__ __forceinline__ bool aeo_ix_keep(const AeoIxArgs& a, uint32_t s, uint32_t w, uint32_t qow, int64_t aq,
                                            int64_t cut) {
  const int64_t oq = qabs(qow);
  return (oq < aq || (oq == aq && w > s)) && (a.L == 0 || oq * cut >= a.L);
}

// Two lanes' worth of lookups at once: both home slots are read before
// either is examined (at most a quarter of the slots are used, so nearly
// every lookup ends there); the rare longer probe continues alone.
__device__ __forceinline__ void aeo_ix_hit2(const AeoIxArgs& a, const bool (&act)[2], const uint32_t (&o)[2],
                                            const uint32_t (&s)[2], const uint32_t (&w)[2], const int64_t (&aq)[2],
                                            const int64_t (&cut)[2], bool (&hit)[2], uint32_t (&qow)[2]) {
  uint64_t k[2], h[2];
  uint4 sl[2];
#pragma unroll
  for (int i = 0; i < 2; i++) {
    k[i] = edge_index_key(o[i], w[i]);
    h[i] = edge_index_home(k[i], a.eshift);
    sl[i] = (act[i] && w[i] != o[i]) ? a.eslots[h[i]] : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
  }
#pragma unroll
  for (int i = 0; i < 2; i++) {
    hit[i] = false;
    qow[i] = 0;
    if (!act[i] || w[i] == o[i]) continue;
    const uint64_t key = ((uint64_t)sl[i].y << 32) | sl[i].x;
    bool found = key == k[i];
    if (found) {
      qow[i] = sl[i].z;
    } else if (key != kEdgeIndexEmpty) {  // the home slot holds another edge: probe on
      found = aeo_ix_find(a, o[i], w[i], qow[i]);
    }
    hit[i] = found && aeo_ix_keep(a, s[i], w[i], qow[i], aq[i], cut[i]);
  }
}

template <class V>
__global__ void __launch_bounds__(512, 2) k_aeo_index(AeoIxArgs a, typename V::P p) {
  static_assert(!V::kPos, "the index form knows no CSR position of the closing edge");
  extern __shared__ __align__(16) char smem[];
  V vis(p, smem);
  vis.block_init();
  __syncthreads();
  const int lane = (int)lane_id();
  while (true) {
    unsigned long long e0 = 0;
    if (lane == 0) e0 = atomicAdd(&a.sc->task[0], 32ull);
    e0 = __shfl_sync(kFull, e0, 0);
    if (e0 >= a.m) break;
    const uint64_t e = e0 + (uint64_t)lane;
    bool ok = e < a.m;
    uint32_t o = 0, sv = 0, qe = 0, vs = 0, dv = 0;
    int64_t aq = 0, cut = 0;
    if (ok) {
      const uint32_t p0 = a.uepos[2 * e], p1 = a.uepos[2 * e + 1];
      if (p0 >= a.m2 || p1 >= a.m2) {
        guard_fail(a.sc, kGuardList, (uint32_t)e);
        ok = false;
      } else {
        const uint64_t ea = a.uadj[p0];
        const uint32_t u = adj_col(a.uadj[p1]), v = adj_col(ea);  // p0 lies in u's row, p1 in v's
        qe = adj_valbits(ea);
        aq = qabs(qe);
        cut = aq * aq;
        if (u >= a.n || v >= a.n || (a.L > 0 && aq * (1ll << 30) < a.L)) {  // Lemma 2 on e
          if (u >= a.n || v >= a.n) guard_fail(a.sc, kGuardVertex, (uint32_t)e);
          ok = false;
        } else {
          const uint32_t ue = a.uptr[u + 1], ve = a.uptr[v + 1];
          const uint32_t cu = a.L > 0 ? a.uptr[u] + prune_prefix(a.uadj + a.uptr[u], ue - a.uptr[u], cut, a.L) : ue;
          const uint32_t cv = a.L > 0 ? a.uptr[v] + prune_prefix(a.uadj + a.uptr[v], ve - a.uptr[v], cut, a.L) : ve;
          const uint32_t lu = cu > p0 + 1 ? cu - (p0 + 1) : 0u, lv = cv > p1 + 1 ? cv - (p1 + 1) : 0u;
          if (lu <= lv) { sv = u; o = v; vs = p0 + 1; dv = lu; }
          else { sv = v; o = u; vs = p1 + 1; dv = lv; }
        }
      }
    }
    if (!ok) dv = 0;
    // long windows: the whole warp, one window at a time
    constexpr uint32_t kLong = 48;
    unsigned longm = __ballot_sync(kFull, dv >= kLong);
    while (longm) {
      const int j = __ffs(longm) - 1;
      longm &= longm - 1;
      const uint32_t oj = __shfl_sync(kFull, o, j), sj = __shfl_sync(kFull, sv, j);
      const uint32_t vsj = __shfl_sync(kFull, vs, j), dvj = __shfl_sync(kFull, dv, j);
      const uint32_t qj = __shfl_sync(kFull, qe, j);
      const long long aqj = __shfl_sync(kFull, (long long)aq, j), cj = __shfl_sync(kFull, (long long)cut, j);
      for (uint32_t off = 0; off < dvj; off += 64) {
        bool act[2], hit[2];
        uint32_t oo[2], ss[2], ww[2], qow[2];
        int64_t aa[2], cc[2];
        uint64_t ew[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const uint32_t i = off + 32 * u + lane;
          act[u] = i < dvj;
          ew[u] = act[u] ? a.uadj[vsj + i] : 0ull;
          oo[u] = oj;
          ss[u] = sj;
          ww[u] = adj_col(ew[u]);
          aa[u] = aqj;
          cc[u] = cj;
        }
        aeo_ix_hit2(a, act, oo, ss, ww, aa, cc, hit, qow);
#pragma unroll
        for (int u = 0; u < 2; u++)
          if (u == 0 || off + 32 < dvj)
            vis.step(hit[u], oj, sj, ww[u], qj, qow[u], adj_valbits(ew[u]), 0u, 0u, vsj + off + 32 * u + lane);
      }
    }
    // short windows: concatenated, one entry per lane per step
    const uint32_t ds = dv >= kLong ? 0u : dv;
    uint32_t incl = ds;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - ds;
    for (uint32_t base = 0; base < total; base += 64) {
      bool act[2], hit[2];
      uint32_t oo[2], ss[2], ww[2], qq[2], pos[2], qow[2];
      int64_t aa[2], cc[2];
      uint64_t ew[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const uint32_t f = base + 32 * u + lane;
        act[u] = f < total;
        int j = 0;
#pragma unroll
        for (int b = 16; b > 0; b >>= 1) {
          const uint32_t tj = __shfl_sync(kFull, incl, j + b - 1);
          if (tj <= f) j += b;
        }
        j = j > 31 ? 31 : j;
        const uint32_t vsj = __shfl_sync(kFull, vs, j), exj = __shfl_sync(kFull, excl, j);
        oo[u] = __shfl_sync(kFull, o, j);
        ss[u] = __shfl_sync(kFull, sv, j);
        qq[u] = __shfl_sync(kFull, qe, j);
        aa[u] = __shfl_sync(kFull, (long long)aq, j);
        cc[u] = __shfl_sync(kFull, (long long)cut, j);
        pos[u] = vsj + (f - exj);
        ew[u] = act[u] ? a.uadj[pos[u]] : 0ull;
        ww[u] = adj_col(ew[u]);
      }
      aeo_ix_hit2(a, act, oo, ss, ww, aa, cc, hit, qow);
#pragma unroll
      for (int u = 0; u < 2; u++)
        if (u == 0 || base + 32 < total)
          vis.step(hit[u], oo[u], ss[u], ww[u], qq[u], qow[u], adj_valbits(ew[u]), 0u, 0u, pos[u]);
    }
  }
  __syncthreads();
  vis.block_end();
}

namespace {

template <class V>
ubt_status launch_aeo(const ubt_graph* g, int64_t L, const typename V::P& p, cudaStream_t s) {
  if (!g->uptr) return UBT_ERR_UNSUPPORTED;
  const Tuning& T = tuning();
  if constexpr (!V::kPos) {
    if (g->eslots && T.edge_index != 0) {
      AeoIxArgs a;
      a.uptr = g->uptr;
      a.uadj = g->uadj;
      a.uepos = g->uepos;
      a.eslots = g->eslots;
      a.emask = (uint64_t)g->eh_slots - 1;
      a.eshift = g->eh_shift;
      a.n = (uint32_t)g->n;
      a.m = (uint32_t)g->m;
      a.m2 = (uint32_t)(2 * g->m);
      a.sc = g->scratch;
      a.L = L;
      UBT_CUDA(cudaMemsetAsync(a.sc, 0, kScratchHeader / 2, s));
      if (g->m == 0) return UBT_OK;
      const int threads = 512;
      const size_t smem = (size_t)((V::smem_bytes(threads) + 15) / 16) * 16;
      UBT_CUDA(cudaFuncSetAttribute(k_aeo_index<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      UBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_aeo_index<V>, threads, smem));
      if (per_sm < 1) return UBT_ERR_INVALID_ARG;
      per_sm = (int)std::min<int64_t>(per_sm, std::max<int64_t>(1, T.blocks_per_sm));
      k_aeo_index<V><<<g->sm_count * per_sm, threads, smem, s>>>(a, p);
      UBT_CUDA(cudaGetLastError());
      return UBT_OK;
    }
  }
  AeoArgs a;
  a.uptr = g->uptr;
  a.uadj = g->uadj;
  a.umir = g->umir;
  a.apair_ptr = g->apair_ptr;
  a.apairs = g->apairs;
  a.alist = g->alist;
  a.n_owners = (uint32_t)g->n_aowners;
  a.n_block = (uint32_t)g->n_ablock;
  a.wcap = (uint32_t)table_slots(std::min<int64_t>(128, std::max<int64_t>(g->max_udeg, 2)));
  a.n = (uint32_t)g->n;
  a.m2 = (uint32_t)(2 * g->m);
  a.sc = g->scratch;
  a.cap = (uint32_t)std::min<int64_t>(table_slots(std::max<int64_t>(g->max_udeg, 2)),
                                      std::max<int64_t>(64, T.smem_table_max));
  a.unit = (uint32_t)std::min<int64_t>(32, std::max<int64_t>(1, T.block_unit));
  a.L = L;
  UBT_CUDA(cudaMemsetAsync(a.sc, 0, kScratchHeader / 2, s));
  if (a.n_owners == 0) return UBT_OK;
  const int threads = 512;
  const size_t tables = std::max<size_t>((size_t)a.cap, (size_t)(threads / 32) * a.wcap) * 3 * 4;
  const size_t smem = (size_t)((V::smem_bytes(threads) + 15) / 16) * 16 + tables;
  UBT_CUDA(cudaFuncSetAttribute(k_aeo<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  UBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_aeo<V>, threads, smem));
  if (per_sm < 1) return UBT_ERR_INVALID_ARG;
  per_sm = (int)std::min<int64_t>(per_sm, std::max<int64_t>(1, T.blocks_per_sm));
  k_aeo<V><<<g->sm_count * per_sm, threads, smem, s>>>(a, p);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}

}  // namespace

}  // namespace ubt
