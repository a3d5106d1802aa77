// ubt_traverse.cuh -- the triangle traversal every query runs.
//
// Forward edge iteration under Node Order (Alg. 1, Sec. 4): triangle {u,v,w}
// with u < v < w in Node Order is found exactly once, from u, as
// w in N>(u) n N>(v) for v in N>(u).  Each forward edge (u, v) is a "pair";
// its work is to probe every w of N>(v) against N>(u).
//
// GPU layout of that loop (one persistent kernel, four kinds of task):
//   * N>(u) is loaded into an open-addressing hash table (neighbour -> edge
//     value, CSR position) in shared memory: 4-slot buckets read with one
//     16-byte load, at most 1/4 full, so nearly every probe is one load.
//   * The pairs of a task are handed to one warp 32 at a time.  The lists N>(v)
//     are streamed with coalesced 8-byte loads: long lists one after another
//     by the whole warp, short lists concatenated ("flattened") so that every
//     lane has an entry; two entries per lane are in flight at once.  Each
//     entry w is probed in u's table; a hit is a triangle and goes to the
//     visitor with the three edge values and CSR positions.
//   * Task kinds, by |N>(u)|:
//       giant   longer than the shared-memory table: whole block, table in a
//               per-block slice of global memory
//       hub     whole block, shared table, warps take `unit` pairs at a time
//       medium  one warp, its own table
//       short   segments: the short lists, concatenated in vertex order, are
//               cut into runs of 32 pairs; one warp takes a run, puts every
//               list the run touches into one table and probes with the row
//               of each pair's u (CSR positions identify the row)
//   * Probability pruning (FIXED graphs, level L > 0): every list is sorted by
//     |q| descending, so the entries that cannot reach |P| >= L are suffixes:
//       u's table and pairs:   |q_e| * qmax(u) * 2^15 >= L   (Lemma 2: each
//                              edge bounds the product of the triangle)
//       v's list for pair u-v: |q_vw| * |q_uv| * qmax(u) >= L (order-free form
//                              of Lemma 3: the other two edges bound it)
//     qmax(u) is the largest |q| in N>(u) (its first entry).
//
// Visitors implement: smem_bytes(threads) (shared memory they need) /
// block_init / task_begin / step (called by all 32 lanes of a warp, converged,
// once per probed entry with a hit flag) / task_end / block_end.  Visitors
// with kBatched also take the hits of U probes of one long list at once
// (steps<U>: hit flags and the u-w and v-w edge values; u-v is common).
#pragma once

#include <algorithm>

#include "ubt_internal.cuh"

// launch bounds of the traversal kernels: at most UBT_LB_THREADS threads per
// block, at least UBT_LB_MINB resident blocks per SM (caps the registers)
#ifndef UBT_LB_THREADS
#define UBT_LB_THREADS 512
#endif
#ifndef UBT_LB_MINB
#define UBT_LB_MINB 1
#endif

namespace ubt {

struct TravArgs {
  const uint32_t* row_ptr;
  const uint64_t* adj;
  const uint32_t* giant_list;
  const uint32_t* hub_list;
  const uint32_t* med_list;
  const uint32_t* seg_row;     // short lists' vertices, in vertex order
  const uint32_t* seg_start;   // start of each short list in the concatenation
  const uint32_t* seg_first;   // first short list touching each 32-pair segment (kEmpty: none)
  uint32_t n_giant, n_hub, n_med, n_srows, n_segs;
  uint32_t n, m;            // vertices, edges (bounds of the self-checks)
  Scratch* sc;              // task counters (zeroed before launch)
  uint32_t* gtab;           // giant tables: gtab_blocks x gtab_slots x 3 words
  uint32_t gtab_slots;      // power of two
  uint32_t gtab_blocks;
  uint32_t hub_slots;       // shared-memory hub table capacity (power of two)
  uint32_t warp_slots;      // per-warp table capacity (power of two)
  uint32_t unit;            // pairs per warp step in block tasks
  uint32_t batch;           // warp tasks / segments taken per grab
  int64_t L;                // prune level, 0 = none
};

__device__ __forceinline__ uint32_t hash_slot(uint32_t w, int shift) { return (w * 0x9E3779B1u) >> shift; }

// Self-checks record the first violated invariant in Scratch::guard and skip
// the offending access: 1 probe limit (find), 2 probe limit (insert),
// 3 neighbour id >= n, 4 list offsets out of order or past m, 5 table larger
// than its region.
enum : unsigned long long { kGuardFind = 1, kGuardInsert = 2, kGuardVertex = 3, kGuardList = 4, kGuardTable = 5 };
static __device__ __noinline__ void guard_fail(Scratch* sc, unsigned long long code, unsigned long long info) {
  atomicCAS(&sc->guard, 0ull, (code << 56) | (info & ((1ull << 56) - 1)));
}

__device__ __forceinline__ int64_t qabs(uint32_t valbits) {
  const int32_t q = (int32_t)valbits;
  return q < 0 ? -(int64_t)q : (int64_t)q;
}

// first index in [0, len) of a |q|-descending list whose |q| * c < L (len if none)
__device__ __forceinline__ uint32_t prune_prefix(const uint64_t* __restrict__ row, uint32_t len, int64_t c, int64_t L) {
  if (len == 0) return 0;
  if (qabs(adj_valbits(row[len - 1])) * c >= L) return len;
  if (qabs(adj_valbits(row[0])) * c < L) return 0;
  uint32_t lo = 0, hi = len - 1;  // row[lo] passes, row[hi] fails
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (qabs(adj_valbits(row[mid])) * c >= L) lo = mid; else hi = mid;
  }
  return hi;
}

// Hash table: key = neighbour id, val = edge value bits, pos = CSR position,
// in buckets of 4 slots (one 16-byte load reads a bucket's keys); at most 1/4
// of the slots are used, so nearly every lookup ends in its home bucket.
struct Table {
  uint32_t* key;
  uint32_t* val;
  uint32_t* pos;
  uint32_t bmask;  // buckets - 1
  int shift;
};

__device__ __forceinline__ Table make_table(uint32_t* base, uint32_t cap, uint32_t slots) {
  Table t;
  t.key = base;
  t.val = base + cap;
  t.pos = base + 2 * cap;
  const uint32_t nb = slots >> 2;
  t.bmask = nb - 1;
  t.shift = 32 - (31 - __clz((int)nb));
  return t;
}

// slots for a list: a power of two >= 4x its entries (min 32, i.e. 8 buckets)
__device__ __forceinline__ uint32_t slots_for(uint32_t entries) {
  uint32_t s = 32;
  while (s < 4 * entries) s <<= 1;
  return s;
}

// A bucket with a free slot ends every probe sequence, and there are more
// buckets than entries, so both loops end within bmask + 1 buckets; the limit
// is a self-check.  Slots of a bucket are taken in order (first free slot).
__device__ __forceinline__ void table_insert(const Table& t, uint32_t w, uint32_t val, uint32_t pos, Scratch* sc) {
  uint32_t b = hash_slot(w, t.shift);
  for (uint32_t it = 0; it <= t.bmask; it++) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (atomicCAS(&t.key[4 * b + i], kEmpty, w) == kEmpty) {
        t.val[4 * b + i] = val;
        t.pos[4 * b + i] = pos;
        return;
      }
    }
    b = (b + 1) & t.bmask;
  }
  guard_fail(sc, kGuardInsert, w);
}

// Find w in the table.  kRow: the table holds several rows (a segment) and
// only entries whose CSR position lies in [rs, rs + rlen) -- the row of this
// pair's u -- count.  kPos: also return the entry's CSR position.
//
// Inserts take the first free slot of a bucket and nothing is ever removed,
// so a bucket's used slots are a prefix and a bucket has room iff its last
// slot is empty; a key missing from a bucket with room is absent.  With at
// most 1/4 of the slots used, nearly every lookup reads one bucket and takes
// no branch.
template <bool kRow, bool kPos>
__device__ __forceinline__ bool table_find(const Table& t, uint32_t w, uint32_t rs, uint32_t rlen, uint32_t& val,
                                           uint32_t& pos, Scratch* sc) {
  uint32_t b = hash_slot(w, t.shift);
  if (!kRow) {
    const uint4 k = reinterpret_cast<const uint4*>(t.key)[b];
    const bool m0 = k.x == w, m1 = k.y == w, m2 = k.z == w, m3 = k.w == w;
    bool hit = m0 | m1 | m2 | m3;
    uint32_t s = 4 * b + (m0 ? 0u : (m1 ? 1u : (m2 ? 2u : 3u)));
    if (!hit && k.w != kEmpty) {  // the home bucket is full: continue in the next ones
      bool ended = false;
      for (uint32_t it = 1; it <= t.bmask; it++) {
        b = (b + 1) & t.bmask;
        const uint4 kk = reinterpret_cast<const uint4*>(t.key)[b];
        const bool n0 = kk.x == w, n1 = kk.y == w, n2 = kk.z == w, n3 = kk.w == w;
        if (n0 | n1 | n2 | n3) {
          hit = true;
          s = 4 * b + (n0 ? 0u : (n1 ? 1u : (n2 ? 2u : 3u)));
          ended = true;
          break;
        }
        if (kk.w == kEmpty) {
          ended = true;
          break;
        }
      }
      if (!ended) guard_fail(sc, kGuardFind, w);
    }
    if (hit) {
      val = t.val[s];
      if (kPos) pos = t.pos[s];
    }
    return hit;
  }
  for (uint32_t it = 0; it <= t.bmask; it++) {
    const uint4 k = reinterpret_cast<const uint4*>(t.key)[b];
    unsigned mt = (k.x == w ? 1u : 0u) | (k.y == w ? 2u : 0u) | (k.z == w ? 4u : 0u) | (k.w == w ? 8u : 0u);
    while (mt) {
      const uint32_t s = 4 * b + (__ffs(mt) - 1);
      mt &= mt - 1;
      const uint32_t p = t.pos[s];
      if (p - rs < rlen) {
        val = t.val[s];
        pos = p;
        return true;
      }
    }
    if (k.w == kEmpty) return false;
    b = (b + 1) & t.bmask;
  }
  guard_fail(sc, kGuardFind, w);
  return false;
}

// Per-lane description of one pair (u, v) handed to probe_pairs.
struct Pair {
  uint32_t u, v, puv, quv;  // vertices, CSR position and value of the u-v edge
  uint32_t urs, ulen;       // u's row as seen by the table (for row matching)
  int64_t qmax;             // largest |q| of u's list (pruning)
  bool ok;
};

// The whole warp probes entries [off, off + 32 U) of one long list N>(v),
// U entries per lane, all loads issued before the probes.  kAll: all 32 U
// entries exist (no bounds tests).
template <class V, bool kRow, int U, bool kAll>
__device__ __forceinline__ void long_steps(const uint64_t* __restrict__ adj, Scratch* sc, V& vis, const Table& t,
                                           int lane, uint32_t uj, uint32_t vj, uint32_t vsj, uint32_t dvj,
                                           uint32_t qj, uint32_t pj, uint32_t rsj, uint32_t rlj, uint32_t off) {
  uint64_t e[U];
#pragma unroll
  for (int s = 0; s < U; s++) {
    const uint32_t i = off + 32 * s + lane;
    e[s] = (kAll || i < dvj) ? adj[vsj + i] : 0ull;
  }
  if constexpr (V::kBatched) {
    // all U probes first, then the visitor takes their hits together
    bool hit[U];
    uint32_t quw[U], qvw[U];
#pragma unroll
    for (int s = 0; s < U; s++) {
      const uint32_t i = off + 32 * s + lane;
      uint32_t puw = 0;
      quw[s] = 0;
      qvw[s] = adj_valbits(e[s]);
      hit[s] = (kAll || i < dvj) && table_find<kRow, false>(t, adj_col(e[s]), rsj, rlj, quw[s], puw, sc);
    }
    vis.template steps<U>(hit, qj, quw, qvw);
  } else {
#pragma unroll
    for (int s = 0; s < U; s++) {
      const uint32_t i = off + 32 * s + lane;
      uint32_t quw = 0, puw = 0;
      const bool hit = (kAll || i < dvj) && table_find<kRow, V::kPos>(t, adj_col(e[s]), rsj, rlj, quw, puw, sc);
      if (kAll || off + 32 * s < dvj)
        vis.step(hit, uj, vj, adj_col(e[s]), qj, quw, adj_valbits(e[s]), pj, puw, vsj + i);
    }
  }
}

// One warp probes the lists of up to 32 pairs (one per lane, `ok` lanes).
// kRow: the table is a segment table (entries must belong to the pair's row).
template <class V, bool kRow>
__device__ __forceinline__ void probe_pairs(const TravArgs& a, V& vis, const Table& t, const Pair& pr) {
  const int lane = (int)lane_id();
  const uint64_t* __restrict__ adj = a.adj;
  Scratch* const sc = a.sc;
  uint32_t vs = 0, dv = 0;
  if (pr.ok) {
    if (pr.v < a.n) {
      vs = a.row_ptr[pr.v];
      const uint32_t ve = a.row_ptr[pr.v + 1];
      if (ve >= vs && ve <= a.m) {
        dv = ve - vs;
        if (a.L > 0) dv = prune_prefix(a.adj + vs, dv, qabs(pr.quv) * pr.qmax, a.L);
      } else {
        guard_fail(a.sc, kGuardList, pr.v);
      }
    } else {
      guard_fail(a.sc, kGuardVertex, pr.v);
    }
  }
  // long lists: one at a time, the whole warp streams it, up to four entries per lane
  constexpr uint32_t kLong = 48;
  unsigned longm = __ballot_sync(kFull, dv >= kLong);
  while (longm) {
    const int j = __ffs(longm) - 1;
    longm &= longm - 1;
    const uint32_t uj = __shfl_sync(kFull, pr.u, j);
    const uint32_t vj = __shfl_sync(kFull, pr.v, j);
    const uint32_t vsj = __shfl_sync(kFull, vs, j);
    const uint32_t dvj = __shfl_sync(kFull, dv, j);
    const uint32_t qj = __shfl_sync(kFull, pr.quv, j);
    const uint32_t pj = __shfl_sync(kFull, pr.puv, j);
    const uint32_t rsj = __shfl_sync(kFull, pr.urs, j);
    const uint32_t rlj = __shfl_sync(kFull, pr.ulen, j);
    uint32_t off = 0;
    while (dvj - off >= 128) {
      long_steps<V, kRow, 4, true>(adj, sc, vis, t, lane, uj, vj, vsj, dvj, qj, pj, rsj, rlj, off);
      off += 128;
    }
    while (off < dvj) {
      long_steps<V, kRow, 2, false>(adj, sc, vis, t, lane, uj, vj, vsj, dvj, qj, pj, rsj, rlj, off);
      off += 64;
    }
  }
  // short lists: concatenated so that every lane probes one entry per half-step
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
    uint32_t f[2], jj[2];
    bool act[2];
    uint64_t e[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
      f[s] = base + 32 * s + lane;
      act[s] = f[s] < total;
      // owner: number of lanes whose inclusive end is <= f
      int j = 0;
#pragma unroll
      for (int b = 16; b > 0; b >>= 1) {
        const uint32_t tj = __shfl_sync(kFull, incl, j + b - 1);
        if (tj <= f[s]) j += b;
      }
      jj[s] = (uint32_t)(j > 31 ? 31 : j);
      const uint32_t vsj = __shfl_sync(kFull, vs, jj[s]);
      const uint32_t exj = __shfl_sync(kFull, excl, jj[s]);
      e[s] = act[s] ? adj[vsj + (f[s] - exj)] : 0ull;
      f[s] = vsj + (f[s] - exj);  // now the CSR position of the entry
    }
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const int j = (int)jj[s];
      const uint32_t rsj = __shfl_sync(kFull, pr.urs, j);
      const uint32_t rlj = __shfl_sync(kFull, pr.ulen, j);
      uint32_t quw = 0, puw = 0;
      const bool hit = act[s] && table_find<kRow, V::kPos>(t, adj_col(e[s]), rsj, rlj, quw, puw, sc);
      const uint32_t uj = __shfl_sync(kFull, pr.u, j);
      const uint32_t vj = __shfl_sync(kFull, pr.v, j);
      const uint32_t qj = __shfl_sync(kFull, pr.quv, j);
      const uint32_t pj = __shfl_sync(kFull, pr.puv, j);
      if (s == 0 || base + 32 < total)
        vis.step(hit, uj, vj, adj_col(e[s]), qj, quw, adj_valbits(e[s]), pj, puw, f[s]);
    }
  }
}

// Pair of this lane among the pairs [cs, cs + cnt) of a single-row table.
__device__ __forceinline__ Pair row_pair(const TravArgs& a, uint32_t u, int64_t qmax, uint32_t cs, uint32_t cnt) {
  const int lane = (int)lane_id();
  Pair pr;
  pr.u = u;
  pr.urs = 0;
  pr.ulen = ~0u;
  pr.qmax = qmax;
  pr.ok = (uint32_t)lane < cnt;
  pr.puv = cs + lane;
  const uint64_t e = pr.ok ? a.adj[pr.puv] : 0ull;
  pr.v = adj_col(e);
  pr.quv = adj_valbits(e);
  return pr;
}

// u's list length after pruning (and qmax); identical in every calling thread
__device__ __forceinline__ uint32_t pruned_len(const TravArgs& a, uint32_t rs, uint32_t len, int64_t& qmax) {
  qmax = 0;
  if (a.L > 0 && len > 0) {
    qmax = qabs(adj_valbits(a.adj[rs]));
    return prune_prefix(a.adj + rs, len, qmax * 32768, a.L);
  }
  return len;
}

// A whole block handles u; `tab` is shared memory (hub) or a global slice (giant).
template <class V>
__device__ __forceinline__ void block_task(const TravArgs& a, V& vis, uint32_t u, uint32_t* tab, uint32_t cap,
                                           uint32_t* s_misc) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (u >= a.n) {
    if (tid == 0) guard_fail(a.sc, kGuardVertex, u);
    return;
  }
  const uint32_t rs = a.row_ptr[u], re = a.row_ptr[u + 1];
  if (re < rs || re > a.m) {
    if (tid == 0) guard_fail(a.sc, kGuardList, u);
    return;
  }
  int64_t qmax = 0;
  if (tid == 0) s_misc[0] = pruned_len(a, rs, re - rs, qmax);
  __syncthreads();
  const uint32_t len = s_misc[0];
  if (a.L > 0 && len > 0) qmax = qabs(adj_valbits(a.adj[rs]));
  const uint32_t slots = slots_for(len);
  if (len == 0 || slots > cap) {
    if (len && tid == 0) guard_fail(a.sc, kGuardTable, u);
    __syncthreads();
    return;
  }
  const Table t = make_table(tab, cap, slots);
  for (uint32_t i = tid; i < slots; i += blockDim.x) t.key[i] = kEmpty;
  if (tid == 0) s_misc[1] = 0;
  __syncthreads();
  for (uint32_t i = tid; i < len; i += blockDim.x) {
    const uint64_t e = a.adj[rs + i];
    table_insert(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
  }
  __syncthreads();
  vis.task_begin(u);
  // warps take pairs `unit` at a time, fewer as the list runs out, so that
  // they reach the closing barrier at about the same time
  const uint32_t nw = blockDim.x >> 5;
  while (true) {
    uint32_t c = 0, cnt = 0;
    if (lane == 0) {
      const uint32_t seen = *(volatile uint32_t*)&s_misc[1];
      const uint32_t rem = seen < len ? len - seen : 0u;
      const uint32_t want = max(1u, min(a.unit, rem / (2 * nw)));
      c = atomicAdd(&s_misc[1], want);
      cnt = c < len ? min(want, len - c) : 0u;
    }
    c = __shfl_sync(kFull, c, 0);
    cnt = __shfl_sync(kFull, cnt, 0);
    if (cnt == 0) break;
    probe_pairs<V, false>(a, vis, t, row_pair(a, u, qmax, rs + c, cnt));
  }
  vis.task_end(u);
  __syncthreads();
}

// One warp handles u (a medium list).
template <class V>
__device__ __forceinline__ void warp_task(const TravArgs& a, V& vis, uint32_t u, uint32_t* tab) {
  const int lane = (int)lane_id();
  if (u >= a.n) {
    if (lane == 0) guard_fail(a.sc, kGuardVertex, u);
    return;
  }
  const uint32_t rs = a.row_ptr[u], re = a.row_ptr[u + 1];
  if (re < rs || re > a.m) {
    if (lane == 0) guard_fail(a.sc, kGuardList, u);
    return;
  }
  int64_t qmax = 0;
  const uint32_t len = pruned_len(a, rs, re - rs, qmax);
  if (len == 0) return;
  const uint32_t slots = slots_for(len);
  if (slots > a.warp_slots) {
    if (lane == 0) guard_fail(a.sc, kGuardTable, u);
    return;
  }
  const Table t = make_table(tab, a.warp_slots, slots);
  for (uint32_t i = lane; i < slots; i += 32) t.key[i] = kEmpty;
  __syncwarp();
  for (uint32_t i = lane; i < len; i += 32) {
    const uint64_t e = a.adj[rs + i];
    table_insert(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
  }
  __syncwarp();
  vis.task_begin(u);
  for (uint32_t cs = 0; cs < len; cs += 32)
    probe_pairs<V, false>(a, vis, t, row_pair(a, u, qmax, rs + cs, min(32u, len - cs)));
  vis.task_end(u);
  __syncwarp();
}

// One warp handles segment k: pairs [32k, 32k + 32) of the concatenated short lists.
template <class V>
__device__ __forceinline__ void segment_task(const TravArgs& a, V& vis, uint32_t k, uint32_t* tab) {
  const int lane = (int)lane_id();
  const uint32_t r0 = a.seg_first[k];
  if (r0 == kEmpty) return;
  const uint32_t sp0 = 32 * k, sp1 = sp0 + 32;
  // lane i describes short list r0 + i, if that list starts before the segment ends
  const uint32_t r = r0 + lane;
  uint32_t ss = 0xFFFFFFFFu, u = 0, rs = 0, raw = 0, len = 0;
  int64_t qmax = 0;
  bool row = false;
  if (r < a.n_srows && a.seg_start[r] < sp1) {
    ss = a.seg_start[r];
    u = a.seg_row[r];
    if (u < a.n) {
      rs = a.row_ptr[u];
      const uint32_t re = a.row_ptr[u + 1];
      if (re >= rs && re <= a.m) {
        row = true;
        raw = re - rs;
      } else {
        guard_fail(a.sc, kGuardList, u);
      }
    } else {
      guard_fail(a.sc, kGuardVertex, u);
    }
  }
  if (__ballot_sync(kFull, row) == 0) return;
  if (row) len = pruned_len(a, rs, raw, qmax);
  // table: every entry of the touched lists (their pruned prefixes)
  const uint32_t tl = row ? len : 0u;
  uint32_t incl = tl;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t slots = slots_for(total);
  if (slots > a.warp_slots) {
    if (lane == 0) guard_fail(a.sc, kGuardTable, k);
    return;
  }
  const Table t = make_table(tab, a.warp_slots, slots);
  for (uint32_t i = lane; i < slots; i += 32) t.key[i] = kEmpty;
  __syncwarp();
  const uint32_t excl = incl - tl;
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t f = base + lane;
    int j = 0;
#pragma unroll
    for (int b = 16; b > 0; b >>= 1) {
      const uint32_t tj = __shfl_sync(kFull, incl, j + b - 1);
      if (tj <= f) j += b;
    }
    j = j > 31 ? 31 : j;
    const uint32_t rsj = __shfl_sync(kFull, rs, j);
    const uint32_t exj = __shfl_sync(kFull, excl, j);
    if (f < total) {
      const uint32_t p = rsj + (f - exj);
      const uint64_t e = a.adj[p];
      table_insert(t, adj_col(e), adj_valbits(e), p, a.sc);
    }
  }
  __syncwarp();
  // the segment's pairs: lane e takes position sp0 + e of the concatenation;
  // its list is the last one that starts at or before that position
  const uint32_t sp = sp0 + lane;
  int j = 0;  // number of lists starting at or before sp
#pragma unroll
  for (int b = 16; b > 0; b >>= 1) {
    const uint32_t sj = __shfl_sync(kFull, ss, j + b - 1);
    if (sj <= sp) j += b;
  }
  const bool have = j > 0;
  j = have ? j - 1 : 0;
  const uint32_t ssj = __shfl_sync(kFull, ss, j);
  const uint32_t rsj = __shfl_sync(kFull, rs, j);
  const uint32_t rawj = __shfl_sync(kFull, raw, j);
  Pair pr;
  pr.u = __shfl_sync(kFull, u, j);
  pr.urs = rsj;
  pr.ulen = __shfl_sync(kFull, len, j);
  pr.qmax = __shfl_sync(kFull, qmax, j);
  const bool rowj = __shfl_sync(kFull, (int)row, j) != 0;
  const uint32_t off = sp - ssj;
  // a pair outside its list's pruned prefix cannot be in a classified triangle
  pr.ok = have && rowj && off < rawj && off < pr.ulen;
  pr.puv = rsj + off;
  const uint64_t e = pr.ok ? a.adj[pr.puv] : 0ull;
  pr.v = adj_col(e);
  pr.quv = adj_valbits(e);
  const uint32_t u0 = __shfl_sync(kFull, u, 0);
  vis.task_begin(u0);
  probe_pairs<V, true>(a, vis, t, pr);
  vis.task_end(u0);
  __syncwarp();
}

// The traversal runs as two persistent kernels, so that each can have the
// block size and shared memory its tasks need: the block kernel (giant and
// hub lists, one large table per block) and the warp kernel (medium lists and
// short-list segments, one small table per warp).
enum : int { kBlockTasks = 1, kWarpTasks = 2 };

// Persistent traversal kernel body.  Shared memory: [visitor bytes][tables].
template <class V, int kPhases>
__device__ void traverse(const TravArgs& a, V& vis, char* smem_tables) {
  __shared__ uint32_t s_misc[4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t* tab = (uint32_t*)smem_tables;
  if (kPhases & kBlockTasks) {
    // giant lists, tables in global memory (first gtab_blocks blocks)
    if (blockIdx.x < a.gtab_blocks) {
      uint32_t* gt = a.gtab + (size_t)blockIdx.x * a.gtab_slots * 3;
      while (true) {
        if (tid == 0) s_misc[2] = (uint32_t)atomicAdd(&a.sc->task[0], 1ull);
        __syncthreads();
        const uint32_t task = s_misc[2];
        __syncthreads();
        if (task >= a.n_giant) break;
        block_task(a, vis, a.giant_list[task], gt, a.gtab_slots, s_misc);
      }
    }
    // hub lists, block-wide shared-memory tables
    while (true) {
      if (tid == 0) s_misc[2] = (uint32_t)atomicAdd(&a.sc->task[1], 1ull);
      __syncthreads();
      const uint32_t task = s_misc[2];
      __syncthreads();
      if (task >= a.n_hub) break;
      block_task(a, vis, a.hub_list[task], tab, a.hub_slots, s_misc);
    }
  }
  if (kPhases & kWarpTasks) {
    uint32_t* wtab = tab + (size_t)wid * a.warp_slots * 3;
    // medium lists, one warp each
    while (true) {
      unsigned long long t0 = 0;
      if (lane == 0) t0 = atomicAdd(&a.sc->task[2], (unsigned long long)a.batch);
      t0 = __shfl_sync(kFull, t0, 0);
      if (t0 >= a.n_med) break;
      const uint32_t t1 = (uint32_t)min((unsigned long long)a.n_med, t0 + a.batch);
      for (uint32_t t = (uint32_t)t0; t < t1; t++) warp_task(a, vis, a.med_list[t], wtab);
    }
    // segments of short lists
    while (true) {
      unsigned long long t0 = 0;
      if (lane == 0) t0 = atomicAdd(&a.sc->task[3], (unsigned long long)a.batch);
      t0 = __shfl_sync(kFull, t0, 0);
      if (t0 >= a.n_segs) break;
      const uint32_t t1 = (uint32_t)min((unsigned long long)a.n_segs, t0 + a.batch);
      for (uint32_t t = (uint32_t)t0; t < t1; t++) segment_task(a, vis, t, wtab);
    }
  }
  __syncthreads();
  vis.block_end();
}

// Shared memory of one block of a traversal kernel: visitor bytes + tables.
inline size_t traverse_smem_bytes(const TravArgs& a, int phases, int threads, int vis_smem) {
  const size_t vis_bytes = (size_t)((vis_smem + 15) / 16) * 16;
  size_t tables = 0;
  if (phases & kBlockTasks) tables = std::max(tables, (size_t)a.hub_slots * 3 * 4);
  if (phases & kWarpTasks) tables = std::max(tables, (size_t)(threads / 32) * a.warp_slots * 3 * 4);
  return vis_bytes + tables;
}

namespace {

// Launch bounds per kernel: the block kernel runs 512-thread blocks, the warp
// kernel 128-thread blocks, and a visitor's register cap (V::kRegCap) sets how
// many of them must fit on one SM (65536 registers).
template <class V, int kPhases>
struct Bounds {
  static constexpr int kThreads = (kPhases & kBlockTasks) ? UBT_LB_THREADS : 128;
  static constexpr int kMinBlocks = 65536 / (kThreads * V::kRegCap) > 0 ? 65536 / (kThreads * V::kRegCap) : 1;
};

template <class V, int kPhases>
__global__ void __launch_bounds__(Bounds<V, kPhases>::kThreads, Bounds<V, kPhases>::kMinBlocks)
    k_traverse(TravArgs a, typename V::P p) {
  extern __shared__ __align__(16) char smem[];
  V vis(p, smem);
  vis.block_init();
  __syncthreads();
  traverse<V, kPhases>(a, vis, smem + ((V::smem_bytes((int)blockDim.x) + 15) / 16) * 16);
}

template <class V, int kPhases>
ubt_status launch_phase(const ubt_graph* g, const TravArgs& a, const typename V::P& p, int threads, cudaStream_t s) {
  const Tuning& T = tuning();
  threads = (int)std::min<int64_t>(Bounds<V, kPhases>::kThreads, std::max<int64_t>(64, threads / 32 * 32));
  const size_t smem = traverse_smem_bytes(a, kPhases, threads, V::smem_bytes(threads));
  UBT_CUDA(cudaFuncSetAttribute(k_traverse<V, kPhases>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  UBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse<V, kPhases>, threads, smem));
  if (per_sm < 1) return UBT_ERR_INVALID_ARG;
  per_sm = (int)std::min<int64_t>(per_sm, std::max<int64_t>(1, T.blocks_per_sm));
  k_traverse<V, kPhases><<<g->sm_count * per_sm, threads, smem, s>>>(a, p);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}

// One traversal: the task counters in a.sc are cleared, then the block kernel
// (if the graph has giant or hub lists) and the warp kernel (if it has medium
// lists or segments) run one after the other on `s`.
template <class V>
ubt_status launch_traversal(const ubt_graph* g, const TravArgs& a, const typename V::P& p, cudaStream_t s) {
  const Tuning& T = tuning();
  UBT_CUDA(cudaMemsetAsync(a.sc, 0, kScratchHeader / 2, s));
  if (a.n_giant + a.n_hub > 0) {
    const ubt_status st = launch_phase<V, kBlockTasks>(g, a, p, (int)T.block_threads, s);
    if (st != UBT_OK) return st;
  }
  if (a.n_med + a.n_segs > 0) {
    const ubt_status st = launch_phase<V, kWarpTasks>(g, a, p, (int)T.warp_threads, s);
    if (st != UBT_OK) return st;
  }
  return UBT_OK;
}

}  // namespace

}  // namespace ubt
