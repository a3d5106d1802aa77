// ubt_traverse.cuh -- the triangle traversal every query runs.
//
// Forward edge iteration under Node Order (Alg. 1, Sec. 4): triangle {u,v,w}
// with u < v < w in Node Order is found exactly once, from its pair (u, v),
// as w in N>(u) n N>(v).  Every forward edge is one pair.  Alg. 1 streams
// N>(v) through a table of N>(u); streaming N>(u) through a table of N>(v)
// intersects the same two lists, and the build gives each pair to the
// endpoint (its "owner" x) whose list is the longer, so that the shorter list
// N>(s) is streamed (the pair partition of ubt_build.cu).
//
// GPU layout of that loop (two persistent kernels, three kinds of task):
//   * N>(x) is loaded into an open-addressing hash table (neighbour -> edge
//     value, CSR position) in shared memory: 4-slot buckets read with one
//     16-byte load, at most 1/4 full, so nearly every probe is one load.
//   * The pairs of x are handed to one warp 32 at a time.  The lists N>(s)
//     are streamed with coalesced 8-byte loads: long lists one after another
//     by the whole warp, short lists concatenated ("flattened") so that every
//     lane has an entry.  Each entry w is probed in x's table; a hit is a
//     triangle and goes to the visitor with the three edge values and CSR
//     positions.
//   * Task kinds, by owner:
//       giant   list longer than the shared-memory table: whole block, table
//               in a per-block slice of global memory
//       hub     long list or heavy streamed work: whole block, shared table,
//               warps take `unit` pairs at a time
//       medium  the rest: one warp, its own table
//   * Probability pruning (FIXED graphs, level L > 0): every list is sorted by
//     |q| descending, so the entries that cannot reach |P| >= L are suffixes:
//       table and pairs:   |q_e| * 2^30 >= L              (Lemma 2: the other
//                                                         two factors are at
//                                                         most 2^15)
//       streamed N>(s):    |q_sw| * |q_xs| * qmax(x) >= L (order-free form of
//                                                         Lemma 3: the other
//                                                         two edges bound it)
//     qmax(x) is the largest |q| in N>(x) (its first entry).
//
// Visitors implement: smem_bytes(threads) (shared memory they need) /
// block_init / task_begin / step (called by all 32 lanes of a warp, converged,
// once per probed entry with a hit flag) / task_end / block_end.  Visitors
// with kBatched also take the hits of U probes of one long list at once
// (steps<U>: hit flags and the two streamed-edge values; the pair's is common).
// A visitor sees a triangle as (x, s, w): the pair edge x-s, the table edge
// x-w and the streamed edge s-w; under pull x is the later vertex of the pair,
// so visitors treat the three edges symmetrically (they all do).  A visitor
// may also define probed(n): after each batch of at most 32 pairs the whole
// warp calls it with n >= the number of entries the batch probed (the same n
// in every lane).
#pragma once

#include <algorithm>
#include <type_traits>
#include <utility>

#include "ubt_internal.cuh"

// launch bounds of the traversal kernels: at most UBT_LB_THREADS threads per
// block, at least UBT_LB_MINB resident blocks per SM (caps the registers)
#ifndef UBT_LB_THREADS
#define UBT_LB_THREADS 512
#endif
#ifndef UBT_LB_MINB
#define UBT_LB_MINB 1
#endif
// entries per lane of a full chunk of a long list (4 or 8)
#ifndef UBT_LONG_U
#define UBT_LONG_U 4
#endif

namespace ubt {

struct TravArgs {
  const uint32_t* row_ptr;
  const uint64_t* adj;
  const uint32_t* pair_ptr;    // pairs of owner x: [pair_ptr[x], pair_ptr[x + 1])
  const uint64_t* pairs;       // streamed vertex | CSR position of the pair edge << 32
  const uint32_t* giant_list;
  const uint32_t* hub_list;
  const uint32_t* med_list;
  uint32_t n_giant, n_hub, n_med;
  uint32_t n, m;            // vertices, edges (bounds of the self-checks)
  Scratch* sc;              // task counters (zeroed before launch)
  uint32_t* gtab;           // giant tables: gtab_blocks x gtab_slots x 3 words
  uint32_t gtab_slots;      // power of two
  uint32_t gtab_blocks;
  uint32_t hub_slots;       // shared-memory hub table capacity (power of two)
  uint32_t warp_slots;      // per-warp table capacity (power of two)
  uint32_t unit;            // pairs per warp step in block tasks
  uint32_t batch;           // warp tasks taken per grab
  uint32_t long_min;        // streamed lists at least this long take the whole-warp path
  uint32_t long_tail;       // 1: a long list's last < 64 entries join the concatenated short lists
  int64_t L;                // prune level, 0 = none
  uint32_t light_prune;     // 1: streamed lists kept whole (owner tables and pairs still pruned)
};

// At a low prune level (2t - 1 < 1/10) a streamed list rarely loses more than
// a few entries, and streaming them costs less than the load of the list's
// last entry that decides whether any go.  The kept entries form no triangle
// with |P| >= L, so every query answers the same.
inline uint32_t light_prune_for(int64_t L) { return L > 0 && L < (1ll << 45) / 10 ? 1u : 0u; }

__device__ __forceinline__ uint32_t hash_slot(uint32_t w, int shift) { return (w * 0x9E3779B1u) >> shift; }

// visitors with a probed(n) member are told how many entries each batch probed
template <class V, class = void>
struct HasProbed : std::false_type {};
template <class V>
struct HasProbed<V, std::void_t<decltype(std::declval<V&>().probed(0u))>> : std::true_type {};

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
template <bool kPos = true>
__device__ __forceinline__ void table_insert(const Table& t, uint32_t w, uint32_t val, uint32_t pos, Scratch* sc) {
  uint32_t b = hash_slot(w, t.shift);
  for (uint32_t it = 0; it <= t.bmask; it++) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (atomicCAS(&t.key[4 * b + i], kEmpty, w) == kEmpty) {
        t.val[4 * b + i] = val;
        if (kPos) t.pos[4 * b + i] = pos;
        return;
      }
    }
    b = (b + 1) & t.bmask;
  }
  guard_fail(sc, kGuardInsert, w);
}

// Find w in the table (kPos: also return the entry's CSR position).
//
// Inserts take the first free slot of a bucket and nothing is ever removed,
// so a bucket's used slots are a prefix and a bucket has room iff its last
// slot is empty; a key missing from a bucket with room is absent.  With at
// most 1/4 of the slots used, nearly every lookup reads one bucket and takes
// no branch.
template <bool kPos>
__device__ __forceinline__ bool table_find(const Table& t, uint32_t w, uint32_t& val, uint32_t& pos, Scratch* sc) {
  uint32_t b = hash_slot(w, t.shift);
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

// Words of table memory per slot: visitors that need no CSR position keep
// only keys and values (8 bytes a slot), which lets more warp tables share
// an SM's shared memory.
template <bool kPos>
struct TableWords {
  static constexpr uint32_t kWords = kPos ? 3u : 2u;
};
// 32-bit words of shared memory a table of `slots` slots takes for visitor V
template <class V>
__host__ __device__ constexpr uint32_t table_words(uint32_t slots) {
  return slots * TableWords<V::kPos>::kWords;
}

// table_find for the 32 converged lanes of a warp (every lane calls it; a
// lane without an entry passes any key and ignores the result): the search
// past a full home bucket -- rare, at most 1/4 of the slots are used -- is
// entered by the whole warp only when some lane needs it, and the value is
// read from the slot the bucket search ends at, hit or not, so that the
// common case runs without a divergent branch.
template <bool kPos>
__device__ __forceinline__ bool table_find_warp(const Table& t, uint32_t w, uint32_t& val, uint32_t& pos,
                                                Scratch* sc) {
  uint32_t b = hash_slot(w, t.shift);
  const uint4 k = reinterpret_cast<const uint4*>(t.key)[b];
  const bool m0 = k.x == w, m1 = k.y == w, m2 = k.z == w, m3 = k.w == w;
  bool hit = m0 | m1 | m2 | m3;
  uint32_t s = 4 * b + (m0 ? 0u : (m1 ? 1u : (m2 ? 2u : 3u)));
  const bool more = !hit && k.w != kEmpty;
  if (__any_sync(kFull, more)) {
    if (more) {  // the home bucket is full: continue in the next ones
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
  }
  val = t.val[s];
  if (kPos) pos = t.pos[s];
  return hit;
}

// Per-lane description of one pair handed to probe_pairs: owner x (its list
// is the table), streamed vertex s, CSR position and value of the x-s edge.
struct Pair {
  uint32_t x, s, pe, qe;
  int64_t qmax;  // largest |q| of x's list (pruning)
  bool ok;
};

// The whole warp probes entries [off, off + 32 U) of one long list N>(v),
// U entries per lane, all loads issued before the probes.  kAll: all 32 U
// entries exist (no bounds tests).
template <class V, int U, bool kAll>
__device__ __forceinline__ void long_steps(const uint64_t* __restrict__ adj, Scratch* sc, V& vis, const Table& t,
                                           int lane, uint32_t uj, uint32_t vj, uint32_t vsj, uint32_t dvj,
                                           uint32_t qj, uint32_t pj, uint32_t off) {
  uint64_t e[U];
  const uint64_t* __restrict__ row = adj + vsj + off + lane;
#pragma unroll
  for (int s = 0; s < U; s++) e[s] = (kAll || off + 32 * s + lane < dvj) ? row[32 * s] : 0ull;
  if constexpr (V::kBatched) {
    // all U probes first, then the visitor takes their hits together
    bool hit[U];
    uint32_t quw[U], qvw[U];
#pragma unroll
    for (int s = 0; s < U; s++) {
      uint32_t puw = 0;
      qvw[s] = adj_valbits(e[s]);
      const bool f = table_find_warp<false>(t, adj_col(e[s]), quw[s], puw, sc);
      hit[s] = (kAll || off + 32 * s + lane < dvj) && f;
    }
    vis.template steps<U>(hit, qj, quw, qvw);
  } else {
#pragma unroll
    for (int s = 0; s < U; s++) {
      const uint32_t i = off + 32 * s + lane;
      uint32_t quw = 0, puw = 0;
      const bool f = table_find_warp<V::kPos>(t, adj_col(e[s]), quw, puw, sc);
      const bool hit = (kAll || i < dvj) && f;
      if (kAll || off + 32 * s < dvj)
        vis.step(hit, uj, vj, adj_col(e[s]), qj, quw, adj_valbits(e[s]), pj, puw, vsj + i);
    }
  }
}

// One warp probes the lists of up to 32 pairs (one per lane, `ok` lanes).
template <class V>
__device__ __forceinline__ void probe_pairs(const TravArgs& a, V& vis, const Table& t, const Pair& pr) {
  const int lane = (int)lane_id();
  const uint64_t* __restrict__ adj = a.adj;
  Scratch* const sc = a.sc;
  uint32_t vs = 0, dv = 0;
  if (pr.ok) {
    if (pr.s < a.n) {
      vs = a.row_ptr[pr.s];
      const uint32_t ve = a.row_ptr[pr.s + 1];
      if (ve >= vs && ve <= a.m) {
        dv = ve - vs;
        if (a.L > 0 && !a.light_prune) dv = prune_prefix(a.adj + vs, dv, qabs(pr.qe) * pr.qmax, a.L);
      } else {
        guard_fail(a.sc, kGuardList, pr.s);
      }
    } else {
      guard_fail(a.sc, kGuardVertex, pr.s);
    }
  }
  // long lists: one at a time, the whole warp streams it, up to four entries per lane
  const uint32_t kLong = a.long_min;
  const bool tail_short = a.long_tail != 0;
  const bool was_long = dv >= kLong;
  unsigned longm = __ballot_sync(kFull, was_long);
  uint32_t probed = 0;  // entries of the long lists (the same in every lane)
  while (longm) {
    const int j = __ffs(longm) - 1;
    longm &= longm - 1;
    const uint32_t uj = __shfl_sync(kFull, pr.x, j);
    const uint32_t vj = __shfl_sync(kFull, pr.s, j);
    const uint32_t vsj = __shfl_sync(kFull, vs, j);
    const uint32_t dvj = __shfl_sync(kFull, dv, j);
    if constexpr (HasProbed<V>::value) probed += dvj;
    const uint32_t qj = __shfl_sync(kFull, pr.qe, j);
    const uint32_t pj = __shfl_sync(kFull, pr.pe, j);
    uint32_t off = 0;
    while (dvj - off >= 32 * UBT_LONG_U) {
      long_steps<V, UBT_LONG_U, true>(adj, sc, vis, t, lane, uj, vj, vsj, dvj, qj, pj, off);
      off += 32 * UBT_LONG_U;
    }
    if (UBT_LONG_U > 4 && dvj - off >= 128) {
      long_steps<V, 4, true>(adj, sc, vis, t, lane, uj, vj, vsj, dvj, qj, pj, off);
      off += 128;
    }
    if (tail_short) {
      // full half-chunk, then the rest (< 64 entries) is streamed with the short lists
      if (dvj - off >= 64) {
        long_steps<V, 2, true>(adj, sc, vis, t, lane, uj, vj, vsj, dvj, qj, pj, off);
        off += 64;
      }
      if (lane == j) {
        vs += off;
        dv -= off;
      }
    } else {
      while (off < dvj) {
        long_steps<V, 2, false>(adj, sc, vis, t, lane, uj, vj, vsj, dvj, qj, pj, off);
        off += 64;
      }
    }
  }
  // short lists: concatenated so that every lane probes one entry per half-step
  const uint32_t ds = (was_long && !tail_short) ? 0u : dv;
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
      uint32_t quw = 0, puw = 0;
      const bool found = table_find_warp<V::kPos>(t, adj_col(e[s]), quw, puw, sc);
      const bool hit = act[s] && found;
      const uint32_t uj = __shfl_sync(kFull, pr.x, j);
      const uint32_t vj = __shfl_sync(kFull, pr.s, j);
      const uint32_t qj = __shfl_sync(kFull, pr.qe, j);
      const uint32_t pj = __shfl_sync(kFull, pr.pe, j);
      if (s == 0 || base + 32 < total)
        vis.step(hit, uj, vj, adj_col(e[s]), qj, quw, adj_valbits(e[s]), pj, puw, f[s]);
    }
  }
  // a long list's tail streamed with the short lists is counted twice: an upper bound
  if constexpr (HasProbed<V>::value) vis.probed(probed + total);
}

// This lane's pair among the pairs [ps, ps + cnt) of owner x.  A pair whose
// edge fails Lemma 2 (|q_e| 2^30 < L) cannot be in a classified triangle.
__device__ __forceinline__ Pair owner_pair(const TravArgs& a, uint32_t x, int64_t qmax, uint32_t ps, uint32_t cnt) {
  const int lane = (int)lane_id();
  Pair pr;
  pr.x = x;
  pr.qmax = qmax;
  pr.ok = (uint32_t)lane < cnt;
  const uint64_t d = pr.ok ? a.pairs[ps + lane] : 0ull;
  pr.s = (uint32_t)d;
  pr.pe = (uint32_t)(d >> 32);
  if (pr.ok && pr.pe >= a.m) {
    guard_fail(a.sc, kGuardList, x);
    pr.ok = false;
  }
  const uint64_t e = pr.ok ? a.adj[pr.pe] : 0ull;
  pr.qe = adj_valbits(e);
  if (a.L > 0 && qabs(pr.qe) * (1ll << 30) < a.L) pr.ok = false;
  return pr;
}

// Entries of x's list that go into its table (the Lemma 2 prefix) and qmax(x);
// identical in every calling thread.
__device__ __forceinline__ uint32_t table_len(const TravArgs& a, uint32_t rs, uint32_t len, int64_t& qmax) {
  qmax = 0;
  if (a.L > 0 && len > 0) {
    qmax = qabs(adj_valbits(a.adj[rs]));
    return prune_prefix(a.adj + rs, len, 1ll << 30, a.L);
  }
  return len;
}

// Pair range of owner x, checked against the pair array's bounds.
__device__ __forceinline__ bool pair_range(const TravArgs& a, uint32_t x, uint32_t& ps, uint32_t& np) {
  ps = a.pair_ptr[x];
  const uint32_t pe = a.pair_ptr[x + 1];
  if (pe < ps || pe > a.m) return false;
  np = pe - ps;
  return true;
}

// A whole block handles owner x; `tab` is shared memory (hub) or a global
// slice (giant).
template <class V>
__device__ __forceinline__ void block_task(const TravArgs& a, V& vis, uint32_t x, uint32_t* tab, uint32_t cap,
                                           uint32_t* s_misc) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (x >= a.n) {
    if (tid == 0) guard_fail(a.sc, kGuardVertex, x);
    return;
  }
  const uint32_t rs = a.row_ptr[x], re = a.row_ptr[x + 1];
  uint32_t ps = 0, np = 0;
  if (re < rs || re > a.m || !pair_range(a, x, ps, np)) {
    if (tid == 0) guard_fail(a.sc, kGuardList, x);
    return;
  }
  int64_t qmax = 0;
  if (tid == 0) s_misc[0] = table_len(a, rs, re - rs, qmax);
  __syncthreads();
  const uint32_t len = s_misc[0];
  if (a.L > 0 && len > 0) qmax = qabs(adj_valbits(a.adj[rs]));
  const uint32_t slots = slots_for(len);
  if (len == 0 || np == 0 || slots > cap) {
    if (len && np && slots > cap && tid == 0) guard_fail(a.sc, kGuardTable, x);
    __syncthreads();
    return;
  }
  const Table t = make_table(tab, cap, slots);
  for (uint32_t i = tid; i < slots; i += blockDim.x) t.key[i] = kEmpty;
  if (tid == 0) s_misc[1] = 0;
  __syncthreads();
  for (uint32_t i = tid; i < len; i += blockDim.x) {
    const uint64_t e = a.adj[rs + i];
    table_insert<V::kPos>(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
  }
  __syncthreads();
  vis.task_begin(x);
  // warps take pairs `unit` at a time, fewer as the pairs run out, so that
  // they reach the closing barrier at about the same time
  const uint32_t nw = blockDim.x >> 5;
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
    probe_pairs<V>(a, vis, t, owner_pair(a, x, qmax, ps + c, cnt));
  }
  vis.task_end(x);
  __syncthreads();
}

// One warp handles owner x.
template <class V>
__device__ __forceinline__ void warp_task(const TravArgs& a, V& vis, uint32_t x, uint32_t* tab) {
  const int lane = (int)lane_id();
  if (x >= a.n) {
    if (lane == 0) guard_fail(a.sc, kGuardVertex, x);
    return;
  }
  const uint32_t rs = a.row_ptr[x], re = a.row_ptr[x + 1];
  uint32_t ps = 0, np = 0;
  if (re < rs || re > a.m || !pair_range(a, x, ps, np)) {
    if (lane == 0) guard_fail(a.sc, kGuardList, x);
    return;
  }
  int64_t qmax = 0;
  const uint32_t len = table_len(a, rs, re - rs, qmax);
  if (len == 0 || np == 0) return;
  const uint32_t slots = slots_for(len);
  if (slots > a.warp_slots) {
    if (lane == 0) guard_fail(a.sc, kGuardTable, x);
    return;
  }
  const Table t = make_table(tab, a.warp_slots, slots);
  for (uint32_t i = lane; i < slots; i += 32) t.key[i] = kEmpty;
  __syncwarp();
  for (uint32_t i = lane; i < len; i += 32) {
    const uint64_t e = a.adj[rs + i];
    table_insert<V::kPos>(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
  }
  __syncwarp();
  vis.task_begin(x);
  for (uint32_t cs = 0; cs < np; cs += 32)
    probe_pairs<V>(a, vis, t, owner_pair(a, x, qmax, ps + cs, min(32u, np - cs)));
  vis.task_end(x);
  __syncwarp();
}

// The traversal runs as two persistent kernels, so that each can have the
// block size and shared memory its tasks need: the block kernel (giant and
// hub tasks, one large table per block) and the warp kernel (medium tasks,
// one small table per warp).
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
    uint32_t* wtab = tab + (size_t)wid * table_words<V>(a.warp_slots);
    // medium tasks, one warp each
    while (true) {
      unsigned long long t0 = 0;
      if (lane == 0) t0 = atomicAdd(&a.sc->task[2], (unsigned long long)a.batch);
      t0 = __shfl_sync(kFull, t0, 0);
      if (t0 >= a.n_med) break;
      const uint32_t t1 = (uint32_t)min((unsigned long long)a.n_med, t0 + a.batch);
      for (uint32_t t = (uint32_t)t0; t < t1; t++) warp_task(a, vis, a.med_list[t], wtab);
    }
  }
  __syncthreads();
  vis.block_end();
}

// Shared memory of one block of a traversal kernel: visitor bytes + tables
// (words 32-bit words per table slot).
template <class V>
inline size_t traverse_smem_bytes(const TravArgs& a, int phases, int threads) {
  const size_t vis_bytes = (size_t)((V::smem_bytes(threads) + 15) / 16) * 16;
  size_t tables = 0;
  if (phases & kBlockTasks) tables = std::max(tables, (size_t)table_words<V>(a.hub_slots) * 4);
  if (phases & kWarpTasks) tables = std::max(tables, (size_t)(threads / 32) * table_words<V>(a.warp_slots) * 4);
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
  const size_t smem = traverse_smem_bytes<V>(a, kPhases, threads);
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
// tasks) run one after the other on `s`.
template <class V>
ubt_status launch_traversal(const ubt_graph* g, const TravArgs& a, const typename V::P& p, cudaStream_t s) {
  UBT_RANGE("traversal launch");
  const Tuning& T = tuning();
  UBT_CUDA(cudaMemsetAsync(a.sc, 0, kScratchHeader / 2, s));
  if (a.n_giant + a.n_hub > 0) {
    const ubt_status st = launch_phase<V, kBlockTasks>(g, a, p, (int)T.block_threads, s);
    if (st != UBT_OK) return st;
  }
  if (a.n_med > 0) {
    const ubt_status st = launch_phase<V, kWarpTasks>(g, a, p, (int)T.warp_threads, s);
    if (st != UBT_OK) return st;
  }
  return UBT_OK;
}

}  // namespace

}  // namespace ubt
