// ubt_traverse.cuh -- the triangle traversal every query runs.
//
// Forward edge iteration under Node Order (Alg. 1, Sec. 4): triangle {u,v,w}
// with u < v < w in Node Order is found exactly once, from u, as
// w in N>(u) n N>(v) for v in N>(u).
//
// GPU layout of that loop:
//   * u's forward list is loaded once into an open-addressing hash table
//     (neighbour -> edge value [, CSR position]) in shared memory: a whole
//     thread block shares it when the list is long ("hub" task), a single warp
//     owns a small one otherwise.  Lists too long for shared memory use a
//     per-block table in global memory ("giant" task).
//   * The out-neighbours v of u are taken 32 at a time by one warp.  Their
//     lists N>(v) are streamed with coalesced 8-byte loads: long lists one at
//     a time by the whole warp, short lists concatenated ("flattened") so that
//     every lane has an entry to probe.  Each streamed entry w is probed in
//     u's table; a hit is a triangle, handed to the visitor with the three
//     edge values and CSR positions.
//   * Probability pruning (FIXED graphs, level L > 0): every list is sorted by
//     |q| descending, so the entries that cannot reach |P| >= L are suffixes:
//       u's table and v-loop:  |q_e| * qmax(u) * 2^15 >= L   (Lemma 2: each
//                              edge bounds the product of the triangle)
//       v's list for pair u-v: |q_vw| * |q_uv| * qmax(u) >= L (order-free form
//                              of Lemma 3: the other two edges bound it)
//     qmax(u) is the largest |q| in N>(u) (its first entry).
//
// Visitors implement: block_init / task_begin / step (called by all 32 lanes
// of a warp, converged, once per probed entry with a hit flag) / task_end /
// block_end.
#pragma once

#include "ubt_internal.cuh"

namespace ubt {

struct TravArgs {
  const uint32_t* row_ptr;
  const uint64_t* adj;
  const uint32_t* giant_list;
  const uint32_t* hub_list;
  const uint32_t* small_list;
  uint32_t n_giant, n_hub, n_small;
  Scratch* sc;              // task counters (zeroed before launch)
  uint32_t* gtab;           // giant tables: gtab_blocks x gtab_slots x 3 words
  uint32_t gtab_slots;      // power of two
  uint32_t gtab_blocks;
  uint32_t hub_slots;       // shared-memory hub table capacity (power of two)
  uint32_t small_slots;     // per-warp table capacity (power of two)
  uint32_t small_batch;     // small tasks taken per grab
  uint32_t table_words;     // 2 (key, value) or 3 (+ CSR position)
  int64_t L;                // prune level, 0 = none
};

__device__ __forceinline__ uint32_t hash_slot(uint32_t w, int shift) { return (w * 0x9E3779B1u) >> shift; }

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

struct Table {
  uint32_t* key;
  uint32_t* val;
  uint32_t* pos;
  uint32_t mask;
  int shift;
};

__device__ __forceinline__ Table make_table(uint32_t* base, uint32_t cap, uint32_t slots, bool with_pos) {
  Table t;
  t.key = base;
  t.val = base + cap;
  t.pos = with_pos ? base + 2 * cap : nullptr;
  t.mask = slots - 1;
  t.shift = 32 - (31 - __clz((int)slots));
  return t;
}

__device__ __forceinline__ void table_insert(const Table& t, uint32_t w, uint32_t val, uint32_t pos) {
  uint32_t h = hash_slot(w, t.shift);
  while (true) {
    const uint32_t old = atomicCAS(&t.key[h], kEmpty, w);
    if (old == kEmpty) {
      t.val[h] = val;
      if (t.pos) t.pos[h] = pos;
      return;
    }
    h = (h + 1) & t.mask;
  }
}

__device__ __forceinline__ bool table_find(const Table& t, uint32_t w, uint32_t& val, uint32_t& pos) {
  uint32_t h = hash_slot(w, t.shift);
  while (true) {
    const uint32_t k = t.key[h];
    if (k == w) {
      val = t.val[h];
      if (t.pos) pos = t.pos[h];
      return true;
    }
    if (k == kEmpty) return false;
    h = (h + 1) & t.mask;
  }
}

__device__ __forceinline__ uint32_t slots_for(uint32_t len) {
  uint32_t s = 32;
  while (s < 2 * len) s <<= 1;
  return s;
}

// One warp: the out-neighbours at CSR positions [cs, cs + cnt) of u (cnt <= 32).
template <class V>
__device__ __forceinline__ void process_chunk(const TravArgs& a, V& vis, const Table& t, uint32_t u, int64_t qmax_u,
                                              uint32_t cs, uint32_t cnt) {
  const int lane = threadIdx.x & 31;
  uint32_t v = 0, vs = 0, dv = 0, quv = 0, puv = 0;
  if ((uint32_t)lane < cnt) {
    puv = cs + lane;
    const uint64_t e = a.adj[puv];
    v = adj_col(e);
    quv = adj_valbits(e);
    vs = a.row_ptr[v];
    dv = a.row_ptr[v + 1] - vs;
    if (a.L > 0) dv = prune_prefix(a.adj + vs, dv, qabs(quv) * qmax_u, a.L);
  }
  // long lists: one at a time, the whole warp streams it
  unsigned longm = __ballot_sync(kFull, dv >= 24);
  while (longm) {
    const int j = __ffs(longm) - 1;
    longm &= longm - 1;
    const uint32_t vj = __shfl_sync(kFull, v, j);
    const uint32_t vsj = __shfl_sync(kFull, vs, j);
    const uint32_t dvj = __shfl_sync(kFull, dv, j);
    const uint32_t qj = __shfl_sync(kFull, quv, j);
    const uint32_t pj = __shfl_sync(kFull, puv, j);
    for (uint32_t off = 0; off < dvj; off += 32) {
      const uint32_t i = off + lane;
      const bool act = i < dvj;
      uint64_t e2 = act ? a.adj[vsj + i] : 0ull;
      uint32_t quw = 0, puw = 0;
      const bool hit = act && table_find(t, adj_col(e2), quw, puw);
      vis.step(hit, u, vj, adj_col(e2), qj, quw, adj_valbits(e2), pj, puw, vsj + i);
    }
  }
  // short lists: concatenated so that every lane probes one entry
  const uint32_t ds = dv >= 24 ? 0u : dv;
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
    // owner: number of lanes whose inclusive end is <= f
    int j = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const uint32_t tj = __shfl_sync(kFull, incl, j + s - 1);
      if (tj <= f) j += s;
    }
    j = j > 31 ? 31 : j;
    const uint32_t vj = __shfl_sync(kFull, v, j);
    const uint32_t vsj = __shfl_sync(kFull, vs, j);
    const uint32_t exj = __shfl_sync(kFull, excl, j);
    const uint32_t qj = __shfl_sync(kFull, quv, j);
    const uint32_t pj = __shfl_sync(kFull, puv, j);
    const uint32_t pvw = vsj + (f - exj);
    uint64_t e2 = act ? a.adj[pvw] : 0ull;
    uint32_t quw = 0, puw = 0;
    const bool hit = act && table_find(t, adj_col(e2), quw, puw);
    vis.step(hit, u, vj, adj_col(e2), qj, quw, adj_valbits(e2), pj, puw, pvw);
  }
}

// A whole block handles u; `tab` is shared memory (hub) or a global slice (giant).
template <class V>
__device__ __forceinline__ void block_task(const TravArgs& a, V& vis, uint32_t u, uint32_t* tab, uint32_t cap, uint32_t* s_misc) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const uint32_t rs = a.row_ptr[u], re = a.row_ptr[u + 1];
  uint32_t len = re - rs;
  int64_t qmax = 0;
  if (a.L > 0 && len > 0) {
    qmax = qabs(adj_valbits(a.adj[rs]));
    if (tid == 0) s_misc[0] = prune_prefix(a.adj + rs, len, qmax * 32768, a.L);
    __syncthreads();
    len = s_misc[0];
    __syncthreads();
  }
  if (len == 0) return;
  const uint32_t slots = slots_for(len);
  const Table t = make_table(tab, cap, slots, a.table_words == 3);
  for (uint32_t i = tid; i < slots; i += blockDim.x) t.key[i] = kEmpty;
  if (tid == 0) s_misc[1] = 0;
  __syncthreads();
  for (uint32_t i = tid; i < len; i += blockDim.x) {
    const uint64_t e = a.adj[rs + i];
    table_insert(t, adj_col(e), adj_valbits(e), rs + i);
  }
  __syncthreads();
  vis.task_begin(u);
  const uint32_t nchunks = (len + 31) / 32;
  while (true) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(&s_misc[1], 1u);
    c = __shfl_sync(kFull, c, 0);
    if (c >= nchunks) break;
    const uint32_t cs = c * 32;
    process_chunk(a, vis, t, u, qmax, rs + cs, min(32u, len - cs));
  }
  (void)wid;
  (void)nw;
  vis.task_end(u);
  __syncthreads();
}

// One warp handles u (list of at most hub_threshold entries).
template <class V>
__device__ __forceinline__ void warp_task(const TravArgs& a, V& vis, uint32_t u, uint32_t* tab) {
  const int lane = threadIdx.x & 31;
  const uint32_t rs = a.row_ptr[u], re = a.row_ptr[u + 1];
  uint32_t len = re - rs;
  int64_t qmax = 0;
  if (a.L > 0 && len > 0) {
    qmax = qabs(adj_valbits(a.adj[rs]));
    // prefix of entries with |q| * qmax * 2^15 >= L, by ballot over the list
    uint32_t first_fail = len;
    for (uint32_t off = 0; off < len; off += 32) {
      const uint32_t i = off + lane;
      const bool fail = i < len && qabs(adj_valbits(a.adj[rs + i])) * qmax * 32768 < a.L;
      const unsigned b = __ballot_sync(kFull, fail);
      if (b) {
        first_fail = off + __ffs(b) - 1;
        break;
      }
    }
    len = first_fail;
  }
  if (len == 0) return;
  const uint32_t slots = slots_for(len);
  const Table t = make_table(tab, a.small_slots, slots, a.table_words == 3);
  for (uint32_t i = lane; i < slots; i += 32) t.key[i] = kEmpty;
  __syncwarp();
  for (uint32_t i = lane; i < len; i += 32) {
    const uint64_t e = a.adj[rs + i];
    table_insert(t, adj_col(e), adj_valbits(e), rs + i);
  }
  __syncwarp();
  vis.task_begin(u);
  for (uint32_t cs = 0; cs < len; cs += 32) process_chunk(a, vis, t, u, qmax, rs + cs, min(32u, len - cs));
  vis.task_end(u);
  __syncwarp();
}

// Persistent traversal kernel body.  Shared memory: [visitor bytes][tables].
template <class V>
__device__ void traverse(const TravArgs& a, V& vis, char* smem_tables) {
  __shared__ uint32_t s_misc[4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t* tab = (uint32_t*)smem_tables;
  // phase 0: giant lists, tables in global memory (first gtab_blocks blocks)
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
  // phase 1: hub lists, block-wide shared-memory tables
  while (true) {
    if (tid == 0) s_misc[2] = (uint32_t)atomicAdd(&a.sc->task[1], 1ull);
    __syncthreads();
    const uint32_t task = s_misc[2];
    __syncthreads();
    if (task >= a.n_hub) break;
    block_task(a, vis, a.hub_list[task], tab, a.hub_slots, s_misc);
  }
  // phase 2: small lists, one warp each, `small_batch` consecutive tasks per grab
  uint32_t* wtab = tab + (size_t)wid * a.small_slots * a.table_words;
  while (true) {
    unsigned long long t0 = 0;
    if (lane == 0) t0 = atomicAdd(&a.sc->task[2], (unsigned long long)a.small_batch);
    t0 = __shfl_sync(kFull, t0, 0);
    if (t0 >= a.n_small) break;
    const uint32_t t1 = (uint32_t)min((unsigned long long)a.n_small, t0 + a.small_batch);
    for (uint32_t t = (uint32_t)t0; t < t1; t++) warp_task(a, vis, a.small_list[t], wtab);
  }
  __syncthreads();
  vis.block_end();
}

}  // namespace ubt
