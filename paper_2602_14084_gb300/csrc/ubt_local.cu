// ubt_local.cu -- local counts of sampled edges and vertices, and the
// sampling estimators built on them (Sec. 6).
//
// Edge sampling (Algs. 5-6): for k edges drawn uniformly, the local counts
// |B_t(e)| / |U_t(e)| (t-balanced / t-unbalanced triangles through e) are
// extrapolated as |E| |B_t(e)| / 3 and averaged.  Vertex sampling (Algs.
// 3-4): the same with the triangles through a vertex and |V| |B_t(v)| / 3.
// Both are unbiased: every triangle has three edges and three vertices.  The
// samples are the caller's (the method's random draws are inputs here).
//
// The improved local searches of Algs. 4 and 6 scan neighbour lists in
// Absolute Edge Order and stop at the pruning cutoffs; here the undirected
// rows (|q| descending, UBT_OPT_UNDIRECTED) make every cutoff a prefix:
//   edge e = x-y:  w with |q_xw| |q_e| 2^15 >= L on both rows (the third
//                  factor is at most 2^15), nothing if |q_e| 2^30 < L
//   vertex v:      its row's Lemma 2 prefix; for each a there, a's row up to
//                  |q_ab| |q_va| qmax(v) >= L, and b counts once, at the later
//                  of the two positions in v's row
// One block per sample: the longer list (edge) or v's row (vertex) becomes a
// shared-memory hash table, in chunks when it is longer than one table, and
// the other lists are streamed through it.  Every triangle found is placed
// among the sorted threshold levels by binary search and counted in a
// per-sample shared histogram, turned into per-threshold counts at the end.
#include <algorithm>
#include <numeric>
#include <vector>

#include "ubt_traverse.cuh"

namespace ubt {

namespace {

constexpr int kLocalTau = 64;
constexpr int kLocalSub = 256;  // streamed entries per warp task of an edge sample

struct LocalP {
  int nt;
  int half;                     // 2^(K-1) with 2^K > 2 nt
  int64_t S[2 * kLocalTau];     // levels: every B and every U, ascending
  int perm[kLocalTau];          // caller index of the i-th smallest t
};

// Edge index lookup (UBT_OPT_EDGE_INDEX): the value of edge a-b, if present.
// Probes end at the key or an empty slot (at most a quarter of the slots are
// used); the bound is a self-check.
struct EdgeIndex {
  const uint4* slots;
  uint64_t mask;   // slots - 1
  int shift;
  int mode;        // 0 unused, 1 where cheaper than streaming, 2 always
};

__device__ __forceinline__ bool edge_index_find(const EdgeIndex& ix, uint32_t a, uint32_t b, uint32_t& val,
                                                Scratch* sc) {
  const int r = edge_index_lookup(ix.slots, ix.mask, ix.shift, a, b, val);
  if (r < 0) guard_fail(sc, kGuardFind, a);
  return r > 0;
}

// Vertex queries: the triangles v-a-b with b among `cand` positions of v's
// row are found either by streaming a's row (`len` entries) through v's
// table or by looking every candidate pair a-b up in the edge index; a
// lookup costs a few dependent random reads, a streamed entry one coalesced
// read and a shared-memory probe.
constexpr uint32_t kIndexCost = 8;
__device__ __forceinline__ bool use_index(const EdgeIndex& ix, uint32_t cand, uint32_t len) {
  return ix.mode == 2 || (ix.mode == 1 && (uint64_t)cand * kIndexCost < len);
}

// Triangles v-a-w with w after a in v's row (positions pa + 1 .. rend), from
// the edge index alone (rows longer than one shared-memory table): the
// smaller of
//   every b after a in v's row, looked up as a-b, and
//   every w among the first `len` entries of a's row (from s0), looked up
//   as v-w and kept when w comes after a in v's row -- the rows are in
//   Absolute Edge Order, so that is |q_vw| < |q_va|, or equal and w > a --
//   and lies in v's Lemma 2 prefix (|q_vw| 2^30 >= L, L = 0: all).
// found(P, w) receives every triangle.
// Two lookups of one lane at once: both home slots are read before either
// is examined (at most a quarter of the slots are used, so nearly every
// lookup ends there); the rare longer probe continues alone.
__device__ __forceinline__ void edge_index_find2(const EdgeIndex& ix, const bool (&act)[2], const uint32_t (&a)[2],
                                                 const uint32_t (&b)[2], bool (&hit)[2], uint32_t (&val)[2],
                                                 Scratch* sc) {
  uint64_t k[2];
  uint4 sl[2];
#pragma unroll
  for (int i = 0; i < 2; i++) {
    k[i] = edge_index_key(a[i], b[i]);
    sl[i] = act[i] ? ix.slots[edge_index_home(k[i], ix.shift)] : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
  }
#pragma unroll
  for (int i = 0; i < 2; i++) {
    hit[i] = false;
    val[i] = 0;
    if (!act[i]) continue;
    const uint64_t key = ((uint64_t)sl[i].y << 32) | sl[i].x;
    if (key == k[i]) {
      hit[i] = true;
      val[i] = sl[i].z;
    } else if (key != kEdgeIndexEmpty) {  // the home slot holds another edge: probe on
      hit[i] = edge_index_find(ix, a[i], b[i], val[i], sc);
    }
  }
}

template <class F>
__device__ __forceinline__ void index_pairs(const EdgeIndex& ix, const uint64_t* __restrict__ uadj, uint32_t v,
                                            uint32_t av, uint32_t qa, uint32_t pa, uint32_t rend, uint32_t s0,
                                            uint32_t len, int64_t L, int lane, Scratch* sc, F&& found) {
  if (rend - (pa + 1) <= len) {
    for (uint32_t b0 = pa + 1; b0 < rend; b0 += 64) {
      bool act[2], hit[2];
      uint32_t oo[2], ww[2], qab[2];
      uint64_t eb[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const uint32_t pos = b0 + 32 * u + lane;
        act[u] = pos < rend;
        eb[u] = act[u] ? uadj[pos] : 0ull;
        oo[u] = av;
        ww[u] = adj_col(eb[u]);
      }
      edge_index_find2(ix, act, oo, ww, hit, qab, sc);
#pragma unroll
      for (int u = 0; u < 2; u++)
        if (hit[u])
          found((long long)((int32_t)qa * (int32_t)adj_valbits(eb[u])) * (long long)(int32_t)qab[u], ww[u]);
    }
  } else {
    const int64_t aq = qabs(qa);
    for (uint32_t b0 = s0; b0 < s0 + len; b0 += 64) {
      bool act[2], hit[2];
      uint32_t oo[2], ww[2], qvw[2];
      uint64_t ew[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const uint32_t pos = b0 + 32 * u + lane;
        ew[u] = pos < s0 + len ? uadj[pos] : 0ull;
        ww[u] = adj_col(ew[u]);
        act[u] = pos < s0 + len && ww[u] != v;
        oo[u] = v;
      }
      edge_index_find2(ix, act, oo, ww, hit, qvw, sc);
#pragma unroll
      for (int u = 0; u < 2; u++) {
        if (!hit[u]) continue;
        const int64_t wq = qabs(qvw[u]);
        if ((wq < aq || (wq == aq && ww[u] > av)) && (L == 0 || wq * (1ll << 30) >= L))
          found((long long)((int32_t)qa * (int32_t)qvw[u]) * (long long)(int32_t)adj_valbits(ew[u]), ww[u]);
      }
    }
  }
}

EdgeIndex edge_index_of(const ubt_graph* g) {
  EdgeIndex ix;
  ix.slots = g->eslots;
  ix.mask = g->eh_slots ? (uint64_t)g->eh_slots - 1 : 0;
  ix.shift = g->eh_shift;
  ix.mode = g->eslots ? (int)tuning().edge_index : 0;
  return ix;
}

// Vertex samples whose pruned row is longer than `split` (with the edge
// index) are not counted by one block: the sampling kernel queues them (at
// most kLongCap per query; more are counted in place) and a second launch
// spreads their neighbours over the warps of all blocks.  The queue
// (ubt_graph::lqueue): [0] queued, [1] next warp task, [2 + i] entry i =
// row length << 32 | sample index.
constexpr int kLongCap = kLongQueue;

struct LocalArgs {
  const uint32_t* uptr;
  const uint64_t* uadj;
  EdgeIndex ix;
  uint32_t split;               // pruned rows longer than this are split across blocks
  unsigned long long* lq;       // the queue of long samples (ubt_graph::lqueue)
  const uint32_t* uepos;        // 2m: positions of every edge in its endpoints' rows
  const uint32_t* items;        // sampled edges (input index) or vertices
  uint32_t n_items;
  int vertex_mode;
  uint32_t n, m, m2;
  int64_t L;
  uint32_t cap;                 // table slots
  Scratch* sc;
  int64_t* bal;                 // [item][t]
  int64_t* unbal;
};

// interval of P among the levels: #{S_j < P} (levels padded with +inf)
__device__ __forceinline__ int level_of(const long long* S, int half, long long P) {
  int r = 0;
  for (int b = half; b > 0; b >>= 1)
    if (S[r + b - 1] < P) r += b;
  return r;
}

// Neighbours j0, j0 + step, ... < j1 of vertex x (row at rs, Lemma 2 prefix
// tlen, largest |q| qmax), every pair from the edge index, each triangle
// once (the other vertex after the neighbour in x's row) and binned.
__device__ __forceinline__ void index_neighbours(const LocalArgs& a, const LocalP& p, const long long* S,
                                                 unsigned long long* bins, uint32_t x, uint32_t rs, uint32_t tlen,
                                                 int64_t qmax, uint32_t j0, uint32_t j1, uint32_t step, int lane) {
  for (uint32_t j = j0; j < j1; j += step) {
    const uint64_t ea = a.uadj[rs + j];
    const uint32_t av = adj_col(ea), qp = adj_valbits(ea);
    if (av >= a.n) {
      if (lane == 0) guard_fail(a.sc, kGuardVertex, av);
      continue;
    }
    const uint32_t s0 = a.uptr[av];
    uint32_t len = a.uptr[av + 1] - s0;
    if (a.L > 0) len = prune_prefix(a.uadj + s0, len, qabs(qp) * qmax, a.L);
    index_pairs(a.ix, a.uadj, x, av, qp, rs + j, rs + tlen, s0, len, a.L, lane, a.sc,
                [&](long long P, uint32_t) { atomicAdd(&bins[level_of(S, p.half, P)], 1ull); });
  }
}

__global__ void __launch_bounds__(512, 2) k_local(LocalArgs a, LocalP p) {
  extern __shared__ __align__(16) char smem[];
  __shared__ uint32_t s_misc[8];
  long long* S = (long long*)smem;                       // 256 padded levels
  unsigned long long* bins = (unsigned long long*)(smem + 256 * 8);  // 2 nt + 1 (<= 129) bins
  uint32_t* tab = (uint32_t*)(bins + 144);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < 256; i += blockDim.x) S[i] = i < 2 * p.nt ? p.S[i] : INT64_MAX;
  __syncthreads();
  while (true) {
    if (tid == 0) s_misc[0] = (uint32_t)atomicAdd(&a.sc->task[0], 1ull);
    for (int i = tid; i <= 2 * p.nt; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    const uint32_t item = s_misc[0];
    if (item >= a.n_items) break;
    // the sample: table row x (its prefix tlen), the pair's value and, for an
    // edge, the streamed row y (its prefix ylen)
    uint32_t x = 0, y = 0, tlen = 0, ylen = 0, qe = 0, npv = 0;
    int64_t qmax = 0;
    bool ok = true;
    const uint32_t id = a.items[item];
    if (!a.vertex_mode) {
      if (id >= a.m) {
        if (tid == 0) guard_fail(a.sc, kGuardList, id);
        ok = false;
      } else {
        const uint32_t p0 = a.uepos[2 * (size_t)id], p1 = a.uepos[2 * (size_t)id + 1];
        const uint32_t lo = adj_col(a.uadj[p1]), hi = adj_col(a.uadj[p0]);  // endpoints
        qe = adj_valbits(a.uadj[p0]);
        const uint32_t dlo = a.uptr[lo + 1] - a.uptr[lo], dhi = a.uptr[hi + 1] - a.uptr[hi];
        x = dhi >= dlo ? hi : lo;
        y = x == hi ? lo : hi;
        const int64_t c = qabs(qe) * 32768;
        if (a.L > 0 && qabs(qe) * (1ll << 30) < a.L) ok = false;  // Lemma 2 on e
        tlen = a.uptr[x + 1] - a.uptr[x];
        ylen = a.uptr[y + 1] - a.uptr[y];
        if (a.L > 0) {
          tlen = prune_prefix(a.uadj + a.uptr[x], tlen, c, a.L);
          ylen = prune_prefix(a.uadj + a.uptr[y], ylen, c, a.L);
        }
        npv = (ylen + kLocalSub - 1) / kLocalSub;
      }
    } else {
      if (id >= a.n) {
        if (tid == 0) guard_fail(a.sc, kGuardVertex, id);
        ok = false;
      } else {
        x = id;
        tlen = a.uptr[x + 1] - a.uptr[x];
        if (a.L > 0 && tlen > 0) {
          qmax = qabs(adj_valbits(a.uadj[a.uptr[x]]));
          tlen = prune_prefix(a.uadj + a.uptr[x], tlen, 1ll << 30, a.L);  // Lemma 2
        }
        npv = tlen;
      }
    }
    const uint32_t rs = a.uptr[x];
    const uint32_t chunk = a.cap / 4;
    if (ok && a.vertex_mode && a.ix.mode != 0 && (tlen > chunk || tlen > a.split)) {
      // a long row: no table, every pair from the edge index -- counted by the
      // split launch when the queue has room (its counts here stay 0), else here
      if (tid == 0) {
        uint32_t queued = 0;
        if (tlen > a.split) {
          const unsigned long long slot = atomicAdd(&a.lq[0], 1ull);
          if (slot < (unsigned long long)kLongCap) {
            a.lq[2 + slot] = ((unsigned long long)tlen << 32) | item;
            queued = 1;
          }
        }
        s_misc[1] = queued;
      }
      __syncthreads();
      if (!s_misc[1]) index_neighbours(a, p, S, bins, x, rs, tlen, qmax, wid, tlen ? tlen - 1 : 0, nw, lane);
      ok = false;  // skip the table chunks
    }
    for (uint32_t c0 = 0; ok && c0 < tlen; c0 += chunk) {
      const uint32_t c1 = min(tlen, c0 + chunk);
      const uint32_t slots = slots_for(c1 - c0);
      const Table t = make_table(tab, a.cap, slots);
      for (uint32_t i = tid; i < slots; i += blockDim.x) t.key[i] = kEmpty;
      __syncthreads();
      for (uint32_t i = c0 + tid; i < c1; i += blockDim.x) {
        const uint64_t e = a.uadj[rs + i];
        table_insert(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
      }
      __syncthreads();
      for (uint32_t v = wid; v < npv; v += nw) {
        // the streamed range of this warp task and the pair it belongs to
        uint32_t s0, s1, qp, pp = 0;
        if (!a.vertex_mode) {
          s0 = a.uptr[y] + v * kLocalSub;
          s1 = a.uptr[y] + min(ylen, (v + 1) * kLocalSub);
          qp = qe;
        } else {
          pp = rs + v;                      // x-a at position pp of x's row
          if (pp + 1 >= rs + c1) continue;  // no table entry after it in this chunk
          const uint64_t ea = a.uadj[pp];
          const uint32_t av = adj_col(ea);
          qp = adj_valbits(ea);
          if (av >= a.n) {
            if (lane == 0) guard_fail(a.sc, kGuardVertex, av);
            continue;
          }
          s0 = a.uptr[av];
          uint32_t len = a.uptr[av + 1] - s0;
          if (a.L > 0) len = prune_prefix(a.uadj + s0, len, qabs(qp) * qmax, a.L);
          s1 = s0 + len;
          // the same triangles from v's side: b after a in this chunk of v's
          // row, each pair a-b looked up in the edge index
          const uint32_t b_lo = max(pp + 1, rs + c0), b_hi = rs + c1;
          if (use_index(a.ix, b_hi - b_lo, len)) {
            for (uint32_t b0 = b_lo; b0 < b_hi; b0 += 32) {
              const uint32_t pos = b0 + lane;
              const bool act = pos < b_hi;
              const uint64_t eb = act ? a.uadj[pos] : 0ull;
              uint32_t qab = 0;
              const bool hit = act && edge_index_find(a.ix, av, adj_col(eb), qab, a.sc);
              if (hit) {
                const long long P = (long long)((int32_t)qp * (int32_t)adj_valbits(eb)) * (long long)(int32_t)qab;
                atomicAdd(&bins[level_of(S, p.half, P)], 1ull);
              }
            }
            continue;
          }
        }
        for (uint32_t b0 = s0; b0 < s1; b0 += 32) {
          const uint32_t pos = b0 + lane;
          const bool act = pos < s1;
          const uint64_t e = act ? a.uadj[pos] : 0ull;
          uint32_t qt = 0, pt = 0;
          bool hit = act && table_find<true>(t, adj_col(e), qt, pt, a.sc);
          if (a.vertex_mode) hit = hit && pt > pp;  // each triangle once: at the later position
          if (hit) {
            const long long P = (long long)((int32_t)qp * (int32_t)qt) * (long long)(int32_t)adj_valbits(e);
            atomicAdd(&bins[level_of(S, p.half, P)], 1ull);
          }
        }
      }
      __syncthreads();
    }
    __syncthreads();
    // histogram -> counts: the i-th smallest t has the (nt-1-i)-th smallest B
    // and the i-th smallest U
    if (tid < p.nt) {
      const int i = tid;
      long long b = 0, u = 0;
      for (int r = 0; r <= p.nt - 1 - i; r++) b += bins[r];
      for (int r = p.nt + i + 1; r <= 2 * p.nt; r++) u += bins[r];
      a.bal[(size_t)item * p.nt + p.perm[i]] = b;
      a.unbal[(size_t)item * p.nt + p.perm[i]] = u;
    }
    __syncthreads();
  }
}

// The split launch: the queued vertex samples' neighbours, kWarpNb per warp
// task from one counter over all queued samples, no block barriers.  Each
// warp bins into its own shared histogram and adds its per-threshold counts
// to the sample's outputs (zero after the sampling kernel) when it moves on
// to another sample or runs out of tasks.
constexpr uint32_t kWarpNb = 4;

__device__ __forceinline__ void flush_bins(const LocalArgs& a, const LocalP& p, unsigned long long* wb,
                                           uint32_t item, int lane) {
  __syncwarp();
  for (int i = lane; i < p.nt; i += 32) {
    unsigned long long b = 0, u = 0;
    for (int r = 0; r <= p.nt - 1 - i; r++) b += wb[r];
    for (int r = p.nt + i + 1; r <= 2 * p.nt; r++) u += wb[r];
    if (b) atomicAdd((unsigned long long*)&a.bal[(size_t)item * p.nt + p.perm[i]], b);
    if (u) atomicAdd((unsigned long long*)&a.unbal[(size_t)item * p.nt + p.perm[i]], u);
  }
  __syncwarp();
  for (int r = lane; r <= 2 * p.nt; r += 32) wb[r] = 0;
  __syncwarp();
}

__global__ void __launch_bounds__(512, 2) k_local_split(LocalArgs a, LocalP p) {
  extern __shared__ __align__(16) char smem[];
  __shared__ long long S[256];
  __shared__ uint32_t pref[kLongCap + 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long* wb = (unsigned long long*)smem + (size_t)wid * (2 * p.nt + 1);  // this warp's bins
  for (int i = tid; i < 256; i += blockDim.x) S[i] = i < 2 * p.nt ? p.S[i] : INT64_MAX;
  for (int r = lane; r <= 2 * p.nt; r += 32) wb[r] = 0;
  const uint32_t nq = (uint32_t)min(a.lq[0], (unsigned long long)kLongCap);
  if (wid == 0) {
    // first warp task of every entry: lane l sums entries [l * seg, (l + 1) * seg),
    // a warp scan gives each lane its segment's start
    constexpr uint32_t seg = (kLongCap + 31) / 32;
    const uint32_t b0 = lane * seg, b1 = min(nq, b0 + seg);
    uint32_t mine = 0;
    for (uint32_t i = b0; i < b1; i++)
      mine += ((uint32_t)(a.lq[2 + i] >> 32) - 1 + kWarpNb - 1) / kWarpNb;  // neighbours 0 .. tlen - 2
    uint32_t incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += y;
    }
    uint32_t acc = incl - mine;
    for (uint32_t i = b0; i < b1; i++) {
      pref[i] = acc;
      acc += ((uint32_t)(a.lq[2 + i] >> 32) - 1 + kWarpNb - 1) / kWarpNb;
    }
    if (lane == 31) pref[nq] = incl;
  }
  __syncthreads();
  const uint32_t total = pref[nq];
  uint32_t cur = 0xFFFFFFFFu;  // entry whose counts this warp's bins hold
  uint32_t cur_item = 0;
  while (true) {
    uint32_t task = 0;
    if (lane == 0) task = (uint32_t)atomicAdd(&a.lq[1], 1ull);
    task = __shfl_sync(kFull, task, 0);
    if (task >= total) break;
    uint32_t e = 0, hi = nq - 1;  // the last entry whose first task is <= task
    while (e < hi) {
      const uint32_t mid = (e + hi + 1) >> 1;
      if (pref[mid] <= task) e = mid; else hi = mid - 1;
    }
    const unsigned long long ent = a.lq[2 + e];
    const uint32_t item = (uint32_t)ent, tlen = (uint32_t)(ent >> 32);
    if (e != cur) {
      if (cur != 0xFFFFFFFFu) flush_bins(a, p, wb, cur_item, lane);
      cur = e;
      cur_item = item;
    }
    const uint32_t x = a.items[item], rs = a.uptr[x];
    const int64_t qmax = a.L > 0 ? qabs(adj_valbits(a.uadj[rs])) : 0;
    const uint32_t j0 = (task - pref[e]) * kWarpNb, j1 = min(j0 + kWarpNb, tlen - 1);
    index_neighbours(a, p, S, wb, x, rs, tlen, qmax, j0, j1, 1, lane);
  }
  if (cur != 0xFFFFFFFFu) flush_bins(a, p, wb, cur_item, lane);
}

// estimate[t] = scale / k * sum over samples of the local count
__global__ void k_local_estimate(const int64_t* __restrict__ bal, const int64_t* __restrict__ unbal, uint32_t k,
                                 int nt, double scale, double* __restrict__ est) {
  const int t = blockIdx.x;
  double sb = 0.0, su = 0.0;
  for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
    sb += (double)bal[(size_t)i * nt + t];
    su += (double)unbal[(size_t)i * nt + t];
  }
  __shared__ double rb[256], ru[256];
  rb[threadIdx.x] = sb;
  ru[threadIdx.x] = su;
  __syncthreads();
  for (int d = blockDim.x / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) {
      rb[threadIdx.x] += rb[threadIdx.x + d];
      ru[threadIdx.x] += ru[threadIdx.x + d];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    est[t] = k ? rb[0] * scale / (double)k : 0.0;
    est[nt + t] = k ? ru[0] * scale / (double)k : 0.0;
  }
}

ubt_status local_counts(ubt_graph* g, const uint32_t* d_items, int64_t k, int vertex_mode, const double* h_tau,
                        int32_t n_tau, int64_t* d_bal, int64_t* d_unbal, double* d_est, cudaStream_t s) {
  if (!g || k < 0 || (k > 0 && (!d_items || !d_bal || !d_unbal))) return UBT_ERR_INVALID_ARG;
  if (!h_tau || n_tau < 1 || n_tau > kLocalTau || k >= 0xFFFFFFFFll) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_FIXED || !g->uptr) return UBT_ERR_UNSUPPORTED;
  std::vector<Level> lv(n_tau);
  for (int i = 0; i < n_tau; i++)
    if (!tau_level(h_tau[i], &lv[i])) return UBT_ERR_TAU_OOB;
  std::vector<int> order(n_tau);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lv[x].L < lv[y].L; });
  LocalP p;
  p.nt = n_tau;
  p.half = 1;
  while (2 * p.half <= 2 * n_tau) p.half *= 2;
  for (int i = 0; i < n_tau; i++) {
    p.S[i] = lv[order[n_tau - 1 - i]].B;
    p.S[n_tau + i] = lv[order[i]].U;
    p.perm[i] = order[i];
  }
  const Tuning& T = tuning();
  LocalArgs a;
  a.uptr = g->uptr;
  a.uadj = g->uadj;
  a.ix = edge_index_of(g);
  a.split = (uint32_t)std::min<int64_t>(T.vertex_split, 0xFFFFFFFFll);
  a.lq = g->lqueue;
  a.uepos = g->uepos;
  a.items = d_items;
  a.n_items = (uint32_t)k;
  a.vertex_mode = vertex_mode;
  a.n = (uint32_t)g->n;
  a.m = (uint32_t)g->m;
  a.m2 = (uint32_t)(2 * g->m);
  a.L = lv[order[0]].L;
  a.cap = (uint32_t)std::min<int64_t>(table_slots(std::max<int64_t>(g->max_udeg, 2)),
                                      std::max<int64_t>(64, T.smem_table_max));
  a.sc = g->scratch;
  a.bal = d_bal;
  a.unbal = d_unbal;
  UBT_CUDA(cudaMemsetAsync(a.sc, 0, kScratchHeader / 2, s));
  UBT_CUDA(cudaMemsetAsync(a.lq, 0, 2 * sizeof(unsigned long long), s));
  if (k > 0) {
    const int threads = 512;
    const size_t smem = 256 * 8 + 144 * 8 + (size_t)a.cap * 3 * 4;
    UBT_CUDA(cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    UBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local, threads, smem));
    if (per_sm < 1) return UBT_ERR_INVALID_ARG;
    const int64_t blocks = std::min<int64_t>((int64_t)g->sm_count * per_sm, k);
    k_local<<<(int)blocks, threads, smem, s>>>(a, p);
    UBT_CUDA(cudaGetLastError());
    if (vertex_mode && a.ix.mode != 0) {
      const size_t wbytes = (size_t)(threads / 32) * (2 * n_tau + 1) * 8;  // per-warp bins
      k_local_split<<<(int)(g->sm_count * 2), threads, wbytes, s>>>(a, p);
      UBT_CUDA(cudaGetLastError());
    }
  }
  if (d_est) {
    const double scale = (vertex_mode ? (double)g->n : (double)g->m) / 3.0;
    k_local_estimate<<<n_tau, 256, 0, s>>>(d_bal, d_unbal, (uint32_t)k, n_tau, scale, d_est);
    UBT_CUDA(cudaGetLastError());
  }
  return UBT_OK;
}

// ------------------------------------------------------------ per-vertex top-k

// Per-vertex top-k (Sec. 5: "top-k ... locally for each node"): for every
// listed vertex, its K triangles of highest balance (which = 1) or unbalance
// (which = 2) probability.  One block per vertex, two passes over the
// triangles through it (its row as the table, every neighbour's row
// streamed, each triangle once): a histogram of the triangles' rank key
// r = P + 2^45 (balanced) or 2^45 - P (unbalanced; smaller is better) over
// 2049 slices of 2^35 finds the slice holding the K-th best; the second pass
// keeps the triangles of better slices (fewer than K) and as many of that
// slice as fit, and a shared-memory sort by (r, u, v, w) gives the answer.
constexpr int kTopkSlices = 2049;  // slices of 2^35 over the rank range [0, 2^46]
constexpr int kTopkCap = 1024;   // candidate buffer per vertex
constexpr int kTopkMax = 256;    // largest K

struct TopkArgs {
  const uint32_t* uptr;
  const uint64_t* uadj;
  EdgeIndex ix;
  const uint32_t* items;
  uint32_t n_items, n, m2, K;
  int which;
  uint32_t cap;                  // table slots
  Scratch* sc;
  ubt_tri_rec* out;              // [item][K]
  int32_t* n_out;                // [item]
};

__device__ __forceinline__ uint64_t topk_rank(long long P, int which) {
  return which == 1 ? (uint64_t)(P + (1ll << 45)) : (uint64_t)((1ll << 45) - P);
}

__device__ __forceinline__ bool cand_before(uint64_t ra, const uint32_t* ta, uint64_t rb, const uint32_t* tb) {
  if (ra != rb) return ra < rb;
  if (ta[0] != tb[0]) return ta[0] < tb[0];
  if (ta[1] != tb[1]) return ta[1] < tb[1];
  return ta[2] < tb[2];
}

__global__ void __launch_bounds__(512, 1) k_vertex_topk(TopkArgs a) {
  extern __shared__ __align__(16) char smem[];
  __shared__ uint32_t s_misc[8];
  __shared__ uint32_t s_scan[32];
  uint32_t* hist = (uint32_t*)smem;                                   // 2049 (+pad) slice counts
  uint64_t* crank = (uint64_t*)(smem + 2064 * 4);                     // candidates: rank
  uint32_t* ctri = (uint32_t*)(crank + kTopkCap);                     // candidates: sorted triple
  uint32_t* tab = ctri + 3 * kTopkCap;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  while (true) {
    if (tid == 0) s_misc[0] = (uint32_t)atomicAdd(&a.sc->task[0], 1ull);
    __syncthreads();
    const uint32_t item = s_misc[0];
    if (item >= a.n_items) break;
    const uint32_t v = a.items[item];
    const bool ok = v < a.n;
    if (!ok && tid == 0) guard_fail(a.sc, kGuardVertex, v);
    const uint32_t rs = ok ? a.uptr[v] : 0u, deg = ok ? a.uptr[v + 1] - rs : 0u;
    const uint32_t chunk = a.cap / 4;
    uint32_t sstar = kTopkSlices - 1, below = 0;  // threshold slice, candidates in better slices
    for (int pass = 0; pass < 2; pass++) {
      if (pass == 0) {
        for (int i = tid; i < kTopkSlices; i += blockDim.x) hist[i] = 0;
        if (tid == 0) s_misc[2] = 0;  // pass 0 also keeps every triangle while they fit
      } else if (tid == 0) {
        s_misc[1] = 0;       // cursor of better slices
        s_misc[2] = below;   // cursor of the threshold slice
      }
      __syncthreads();
      const bool index_only = a.ix.mode != 0 && deg > chunk;  // a row longer than one table
      for (uint32_t c0 = 0; c0 < deg; c0 = index_only ? deg : c0 + chunk) {  // index_only: one pass
        const uint32_t c1 = index_only ? deg : min(deg, c0 + chunk);
        const uint32_t slots = slots_for(c1 - c0);
        const Table t = make_table(tab, a.cap, index_only ? 32u : slots);
        if (!index_only) {
          for (uint32_t i = tid; i < slots; i += blockDim.x) t.key[i] = kEmpty;
          __syncthreads();
          for (uint32_t i = c0 + tid; i < c1; i += blockDim.x) {
            const uint64_t e = a.uadj[rs + i];
            table_insert(t, adj_col(e), adj_valbits(e), rs + i, a.sc);
          }
        }
        __syncthreads();
        for (uint32_t j = wid; j < deg; j += nw) {
          const uint32_t pa = rs + j;
          if (pa + 1 >= rs + c1) continue;  // b must come after a in v's row
          const uint64_t ea = a.uadj[pa];
          const uint32_t av = adj_col(ea);
          const uint32_t qa = adj_valbits(ea);
          if (av >= a.n) {
            if (lane == 0) guard_fail(a.sc, kGuardVertex, av);
            continue;
          }
          // triangle v-av-w with P found: histogram and candidate while the
          // buffer has room (pass 0), or candidate of a slice up to the K-th's (pass 1)
          auto found = [&](long long P, uint32_t w) {
            const uint64_t r = topk_rank(P, a.which);
            const uint32_t sl = (uint32_t)(r >> 35);
            if (pass == 0) atomicAdd(&hist[sl], 1u);
            if (pass == 0 || sl <= sstar) {
              const uint32_t at = (pass == 0 || sl == sstar) ? atomicAdd(&s_misc[2], 1u) : atomicAdd(&s_misc[1], 1u);
              if (at < kTopkCap) {
                uint32_t x0 = v, x1 = av, x2 = w, tt;
                if (x0 > x1) { tt = x0; x0 = x1; x1 = tt; }
                if (x1 > x2) { tt = x1; x1 = x2; x2 = tt; }
                if (x0 > x1) { tt = x0; x0 = x1; x1 = tt; }
                crank[at] = r;
                ctri[3 * at] = x0;
                ctri[3 * at + 1] = x1;
                ctri[3 * at + 2] = x2;
              }
            }
          };
          const uint32_t s0 = a.uptr[av], s1 = a.uptr[av + 1];
          if (index_only) {
            index_pairs(a.ix, a.uadj, v, av, qa, pa, rs + deg, s0, s1 - s0, 0, lane, a.sc, found);
            continue;
          }
          const uint32_t b_lo = max(pa + 1, rs + c0), b_hi = rs + c1;
          if (use_index(a.ix, b_hi - b_lo, s1 - s0)) {
            // from v's side: b after a in this chunk, each pair looked up
            for (uint32_t b0 = b_lo; b0 < b_hi; b0 += 32) {
              const uint32_t pos = b0 + lane;
              const bool act = pos < b_hi;
              const uint64_t eb = act ? a.uadj[pos] : 0ull;
              uint32_t qab = 0;
              if (act && edge_index_find(a.ix, av, adj_col(eb), qab, a.sc))
                found((long long)((int32_t)qa * (int32_t)adj_valbits(eb)) * (long long)(int32_t)qab, adj_col(eb));
            }
            continue;
          }
          for (uint32_t b0 = s0; b0 < s1; b0 += 32) {
            const uint32_t pos = b0 + lane;
            const bool act = pos < s1;
            const uint64_t e = act ? a.uadj[pos] : 0ull;
            uint32_t qt = 0, pt = 0;
            const bool hit = act && table_find<true>(t, adj_col(e), qt, pt, a.sc) && pt > pa;
            if (hit) found((long long)((int32_t)qa * (int32_t)qt) * (long long)(int32_t)adj_valbits(e), adj_col(e));
          }
        }
        __syncthreads();
      }
      if (pass == 0) {
        // every triangle fitted the buffer: they are the candidates
        if (s_misc[2] <= (uint32_t)kTopkCap) break;
        // else the slice of the K-th best (more than kTopkCap >= K triangles,
        // so it exists): the first slice whose running count reaches K, by a
        // block-wide scan over contiguous runs of slices
        const uint32_t per = (kTopkSlices + blockDim.x - 1) / blockDim.x;
        const uint32_t i0 = min((uint32_t)kTopkSlices, tid * per), i1 = min((uint32_t)kTopkSlices, i0 + per);
        uint32_t mine = 0;
        for (uint32_t i = i0; i < i1; i++) mine += hist[i];
        uint32_t incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += y;
        }
        if (lane == 31) s_scan[wid] = incl;
        __syncthreads();
        if (wid == 0) {
          const uint32_t w0 = lane < nw ? s_scan[lane] : 0u;
          uint32_t wi = w0;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
          }
          if (lane < nw) s_scan[lane] = wi - w0;  // exclusive offset of each warp
        }
        __syncthreads();
        uint32_t acc = incl - mine + s_scan[wid];
        if (acc < a.K && acc + mine >= a.K) {
          for (uint32_t i = i0; i < i1; i++) {
            if (acc + hist[i] >= a.K) {
              s_misc[3] = i;
              s_misc[4] = acc;
              break;
            }
            acc += hist[i];
          }
        }
        __syncthreads();
        sstar = s_misc[3];
        below = s_misc[4];
      }
    }
    __syncthreads();
    const uint32_t ncand = min((uint32_t)kTopkCap, s_misc[2]);
    // sort the candidates by (rank, triple): bitonic network, mirror-first merges
    uint32_t cap2 = 2;
    while (cap2 < ncand) cap2 <<= 1;
    for (uint32_t kk = 2; kk <= cap2; kk <<= 1) {
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        for (uint32_t i = tid; i < cap2; i += blockDim.x) {
          const uint32_t ixj = (j == (kk >> 1)) ? (i ^ (kk - 1)) : (i ^ j);
          if (ixj > i && ixj < ncand && cand_before(crank[ixj], &ctri[3 * ixj], crank[i], &ctri[3 * i])) {
            const uint64_t r = crank[i];
            crank[i] = crank[ixj];
            crank[ixj] = r;
            for (int q = 0; q < 3; q++) {
              const uint32_t t2 = ctri[3 * i + q];
              ctri[3 * i + q] = ctri[3 * ixj + q];
              ctri[3 * ixj + q] = t2;
            }
          }
        }
        __syncthreads();
      }
    }
    const uint32_t nout = min(a.K, ncand);
    for (uint32_t i = tid; i < nout; i += blockDim.x) {
      ubt_tri_rec rec;
      rec.u = ctri[3 * i];
      rec.v = ctri[3 * i + 1];
      rec.w = ctri[3 * i + 2];
      rec.cls = (uint32_t)a.which;
      const long long P = a.which == 1 ? (long long)crank[i] - (1ll << 45) : (1ll << 45) - (long long)crank[i];
      rec.p_bal = (double)((1ll << 45) - P) * 0x1p-46;
      a.out[(size_t)item * a.K + i] = rec;
    }
    if (tid == 0) a.n_out[item] = (int32_t)nout;
    __syncthreads();
  }
}

}  // namespace

}  // namespace ubt

using namespace ubt;

extern "C" ubt_status ubt_edge_local_counts(ubt_graph* g, const uint32_t* d_edges, int64_t k, const double* h_tau,
                                            int32_t n_tau, int64_t* d_bal, int64_t* d_unbal, double* d_estimate,
                                            void* stream) {
  UBT_RANGE("ubt_edge_local_counts");
  return local_counts(g, d_edges, k, 0, h_tau, n_tau, d_bal, d_unbal, d_estimate, (cudaStream_t)stream);
}

extern "C" ubt_status ubt_vertex_local_counts(ubt_graph* g, const uint32_t* d_vertices, int64_t k,
                                              const double* h_tau, int32_t n_tau, int64_t* d_bal, int64_t* d_unbal,
                                              double* d_estimate, void* stream) {
  UBT_RANGE("ubt_vertex_local_counts");
  return local_counts(g, d_vertices, k, 1, h_tau, n_tau, d_bal, d_unbal, d_estimate, (cudaStream_t)stream);
}

extern "C" ubt_status ubt_vertex_topk(ubt_graph* g, const uint32_t* d_vertices, int64_t k, int32_t K, int32_t which,
                                      ubt_tri_rec* d_out, int32_t* d_n_out, void* stream) {
  UBT_RANGE("ubt_vertex_topk");
  if (!g || k < 0 || (k > 0 && (!d_vertices || !d_out || !d_n_out))) return UBT_ERR_INVALID_ARG;
  if (K < 1 || K > kTopkMax || (which != 1 && which != 2) || k >= 0xFFFFFFFFll) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_FIXED || !g->uptr) return UBT_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  TopkArgs a;
  a.uptr = g->uptr;
  a.uadj = g->uadj;
  a.ix = edge_index_of(g);
  a.items = d_vertices;
  a.n_items = (uint32_t)k;
  a.n = (uint32_t)g->n;
  a.m2 = (uint32_t)(2 * g->m);
  a.K = (uint32_t)K;
  a.which = which;
  a.cap = (uint32_t)std::min<int64_t>(table_slots(std::max<int64_t>(g->max_udeg, 2)),
                                      std::max<int64_t>(64, std::min<int64_t>(tuning().smem_table_max, 4096)));
  a.sc = g->scratch;
  a.out = d_out;
  a.n_out = d_n_out;
  UBT_CUDA(cudaMemsetAsync(a.sc, 0, kScratchHeader / 2, s));
  if (k == 0) return UBT_OK;
  const int threads = 512;
  const size_t smem = 2064 * 4 + (size_t)kTopkCap * (8 + 12) + (size_t)a.cap * 3 * 4;
  UBT_CUDA(cudaFuncSetAttribute(k_vertex_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  UBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vertex_topk, threads, smem));
  if (per_sm < 1) return UBT_ERR_INVALID_ARG;
  const int64_t blocks = std::min<int64_t>((int64_t)g->sm_count * per_sm, k);
  k_vertex_topk<<<(int)blocks, threads, smem, s>>>(a);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}
