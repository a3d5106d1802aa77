// ubt_build.cu -- building the graph the exact algorithms traverse.
//
//   validate   ids < n, no self-loops, probabilities in range       (Def. 1)
//   degree     undirected degree of every vertex
//   orient     each edge from its earlier endpoint in Node Order (degree,
//              then id) to the later one                (Def. Node Order, Sec. 4)
//   CSR        forward lists N>(u) as offsets + packed (neighbour, value)
//   sort       REAL graphs' lists by neighbour id (duplicates are equal
//              neighbours); FIXED graphs' lists by |q| descending, then id,
//              so that pruned entries (Lemma 2) form a suffix of every list,
//              after a duplicate check (a lane match or a hash set per list;
//              lists past the shared-memory limit are sorted by id first)
//   pairs      every forward edge x-s is a pair owned by one endpoint: the
//              one whose list becomes the hash table while the other
//              endpoint's list is streamed through it (the shorter list is
//              streamed); pairs grouped by owner
//   work lists owners (>= 2 forward entries, >= 1 pair) split by list length
//              and streamed work into block tasks and warp tasks, each
//              ordered by decreasing work
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "ubt_internal.cuh"

namespace ubt {

namespace {

constexpr int kSortHugeBlocks = 16;  // blocks sorting lists longer than that

// error word: lowest (edge index << 8 | code) wins, so the report is deterministic
__device__ inline void report(unsigned long long* err, uint64_t index, int code) {
  atomicMin(err, (unsigned long long)((index << 8) | (uint64_t)code));
}

__global__ void k_vertex_graph(const int64_t* __restrict__ voff, int64_t ng, int64_t n, uint32_t* vgraph) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = ng;  // find g with voff[g] <= v < voff[g+1]
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) / 2;
      if (voff[mid] <= v) lo = mid; else hi = mid;
    }
    vgraph[v] = (uint32_t)lo;
  }
}

// Adds 1 to ctr[key] for every lane with `on`, with one atomic per run of
// equal keys in consecutive lanes (edge lists sorted by source put a
// vertex's edges together, and one counter then takes every lane's add);
// returns the lane's slot: the counter's old value plus its rank in the run.
// All 32 lanes call it.
__device__ __forceinline__ uint32_t add_by_runs(uint32_t* ctr, uint32_t key, bool on) {
  const uint32_t lane = lane_id();
  const unsigned act = __ballot_sync(kFull, on);
  const uint32_t prev = __shfl_up_sync(kFull, key, 1);
  const bool head = on && !(lane > 0 && ((act >> (lane - 1)) & 1u) && prev == key);
  const unsigned heads = __ballot_sync(kFull, head);
  const unsigned upto = (2u << lane) - 1u;          // lanes 0..lane (all bits for lane 31)
  const unsigned after = (heads | ~act) & ~upto;     // where runs end, after this lane
  const uint32_t next = after ? (uint32_t)__ffs(after) - 1u : 32u;
  uint32_t old = 0;
  if (head) old = atomicAdd(&ctr[key], next - lane);
  const unsigned mine = heads & upto;
  const uint32_t my_head = mine ? 31u - (uint32_t)__clz(mine) : lane;
  return __shfl_sync(kFull, old, my_head) + (lane - my_head);
}

// Grid-stride loops over the edges in which every warp takes 32 consecutive
// edges per step, so that warp-wide runs (add_by_runs) see neighbours.
#define UBT_FOR_EDGE_WARPS(base, m)                                                                     \
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < (m);               \
       base += (int64_t)gridDim.x * blockDim.x)

__global__ void k_validate_degree(int64_t n, int64_t m, const uint32_t* __restrict__ src,
                                  const uint32_t* __restrict__ dst, const uint32_t* __restrict__ k,
                                  const float* __restrict__ p, const uint32_t* __restrict__ vgraph,
                                  uint32_t* __restrict__ deg, unsigned long long* err) {
  const uint32_t lane = lane_id();
  UBT_FOR_EDGE_WARPS(base, m) {
    const int64_t i = base + lane;
    bool ok = i < m;
    const uint32_t a = ok ? src[i] : 0u, b = ok ? dst[i] : 0u;
    if (ok && ((int64_t)a >= n || (int64_t)b >= n)) { report(err, i, -UBT_ERR_VERTEX_OOB); ok = false; }
    if (ok && a == b) { report(err, i, -UBT_ERR_SELF_LOOP); ok = false; }
    if (ok) {
      if (k) {
        if (k[i] > 65536u) report(err, i, -UBT_ERR_PROB_OOB);
      } else {
        const float x = p[i];
        if (!(x >= 0.0f && x <= 1.0f)) report(err, i, -UBT_ERR_PROB_OOB);
      }
      if (vgraph && vgraph[a] != vgraph[b]) { report(err, i, -UBT_ERR_INVALID_ARG); ok = false; }
    }
    add_by_runs(deg, a, ok);
    if (ok) atomicAdd(&deg[b], 1u);
  }
}

// Node Order: a before b iff (deg a, a) < (deg b, b)
__device__ inline bool node_before(const uint32_t* deg, uint32_t a, uint32_t b) {
  const uint32_t da = deg[a], db = deg[b];
  return da < db || (da == db && a < b);
}

__global__ void k_out_degree(int64_t m, const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                             const uint32_t* __restrict__ deg, uint32_t* __restrict__ outdeg) {
  const uint32_t lane = lane_id();
  UBT_FOR_EDGE_WARPS(base, m) {
    const int64_t i = base + lane;
    const bool on = i < m;
    const uint32_t a = on ? src[i] : 0u, b = on ? dst[i] : 0u;
    add_by_runs(outdeg, on && node_before(deg, a, b) ? a : b, on);
  }
}

__global__ void k_scatter(int64_t m, const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                          const uint32_t* __restrict__ k, const float* __restrict__ p,
                          const uint32_t* __restrict__ deg, const uint32_t* __restrict__ row_ptr,
                          uint32_t* __restrict__ fill, uint64_t* __restrict__ adj, uint32_t* __restrict__ eid,
                          const uint32_t* __restrict__ key_in, uint32_t* __restrict__ key_out) {
  const uint32_t lane = lane_id();
  UBT_FOR_EDGE_WARPS(base, m) {
    const int64_t i = base + lane;
    const bool on = i < m;
    const uint32_t a = on ? src[i] : 0u, b = on ? dst[i] : 0u;
    const bool ab = on && node_before(deg, a, b);
    const uint32_t lo = ab ? a : b, hi = ab ? b : a;
    const uint32_t slot = add_by_runs(fill, lo, on);
    if (!on) continue;
    const uint32_t pos = row_ptr[lo] + slot;
    uint32_t val;
    if (k) {
      val = (uint32_t)(int32_t)(32768 - (int32_t)k[i]);     // q = 32768 - k
    } else {
      val = real_valbits(p[i]);
    }
    adj[pos] = adj_pack(hi, val);
    eid[pos] = (uint32_t)i;
    if (key_out) key_out[pos] = key_in[i];
  }
}

// sort keys: by neighbour id (REAL rows); by (32768 - |q|, id) (FIXED and undirected rows)
__device__ inline uint64_t key_by_col(uint64_t e) { return (uint64_t)adj_col(e); }
__device__ inline uint64_t key_by_absq(uint64_t e) {
  const int32_t q = adj_q(e);
  const uint32_t aq = (uint32_t)(q < 0 ? -q : q);
  return ((uint64_t)(32768u - aq) << 32) | adj_col(e);
}

// How a row is sorted: REAL forward rows by neighbour id (a duplicate edge
// shows as two equal neighbouring keys); FIXED forward rows by (|q|
// descending, id) with duplicates found by a hash set or a lane match before
// the one sort; undirected rows like FIXED ones but unchecked (the forward
// rows of the same edges were checked first).
enum : int { kSortById = 0, kSortByAbsqChecked = 1, kSortByAbsq = 2 };

constexpr unsigned long long kSetEmpty = ~0ull;

// Inserts (col, input edge id) into an open-addressing set of mask + 1
// 64-bit slots (at least twice the row); a second entry with the same
// neighbour is a duplicate edge, reported with the larger of the two ids.
__device__ __forceinline__ void dedupe_insert(unsigned long long* set, uint32_t mask, uint32_t col, uint32_t id,
                                              unsigned long long* err) {
  const unsigned long long mine = ((unsigned long long)col << 32) | id;
  uint32_t h = ((col * 0x9E3779B1u) >> 8) & mask;
  for (uint32_t it = 0; it <= mask; it++) {
    const unsigned long long cur = atomicCAS(&set[h], kSetEmpty, mine);
    if (cur == kSetEmpty) return;
    if ((uint32_t)(cur >> 32) == col) {
      report(err, max(id, (uint32_t)cur), -UBT_ERR_DUPLICATE_EDGE);
      return;
    }
    h = (h + 1) & mask;
  }
}

// Lists of <= 32 entries: one warp per list, bitonic network over the lanes.
// Bitonic sort of the values held by each aligned group of W lanes (W = 8,
// 16 or 32), ascending by key within every group.
template <int W>
__device__ __forceinline__ void group_bitonic(uint64_t& key, uint64_t& e, uint32_t& id, uint32_t& ky, int lane) {
  const int li = lane & (W - 1);
#pragma unroll
  for (int kk = 2; kk <= W; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const uint64_t ok = __shfl_xor_sync(kFull, key, j);
      const uint64_t oe = __shfl_xor_sync(kFull, e, j);
      const uint32_t oi = __shfl_xor_sync(kFull, id, j);
      const uint32_t oy = __shfl_xor_sync(kFull, ky, j);
      const bool up = (li & kk) == 0;
      const bool lower = (li & j) == 0;
      const bool take_min = (lower == up);
      const bool sw = take_min ? (ok < key) : (ok > key);
      if (sw) { key = ok; e = oe; id = oi; ky = oy; }
    }
  }
}

// Sorts the rows of one group of W lanes (row rs..rs+len, len <= W; groups
// without a row pass in = false everywhere), as `mode` says.
template <int W>
__device__ __forceinline__ void sort_group_row(uint64_t* adj, uint32_t* eid, uint32_t* ekey, uint32_t rs, uint32_t len,
                                               bool row, int mode, unsigned long long* err, int lane) {
  const int li = lane & (W - 1);
  const bool in = row && (uint32_t)li < len;
  uint64_t e = in ? adj[rs + li] : ~0ull;
  uint32_t id = in ? eid[rs + li] : 0u;
  uint32_t ky = (in && ekey) ? ekey[rs + li] : 0u;
  if (mode == kSortById) {
    uint64_t key = in ? key_by_col(e) : ~0ull;
    group_bitonic<W>(key, e, id, ky, lane);
    const uint64_t prev = __shfl_up_sync(kFull, key, 1);
    if (in && li > 0 && prev == key) report(err, rs + li, -UBT_ERR_DUPLICATE_EDGE);
  } else {
    if (mode == kSortByAbsqChecked) {  // lanes of one group holding the same neighbour
      const unsigned long long v = in ? (((unsigned long long)(lane / W) << 32) | adj_col(e))
                                      : ((0xFFFFFFFFull << 32) | (unsigned long long)lane);
      const unsigned others = __match_any_sync(kFull, v) & ~(1u << lane);
      const uint32_t oid = __shfl_sync(kFull, id, others ? __ffs(others) - 1 : lane);
      if (in && others) report(err, max(id, oid), -UBT_ERR_DUPLICATE_EDGE);
    }
    uint64_t key = in ? key_by_absq(e) : ~0ull;
    group_bitonic<W>(key, e, id, ky, lane);
  }
  if (in) {
    adj[rs + li] = e;
    eid[rs + li] = id;
    if (ekey) ekey[rs + li] = ky;
  }
}

// Rows of 2..32 entries: a warp takes 4 consecutive rows; the rows of at
// most 8 entries are sorted together, one per 8-lane group, the others one
// after another by the whole warp.
__global__ void k_sort_short_rows(int64_t n, const uint32_t* __restrict__ row_ptr, uint64_t* adj, uint32_t* eid,
                                  uint32_t* ekey, int mode, unsigned long long* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u0 = 4 * (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)); u0 < n; u0 += 4 * warps) {
    const int64_t u = u0 + (lane >> 3);
    uint32_t rs = 0, len = 0;
    if (u < n) {
      rs = row_ptr[u];
      len = row_ptr[u + 1] - rs;
    }
    sort_group_row<8>(adj, eid, ekey, rs, len, len >= 2 && len <= 8, mode, err, lane);
    unsigned big = __ballot_sync(kFull, (lane & 7) == 0 && len > 8 && len <= 32);
    while (big) {
      const int g = __ffs(big) - 1;
      big &= big - 1;
      const uint32_t rsg = __shfl_sync(kFull, rs, g), leng = __shfl_sync(kFull, len, g);
      sort_group_row<32>(adj, eid, ekey, rsg, leng, true, mode, err, lane);
    }
  }
}

// Rows of 33..512 entries: one warp per row, R = 4, 8 or 16 words per lane
// (entry r * 32 + lane in register r).  A word is the sort key << 12 | the
// entry's position in the row; the words are distinct, so a bitonic network
// over registers and lanes moves one word per comparator, and the entries are
// gathered by position once at the end.
template <int R>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&k)[R], int lane) {
#pragma unroll
  for (int kk = 2; kk <= 32 * R; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j >= 32) {  // partner in another register of the same lane
        const int rj = j >> 5;
#pragma unroll
        for (int r = 0; r < R; r++) {
          if ((r & rj) == 0) {
            const unsigned long long a = k[r], b = k[r | rj];
            const bool asc = (((r << 5) | lane) & kk) == 0;
            k[r] = (a < b) == asc ? a : b;
            k[r | rj] = (a < b) == asc ? b : a;
          }
        }
      } else {        // partner in another lane, same register
#pragma unroll
        for (int r = 0; r < R; r++) {
          const unsigned long long o = __shfl_xor_sync(kFull, k[r], j);
          const bool up = (((r << 5) | lane) & kk) == 0;
          const bool take_min = ((lane & j) == 0) == up;
          k[r] = take_min ? (o < k[r] ? o : k[r]) : (o > k[r] ? o : k[r]);
        }
      }
    }
  }
}

template <int R>
__device__ __forceinline__ void sort_row_warp(uint64_t* adj, uint32_t* eid, uint32_t* ekey, uint32_t rs, uint32_t len,
                                              int mode, unsigned long long* set, unsigned long long* err, int lane) {
  unsigned long long k[R];
  if (mode == kSortById) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t i = (uint32_t)(r * 32 + lane);
      k[r] = i < len ? (key_by_col(adj[rs + i]) << 12) | i : ~0ull;
    }
    warp_bitonic<R>(k, lane);
#pragma unroll
    for (int r = 0; r < R; r++) {  // duplicates: equal neighbours at adjacent sorted positions
      const unsigned long long up1 = __shfl_up_sync(kFull, k[r], 1);
      const unsigned long long last = __shfl_sync(kFull, k[r > 0 ? r - 1 : 0], 31);
      const unsigned long long prev = lane > 0 ? up1 : last;
      const uint32_t i = (uint32_t)(r * 32 + lane);
      if (i < len && i > 0 && (prev >> 12) == (k[r] >> 12)) report(err, rs + i, -UBT_ERR_DUPLICATE_EDGE);
    }
  } else {
    if (mode == kSortByAbsqChecked) {  // this warp's set: 64 R slots for at most 32 R entries
      for (int i = lane; i < 64 * R; i += 32) set[i] = kSetEmpty;
      __syncwarp();
#pragma unroll
      for (int r = 0; r < R; r++) {
        const uint32_t i = (uint32_t)(r * 32 + lane);
        if (i < len) dedupe_insert(set, 64 * R - 1, adj_col(adj[rs + i]), eid[rs + i], err);
      }
      __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t i = (uint32_t)(r * 32 + lane);
      k[r] = i < len ? (key_by_absq(adj[rs + i]) << 12) | i : ~0ull;
    }
    warp_bitonic<R>(k, lane);
  }
  // gather by position, one array at a time: every lane reads its entries'
  // sources before any lane of the warp overwrites that array
  uint32_t pw[(R + 1) / 2];  // two 12-bit positions per register
#pragma unroll
  for (int r = 0; r < R; r += 2)
    pw[r / 2] = (uint32_t)(k[r] & 0xFFFu) | (r + 1 < R ? (uint32_t)(k[r + 1] & 0xFFFu) << 16 : 0u);
#define UBT_POS(r) ((r) & 1 ? pw[(r) / 2] >> 16 : pw[(r) / 2] & 0xFFFFu)
#pragma unroll
  for (int r = 0; r < R; r++)
    if ((uint32_t)(r * 32 + lane) < len) k[r] = adj[rs + UBT_POS(r)];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; r++)
    if ((uint32_t)(r * 32 + lane) < len) adj[rs + r * 32 + lane] = k[r];
  uint32_t v[R];
#pragma unroll
  for (int r = 0; r < R; r++)
    if ((uint32_t)(r * 32 + lane) < len) v[r] = eid[rs + UBT_POS(r)];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; r++)
    if ((uint32_t)(r * 32 + lane) < len) eid[rs + r * 32 + lane] = v[r];
  if (ekey) {
#pragma unroll
    for (int r = 0; r < R; r++)
      if ((uint32_t)(r * 32 + lane) < len) v[r] = ekey[rs + UBT_POS(r)];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; r++)
      if ((uint32_t)(r * 32 + lane) < len) ekey[rs + r * 32 + lane] = v[r];
  }
#undef UBT_POS
}

// One launch per R takes the rows of the list with 16 R < len <= 32 R (R = 4:
// every row up to 128 entries) and leaves the others to the other launches.
template <int R>
__global__ void k_sort_mid_rows(const uint32_t* __restrict__ rows, uint32_t nrows, const uint32_t* __restrict__ row_ptr,
                                uint64_t* adj, uint32_t* eid, uint32_t* ekey, int mode, unsigned long long* err) {
  extern __shared__ __align__(16) unsigned long long sets[];  // one set of 64 R slots per warp (checked mode)
  unsigned long long* set = sets + (threadIdx.x >> 5) * (64 * R);
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r0 = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r0 < nrows; r0 += warps) {
    const uint32_t u = rows[r0];
    const uint32_t rs = row_ptr[u], len = row_ptr[u + 1] - rs;
    if (len > 32u * R || (R > 4 && len <= 16u * R)) continue;
    sort_row_warp<R>(adj, eid, ekey, rs, len, mode, set, err, lane);
  }
}

// the warp sorts of every row of the list (lengths 33..warp_max)
template <int R>
ubt_status launch_mid_sort(const uint32_t* rows, uint32_t nrows, const uint32_t* row_ptr, uint64_t* adj, uint32_t* eid,
                           uint32_t* ekey, int mode, unsigned long long* err, int g, int thr, cudaStream_t s) {
  const size_t smem = mode == kSortByAbsqChecked ? (size_t)(thr / 32) * 64 * R * 8 : 0;
  UBT_CUDA(cudaFuncSetAttribute(k_sort_mid_rows<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sort_mid_rows<R><<<g, thr, smem, s>>>(rows, nrows, row_ptr, adj, eid, ekey, mode, err);
  return UBT_OK;
}

ubt_status launch_mid_sorts(const uint32_t* rows, uint32_t nrows, const uint32_t* row_ptr, uint64_t* adj,
                            uint32_t* eid, uint32_t* ekey, int mode, unsigned long long* err, uint32_t warp_max,
                            int sms, int thr, cudaStream_t s) {
  const int g = (int)std::min<unsigned long long>((nrows + 7) / 8, (unsigned long long)sms * 32);
  ubt_status st = launch_mid_sort<4>(rows, nrows, row_ptr, adj, eid, ekey, mode, err, g, thr, s);
  if (st == UBT_OK && warp_max >= 256) st = launch_mid_sort<8>(rows, nrows, row_ptr, adj, eid, ekey, mode, err, g, thr, s);
  if (st == UBT_OK && warp_max >= 512)
    st = launch_mid_sort<16>(rows, nrows, row_ptr, adj, eid, ekey, mode, err, g, thr, s);
  return st;
}

// Lists longer than the "warp_sort_max" tuning (256) and at most
// "sort_smem_max" (4096): one block per list sorts 64-bit words (sort key <<
// 12 | position in the list) in shared memory; the keys are distinct by
// construction, so the network only moves one word per comparator, and the
// entries are gathered by position once at the end.
constexpr int kPackedSortThreads = 512;
constexpr int kPackedPerThread = 8;                  // 4096 entries / 512 threads
constexpr uint32_t kPackedMax = kPackedSortThreads * kPackedPerThread;

// ascending bitonic network over pk[0..cap), cap a power of two
__device__ __forceinline__ void bitonic_packed(unsigned long long* pk, uint32_t cap) {
  for (uint32_t kk = 2; kk <= cap; kk <<= 1) {
    for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
      for (uint32_t t = threadIdx.x; t < (cap >> 1); t += blockDim.x) {
        const uint32_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // the comparator's lower index
        const uint32_t ixj = i | j;
        const unsigned long long a = pk[i], b = pk[ixj];
        const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
        const bool asc = (i & kk) == 0;
        pk[i] = asc ? lo : hi;
        pk[ixj] = asc ? hi : lo;
      }
      __syncthreads();
    }
  }
}

// One launch per class takes the rows of the list with lo < len <= hi, with
// hi / 2 threads (at most 512): every thread has a comparator at every stage.
__global__ void __launch_bounds__(kPackedSortThreads)
k_sort_long_rows_packed(const uint32_t* __restrict__ rows, uint32_t nrows, const uint32_t* __restrict__ row_ptr,
                        uint64_t* adj, uint32_t* eid, uint32_t* ekey, int mode, unsigned long long* err,
                        uint32_t lo, uint32_t hi) {
  extern __shared__ __align__(16) unsigned long long pk[];  // hi words, then (checked mode) a set of 2 hi slots
  unsigned long long* set = pk + hi;
  for (uint32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const uint32_t u = rows[r];
    const uint32_t rs = row_ptr[u], len = row_ptr[u + 1] - rs;
    if (len <= lo || len > hi) continue;
    if (len > kPackedMax || len > kPackedPerThread * blockDim.x) {  // the launches never give such a row here
      if (threadIdx.x == 0) report(err, rs, -UBT_ERR_INVALID_ARG);
      continue;
    }
    uint32_t cap = 64;
    while (cap < len) cap <<= 1;
    if (mode == kSortById) {
      for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x)
        pk[i] = i < len ? (key_by_col(adj[rs + i]) << 12) | i : ~0ull;
      __syncthreads();
      bitonic_packed(pk, cap);
      for (uint32_t i = threadIdx.x + 1; i < len; i += blockDim.x)
        if ((pk[i] >> 12) == (pk[i - 1] >> 12)) report(err, rs + i, -UBT_ERR_DUPLICATE_EDGE);
    } else {
      if (mode == kSortByAbsqChecked) {  // 2 cap <= 2 hi slots
        for (uint32_t i = threadIdx.x; i < 2 * cap; i += blockDim.x) set[i] = kSetEmpty;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
          dedupe_insert(set, 2 * cap - 1, adj_col(adj[rs + i]), eid[rs + i], err);
      }
      for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x)
        pk[i] = i < len ? (key_by_absq(adj[rs + i]) << 12) | i : ~0ull;
      __syncthreads();
      bitonic_packed(pk, cap);
    }
    // gather every entry's sources before any thread overwrites the list
    uint64_t e[kPackedPerThread];
    uint32_t d[kPackedPerThread], y[kPackedPerThread];
#pragma unroll
    for (int c = 0; c < kPackedPerThread; c++) {
      const uint32_t i = threadIdx.x + c * blockDim.x;
      if (i < len) {
        const uint32_t w = (uint32_t)(pk[i] & 0xFFFu);
        e[c] = adj[rs + w];
        d[c] = eid[rs + w];
        y[c] = ekey ? ekey[rs + w] : 0u;
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kPackedPerThread; c++) {
      const uint32_t i = threadIdx.x + c * blockDim.x;
      if (i < len) {
        adj[rs + i] = e[c];
        eid[rs + i] = d[c];
        if (ekey) ekey[rs + i] = y[c];
      }
    }
    __syncthreads();
  }
}

// the block sorts of every row of the list (lengths warp_max + 1 .. smem_max),
// by class: (128, 256] with 128 threads, (256, 512] with 256, longer with 512
ubt_status launch_block_sorts(const uint32_t* rows, uint32_t nrows, const uint32_t* row_ptr, uint64_t* adj, uint32_t* eid,
                        uint32_t* ekey, int mode, unsigned long long* err, uint32_t warp_max, uint32_t smem_max,
                        int sms, cudaStream_t s) {
  const uint32_t bounds[4] = {128, 256, 512, kPackedMax};
  for (int c = 0; c < 3; c++) {
    const uint32_t lo = bounds[c], hi = c == 2 ? std::max(smem_max, 512u) : bounds[c + 1];
    if (hi <= warp_max || lo >= smem_max) continue;
    const int threads = (int)std::min<uint32_t>(hi / 2, kPackedSortThreads);
    const size_t smem = (size_t)hi * 8 * (mode == kSortByAbsqChecked ? 3 : 1);
    UBT_CUDA(cudaFuncSetAttribute(k_sort_long_rows_packed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int per_sm = std::max(1, std::min(2048 / threads, (int)(200 * 1024 / smem)));
    const int g = (int)std::min<unsigned long long>(nrows, (unsigned long long)sms * per_sm);
    k_sort_long_rows_packed<<<g, threads, smem, s>>>(rows, nrows, row_ptr, adj, eid, ekey, mode, err, lo, hi);
  }
  return UBT_OK;
}

// Longer lists: one block per list, bitonic network in a per-block global
// slice (lists longer than the "sort_smem_max" tuning).
template <bool kGlobal>
__global__ void k_sort_long_rows(const uint32_t* __restrict__ rows, uint32_t nrows, const uint32_t* __restrict__ row_ptr,
                                 uint64_t* adj, uint32_t* eid, uint32_t* ekey, int fixed, unsigned long long* err,
                                 char* gtmp, int64_t gtmp_cap) {
  extern __shared__ __align__(16) char sm[];
  for (uint32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const uint32_t u = rows[r];
    const uint32_t rs = row_ptr[u], re = row_ptr[u + 1];
    const uint32_t len = re - rs;
    uint32_t cap = 64;
    while (cap < len) cap <<= 1;
    char* base = kGlobal ? gtmp + (size_t)blockIdx.x * (size_t)gtmp_cap * 24 : sm;
    uint64_t* key = (uint64_t*)base;
    uint64_t* ev = key + cap;
    uint32_t* iv = (uint32_t*)(ev + cap);
    uint32_t* yv = iv + cap;
    for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) {
      if (i < len) {
        ev[i] = adj[rs + i];
        iv[i] = eid[rs + i];
        yv[i] = ekey ? ekey[rs + i] : 0u;
        key[i] = key_by_col(ev[i]);
      } else {
        key[i] = ~0ull; ev[i] = ~0ull; iv[i] = 0; yv[i] = 0;
      }
    }
    __syncthreads();
    for (int pass = 0; pass < (fixed ? 2 : 1); pass++) {
      if (pass == 1) {
        for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) key[i] = i < len ? key_by_absq(ev[i]) : ~0ull;
        __syncthreads();
      }
      for (uint32_t kk = 2; kk <= cap; kk <<= 1) {
        for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
          for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) {
            const uint32_t ixj = i ^ j;
            if (ixj > i) {
              const bool asc = (i & kk) == 0;
              const uint64_t a = key[i], b = key[ixj];
              if ((a > b) == asc && a != b) {
                key[i] = b; key[ixj] = a;
                uint64_t te = ev[i]; ev[i] = ev[ixj]; ev[ixj] = te;
                uint32_t ti = iv[i]; iv[i] = iv[ixj]; iv[ixj] = ti;
                uint32_t ty = yv[i]; yv[i] = yv[ixj]; yv[ixj] = ty;
              }
            }
          }
          __syncthreads();
        }
      }
      if (pass == 0) {
        for (uint32_t i = threadIdx.x + 1; i < len; i += blockDim.x)
          if (key[i] == key[i - 1]) report(err, rs + i, -UBT_ERR_DUPLICATE_EDGE);
        __syncthreads();
      }
    }
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
      adj[rs + i] = ev[i];
      eid[rs + i] = iv[i];
      if (ekey) ekey[rs + i] = yv[i];
    }
    __syncthreads();
  }
}

// Rows longer than 32: counts[2] of 33..128, or up to warp_max and at most
// smem_max (warp sort, listed from the end of `mid`), counts[0] of the others
// up to smem_max (block sort in shared memory, from the start of `mid`),
// counts[1] longer (block sort in global memory, `huge`).
__global__ void k_collect_long(int64_t n, const uint32_t* __restrict__ row_ptr, uint32_t smem_max, uint32_t warp_max,
                               uint32_t* mid, uint32_t* huge, unsigned long long* counts) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t len = row_ptr[u + 1] - row_ptr[u];
    if (len <= 32) continue;
    if (len <= 128 || (len <= warp_max && len <= smem_max))
      mid[n - 1 - (int64_t)atomicAdd(&counts[2], 1ull)] = (uint32_t)u;
    else if (len <= smem_max) mid[atomicAdd(&counts[0], 1ull)] = (uint32_t)u;
    else huge[atomicAdd(&counts[1], 1ull)] = (uint32_t)u;
  }
}

// Owner of the pair of forward edge u -> v (u before v in Node Order, du and
// dv their forward-list lengths).  Alg. 1 probes every w of N>(v) in a table
// of N>(u) ("push", owner u).  Probing N>(u) in a table of N>(v) ("pull",
// owner v) intersects the same two lists, so the triangle {u, v, w} is still
// found exactly once, from its two earliest vertices; pull is taken when it
// streams the shorter list.
__device__ inline uint32_t pair_owner(uint32_t u, uint32_t v, uint32_t du, uint32_t dv, int pull) {
  return (pull && dv > du) ? v : u;
}

// rowid[p] = the row that holds CSR position p (one thread per row)
__global__ void k_row_ids(int64_t n, const uint32_t* __restrict__ row_ptr, uint32_t* __restrict__ rowid) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    for (uint32_t p = row_ptr[u]; p < row_ptr[u + 1]; p++) rowid[p] = (uint32_t)u;
}

// pairs per owner, one lane per forward entry (rowid: the row of every CSR
// position; adjacent entries of one row that keep their owner share one
// atomic); also the oriented wedges sum_u sum_{v in N>(u)} |N>(v)| (Alg. 1's
// probes), one atomic per block
__global__ void k_pair_count(int64_t m, const uint32_t* __restrict__ row_ptr, const uint64_t* __restrict__ adj,
                             const uint32_t* __restrict__ rowid, int pull, uint32_t* __restrict__ pcount,
                             unsigned long long* wedges) {
  __shared__ unsigned long long s_w;
  if (threadIdx.x == 0) s_w = 0;
  __syncthreads();
  const uint32_t lane = lane_id();
  unsigned long long wsum = 0;
  UBT_FOR_EDGE_WARPS(base, m) {
    const int64_t i = base + lane;
    const bool on = i < m;
    uint32_t x = 0;
    if (on) {
      const uint32_t u = rowid[i], v = adj_col(adj[i]);
      const uint32_t du = row_ptr[u + 1] - row_ptr[u], dv = row_ptr[v + 1] - row_ptr[v];
      wsum += dv;
      x = pair_owner(u, v, du, dv, pull);
    }
    add_by_runs(pcount, x, on);
  }
  atomicAdd(&s_w, wsum);
  __syncthreads();
  if (threadIdx.x == 0 && s_w) atomicAdd(wedges, s_w);
}

// ctr[key] += val over the active lanes, one atomic per run of adjacent
// active lanes with equal keys (the run's sum from a warp prefix sum)
__device__ __forceinline__ void sum_by_runs(unsigned long long* ctr, uint32_t key, unsigned long long val, bool on) {
  const uint32_t lane = lane_id();
  const unsigned act = __ballot_sync(kFull, on);
  const uint32_t prev = __shfl_up_sync(kFull, key, 1);
  const bool head = on && !(lane > 0 && ((act >> (lane - 1)) & 1u) && prev == key);
  const unsigned heads = __ballot_sync(kFull, head);
  const unsigned upto = (2u << lane) - 1u;
  const unsigned after = (heads | ~act) & ~upto;
  const uint32_t next = after ? (uint32_t)__ffs(after) - 1u : 32u;  // > lane
  unsigned long long x = on ? val : 0ull;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long y = __shfl_up_sync(kFull, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  const unsigned long long end = __shfl_sync(kFull, x, (int)(next - 1u));
  const unsigned long long before = __shfl_sync(kFull, x, (int)((lane + 31u) & 31u));
  if (head) atomicAdd(&ctr[key], end - (lane > 0 ? before : 0ull));
}

// pair words grouped by owner: the streamed vertex and the edge's CSR
// position; work[x] += length of the streamed list (the owner's task size)
__global__ void k_pair_fill(int64_t m, const uint32_t* __restrict__ row_ptr, const uint64_t* __restrict__ adj,
                            const uint32_t* __restrict__ rowid, int pull, const uint32_t* __restrict__ pair_ptr,
                            uint32_t* __restrict__ pfill, uint64_t* __restrict__ pairs,
                            unsigned long long* __restrict__ work) {
  const uint32_t lane = lane_id();
  UBT_FOR_EDGE_WARPS(base, m) {
    const int64_t i = base + lane;
    const bool on = i < m;
    uint32_t x = 0, streamed = 0, slen = 0;
    if (on) {
      const uint32_t u = rowid[i], v = adj_col(adj[i]);
      const uint32_t du = row_ptr[u + 1] - row_ptr[u], dv = row_ptr[v + 1] - row_ptr[v];
      x = pair_owner(u, v, du, dv, pull);
      streamed = x == u ? v : u;
      slen = x == u ? dv : du;
    }
    const uint32_t slot = add_by_runs(pfill, x, on);
    if (on) pairs[pair_ptr[x] + slot] = ((uint64_t)i << 32) | streamed;
    sum_by_runs(work, x, slen, on);
  }
}

// Task classes (by the owner's list length and streamed work)
enum : uint8_t { kClsMedium = 1, kClsHub = 2, kClsGiant = 3 };
constexpr uint8_t kNoTask = 0xFF;
constexpr int kLgMax = 47;  // work buckets 2^0 .. 2^47
constexpr int kBuckets2 = 4 * (kLgMax + 1);

// Per owner x (one thread): its streamed work (from k_pair_fill), the log2
// bucket and class; bucket[x] = lg * 4 + cls, or kNoTask (fewer than 2 list
// entries or no pairs: no triangle can be found there).  Per-block counts in
// shared memory, one global atomic per block and bucket.
// stats: [1] longest list, [2] longest list of a block task, [3] streamed
//        work of all pairs, [4 + lg * 4 + cls] bucket sizes ([0] is set by
//        k_pair_count)
__global__ void k_row_stats(int64_t n, const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ pair_ptr,
                            const unsigned long long* __restrict__ work, uint32_t hub_thr, uint32_t giant_thr,
                            unsigned long long block_work, uint8_t* __restrict__ bucket,
                            unsigned long long* stats) {
  __shared__ uint32_t s_cnt[kBuckets2];
  __shared__ unsigned long long s_work;
  __shared__ uint32_t s_max, s_hmax;
  for (int i = threadIdx.x; i < kBuckets2; i += blockDim.x) s_cnt[i] = 0;
  if (threadIdx.x == 0) { s_work = 0; s_max = 0; s_hmax = 0; }
  __syncthreads();
  unsigned long long wsum = 0;
  uint32_t mx = 0, hmx = 0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t len = row_ptr[x + 1] - row_ptr[x];
    const uint32_t np = pair_ptr[x + 1] - pair_ptr[x];
    const unsigned long long w = np ? work[x] : 0ull;
    uint8_t b = kNoTask;
    if (len >= 2 && np > 0) {
      const int cls = len > giant_thr ? kClsGiant : ((len > hub_thr || w > block_work) ? kClsHub : kClsMedium);
      int lg = w ? 63 - __clzll(w) : 0;
      lg = lg > kLgMax ? kLgMax : lg;
      b = (uint8_t)(lg * 4 + cls);
      atomicAdd(&s_cnt[b], 1u);
      if (cls == kClsHub) hmx = max(hmx, len);
    }
    bucket[x] = b;
    wsum += w;
    mx = max(mx, len);
  }
  atomicAdd(&s_work, wsum);
  atomicMax(&s_max, mx);
  atomicMax(&s_hmax, hmx);
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets2; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&stats[4 + i], (unsigned long long)s_cnt[i]);
  if (threadIdx.x == 0) {
    atomicAdd(&stats[3], s_work);
    atomicMax(&stats[1], (unsigned long long)s_max);
    atomicMax(&stats[2], (unsigned long long)s_hmax);
  }
}

// Task lists: every block ranks its owners per bucket in shared memory and
// reserves one range per bucket with a single global atomic.
__global__ void k_fill_lists(int64_t n, const uint8_t* __restrict__ bucket, unsigned long long* cursor,
                             uint32_t* __restrict__ lists) {
  __shared__ uint32_t s_cnt[kBuckets2];
  __shared__ unsigned long long s_base[kBuckets2];
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    for (int i = threadIdx.x; i < kBuckets2; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    const int64_t x = base + threadIdx.x;
    const uint8_t b = x < n ? bucket[x] : kNoTask;
    uint32_t rank = 0;
    if (b != kNoTask) rank = atomicAdd(&s_cnt[b], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets2; i += blockDim.x)
      if (s_cnt[i]) s_base[i] = atomicAdd(&cursor[i], (unsigned long long)s_cnt[i]);
    __syncthreads();
    if (b != kNoTask) lists[s_base[b] + rank] = (uint32_t)x;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- undirected AEO adjacency

// both directions of every edge, in row order of arrival (sorted below)
__global__ void k_uscatter(int64_t m, const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                           const uint32_t* __restrict__ k, const uint32_t* __restrict__ uptr,
                           uint32_t* __restrict__ ufill, uint64_t* __restrict__ uadj, uint32_t* __restrict__ ueid) {
  const uint32_t lane = lane_id();
  UBT_FOR_EDGE_WARPS(base, m) {
    const int64_t i = base + lane;
    const bool on = i < m;
    const uint32_t a = on ? src[i] : 0u, b = on ? dst[i] : 0u;
    const uint32_t sa = add_by_runs(ufill, a, on);
    if (!on) continue;
    const uint32_t val = (uint32_t)(int32_t)(32768 - (int32_t)k[i]);
    const uint32_t pa = uptr[a] + sa;
    const uint32_t pb = uptr[b] + atomicAdd(&ufill[b], 1u);
    uadj[pa] = adj_pack(b, val);
    ueid[pa] = (uint32_t)i;
    uadj[pb] = adj_pack(a, val);
    ueid[pb] = (uint32_t)i;
  }
}

// Rows longer than the shared-memory sort limit: one block per row, sorted
// in place in global memory by a bitonic network whose comparators all put
// the smaller key first (the first comparator of every merge pairs i with its
// mirror i ^ (kk - 1)); positions >= len act as +infinity, so comparators
// that touch them never swap and are skipped.
__global__ void k_sort_rows_inplace(const uint32_t* __restrict__ rows, uint32_t nrows,
                                    const uint32_t* __restrict__ row_ptr, uint64_t* adj, uint32_t* eid) {
  for (uint32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const uint32_t u = rows[r];
    const uint32_t rs = row_ptr[u], len = row_ptr[u + 1] - rs;
    uint32_t cap = 2;
    while (cap < len) cap <<= 1;
    for (uint32_t kk = 2; kk <= cap; kk <<= 1) {
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) {
          const uint32_t ixj = (j == (kk >> 1)) ? (i ^ (kk - 1)) : (i ^ j);
          if (ixj > i && ixj < len) {
            const uint64_t a = adj[rs + i], b = adj[rs + ixj];
            if (key_by_absq(a) > key_by_absq(b)) {
              adj[rs + i] = b;
              adj[rs + ixj] = a;
              const uint32_t t = eid[rs + i];
              eid[rs + i] = eid[rs + ixj];
              eid[rs + ixj] = t;
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

// epos[2e + side] = position of edge e in the row of its smaller (side 0) or
// larger (side 1) endpoint; then umir[p] = the other one.  One warp per row.
__global__ void k_uepos(int64_t n, const uint32_t* __restrict__ uptr, const uint64_t* __restrict__ uadj,
                        const uint32_t* __restrict__ ueid, uint32_t* __restrict__ epos) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps)
    for (uint32_t p = uptr[x] + lane; p < uptr[x + 1]; p += 32)
      epos[2 * (size_t)ueid[p] + ((uint32_t)x > adj_col(uadj[p]) ? 1 : 0)] = p;
}
__global__ void k_umirror(int64_t n, const uint32_t* __restrict__ uptr, const uint64_t* __restrict__ uadj,
                          const uint32_t* __restrict__ ueid, const uint32_t* __restrict__ epos,
                          uint32_t* __restrict__ umir) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps)
    for (uint32_t p = uptr[x] + lane; p < uptr[x + 1]; p += 32)
      umir[p] = epos[2 * (size_t)ueid[p] + ((uint32_t)x > adj_col(uadj[p]) ? 0 : 1)];
}

// Edge index: every edge once, from the row of its smaller endpoint.  The
// table has at least four times as many slots as edges, so every insert
// finds a free slot; the loop bound is a self-check.
__global__ void k_edge_index(int64_t n, const uint32_t* __restrict__ uptr, const uint64_t* __restrict__ uadj,
                             uint4* __restrict__ eslots, uint64_t slots,
                             int shift, unsigned long long* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps)
    for (uint32_t p = uptr[x] + lane; p < uptr[x + 1]; p += 32) {
      const uint64_t e = uadj[p];
      if ((uint32_t)x > adj_col(e)) continue;
      const uint64_t key = edge_index_key((uint32_t)x, adj_col(e));
      uint64_t h = edge_index_home(key, shift);
      uint64_t it = 0;
      for (; it < slots; it++) {
        unsigned long long* slot_key = reinterpret_cast<unsigned long long*>(&eslots[h]);
        if (atomicCAS(slot_key, (unsigned long long)kEdgeIndexEmpty, (unsigned long long)key) == kEdgeIndexEmpty) {
          eslots[h].z = adj_valbits(e);
          break;
        }
        h = (h + 1) & (slots - 1);
      }
      if (it == slots) report(err, p, -UBT_ERR_INVALID_ARG);
    }
}

// AEO traversal: edge x-y is handled by x, the endpoint with the longer list
// (ties: the larger id), which holds the hash table; y's list is streamed.
__device__ inline bool aeo_owns(uint32_t x, uint32_t y, uint32_t dx, uint32_t dy) {
  return dx > dy || (dx == dy && x > y);
}
__global__ void k_apair_count(int64_t n, const uint32_t* __restrict__ uptr, const uint64_t* __restrict__ uadj,
                              uint32_t* __restrict__ pcount) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps) {
    const uint32_t dx = uptr[x + 1] - uptr[x];
    uint32_t c = 0;
    for (uint32_t p = uptr[x] + lane; p < uptr[x + 1]; p += 32) {
      const uint32_t y = adj_col(uadj[p]);
      c += aeo_owns((uint32_t)x, y, dx, uptr[y + 1] - uptr[y]) ? 1u : 0u;
    }
    c = __reduce_add_sync(kFull, c);
    if (lane == 0) pcount[x] = c;
  }
}
// pair words in row order: streamed endpoint | position of the edge in x's row << 32
__global__ void k_apair_fill(int64_t n, const uint32_t* __restrict__ uptr, const uint64_t* __restrict__ uadj,
                             const uint32_t* __restrict__ apair_ptr, uint64_t* __restrict__ apairs,
                             unsigned long long* __restrict__ work) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps) {
    const uint32_t dx = uptr[x + 1] - uptr[x];
    uint32_t at = apair_ptr[x];
    unsigned long long w = 0;
    for (uint32_t base = uptr[x]; base < uptr[x + 1]; base += 32) {
      const uint32_t p = base + lane;
      bool own = false;
      uint32_t y = 0;
      if (p < uptr[x + 1]) {
        y = adj_col(uadj[p]);
        own = aeo_owns((uint32_t)x, y, dx, uptr[y + 1] - uptr[y]);
      }
      const unsigned msk = __ballot_sync(kFull, own);
      if (own) {
        apairs[at + __popc(msk & lanemask_lt())] = ((uint64_t)p << 32) | y;
        w += uptr[y + 1] - uptr[y];
      }
      at += __popc(msk);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) w += __shfl_xor_sync(kFull, w, d);
    if (lane == 0) work[x] = w;
  }
}
// owners by decreasing log2 of their streamed work, those with rows longer
// than kAeoWarpRow (whole-block tasks) first: bucket = lg * 2 + (1 if block)
constexpr uint32_t kAeoWarpRow = 128;
__global__ void k_afill_lists(int64_t n, const uint32_t* __restrict__ uptr, const uint32_t* __restrict__ apair_ptr,
                              const unsigned long long* __restrict__ work, unsigned long long* cursor,
                              uint32_t* __restrict__ lists, int count_only) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    if (apair_ptr[x + 1] == apair_ptr[x]) continue;
    const unsigned long long w = work[x];
    const int lg = w ? 63 - __clzll(w) : 0;
    const int b = lg * 2 + (uptr[x + 1] - uptr[x] > kAeoWarpRow ? 1 : 0);
    if (count_only) atomicAdd(&cursor[b], 1ull);
    else lists[atomicAdd(&cursor[b], 1ull)] = (uint32_t)x;
  }
}
__global__ void k_max_row(int64_t n, const uint32_t* __restrict__ ptr, unsigned long long* out) {
  unsigned long long best = 0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    best = max(best, (unsigned long long)(ptr[x + 1] - ptr[x]));
  atomicMax(out, best);
}

struct BuildLayout {
  // persistent
  Scratch* scratch;
  uint32_t* row_ptr;
  uint64_t* adj;
  uint32_t* eid;
  uint32_t* ekey;
  uint32_t* pair_ptr;
  uint64_t* pairs;
  uint32_t* lists;       // giant | hub | medium tasks
  uint32_t* vgraph;
  uint32_t* uptr;        // undirected AEO adjacency (optional)
  uint64_t* uadj;
  uint32_t* ueid;
  uint32_t* umir;
  uint32_t* uepos;
  uint32_t* apair_ptr;
  uint64_t* apairs;
  uint32_t* alist;
  unsigned long long* awork;
  unsigned long long* lqueue;  // long vertex samples of a local-count call (with the undirected rows)
  uint4* eslots;               // edge index (optional)
  int64_t eh_slots;
  unsigned long long* gacc;
  unsigned long long* bacc;
  uint32_t* gtab;
  // build temporaries
  uint32_t* deg;
  uint32_t* fill;
  uint32_t* scan_tmp;
  uint32_t* mid_rows;
  uint32_t* huge_rows;
  uint8_t* bucket;
  unsigned long long* work;    // streamed work per owner
  unsigned long long* stats;   // 4 + 4*48 counters, 4*48 cursors, 2 counters
  char* sort_tmp;
  size_t total;
};
constexpr int kStats = 4 + 4 * (kLgMax + 1);

int64_t list_bound(int64_t n, int64_t m) {
  // a forward list under Node Order holds at most sqrt(2m) entries
  int64_t b = (int64_t)sqrt(2.0 * (double)m) + 2;
  return std::min<int64_t>(b, std::max<int64_t>(n, 1));
}

int64_t pow2_at_least(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

BuildLayout layout(void* ws, size_t cap, int64_t n, int64_t m, const ubt_graph_opts* opts, int sm_count) {
  Carver c(ws, cap);
  BuildLayout L;
  const bool has_key = opts && opts->d_edge_key;
  const bool batch = opts && opts->d_vertex_offsets;
  const int64_t ng = batch ? opts->n_graphs : 1;
  const int64_t n1 = std::max<int64_t>(n, 1);
  L.scratch = c.take<Scratch>(1);
  L.row_ptr = c.take<uint32_t>(n + 1);
  L.adj = c.take<uint64_t>(std::max<int64_t>(m, 1));
  L.eid = c.take<uint32_t>(std::max<int64_t>(m, 1));
  L.ekey = has_key ? c.take<uint32_t>(std::max<int64_t>(m, 1)) : nullptr;
  L.pair_ptr = c.take<uint32_t>(n + 1);
  L.pairs = c.take<uint64_t>(std::max<int64_t>(m, 1));
  L.lists = c.take<uint32_t>(n1);
  L.vgraph = batch ? c.take<uint32_t>(n1) : nullptr;
  const bool und = opts && (opts->flags & UBT_OPT_UNDIRECTED);
  L.uptr = und ? c.take<uint32_t>(n + 1) : nullptr;
  L.uadj = und ? c.take<uint64_t>(std::max<int64_t>(2 * m, 1)) : nullptr;
  L.ueid = und ? c.take<uint32_t>(std::max<int64_t>(2 * m, 1)) : nullptr;
  L.umir = und ? c.take<uint32_t>(std::max<int64_t>(2 * m, 1)) : nullptr;
  L.uepos = und ? c.take<uint32_t>(std::max<int64_t>(2 * m, 1)) : nullptr;
  L.apair_ptr = und ? c.take<uint32_t>(n + 1) : nullptr;
  L.apairs = und ? c.take<uint64_t>(std::max<int64_t>(m, 1)) : nullptr;
  L.alist = und ? c.take<uint32_t>(n1) : nullptr;
  L.awork = und ? c.take<unsigned long long>(n1) : nullptr;
  L.lqueue = und ? c.take<unsigned long long>(2 + kLongQueue) : nullptr;
  const bool eidx = und && (opts->flags & UBT_OPT_EDGE_INDEX);
  L.eh_slots = eidx ? pow2_at_least(std::max<int64_t>(4 * m, 64)) : 0;
  L.eslots = eidx ? c.take<uint4>(L.eh_slots) : nullptr;
  L.gacc = c.take<unsigned long long>(std::max<int64_t>(m, 1));
  // per graph: T, sum_lo, sum_hi (expected counts) of a batch
  L.bacc = c.take<unsigned long long>(3 * std::max<int64_t>(ng, 1));
  const int64_t gslots = gtab_slots_for(m);
  L.gtab = gslots ? c.take<uint32_t>((size_t)gslots * 3 * (size_t)sm_count) : nullptr;
  L.deg = c.take<uint32_t>(n + 1);
  L.fill = c.take<uint32_t>(n + 1);
  L.scan_tmp = c.take<uint32_t>(scan_tmp_words(std::max(n, ng)) + 2);
  L.mid_rows = c.take<uint32_t>(n1);
  L.huge_rows = c.take<uint32_t>(n1);
  L.bucket = c.take<uint8_t>(n1);
  L.work = c.take<unsigned long long>(n1);
  L.stats = c.take<unsigned long long>(2 * kStats + 4);
  const int64_t lb = list_bound(n, m);
  L.sort_tmp = lb > tuning().sort_smem_max
                   ? c.take<char>((size_t)kSortHugeBlocks * (size_t)pow2_at_least(lb) * 24) : nullptr;
  L.total = c.off + 256;
  return L;
}

int device_sm_count(int* dev) {
  int d = 0, sms = 0;
  cudaGetDevice(&d);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
  if (dev) *dev = d;
  return sms > 0 ? sms : 1;
}

ubt_status status_from_err(unsigned long long e) {
  if (e == ~0ull) return UBT_OK;
  return -(ubt_status)(e & 0xFF);
}

}  // namespace

int64_t gtab_slots_for(int64_t m) {
  // a list's table holds 4x its entries (power of two); lists whose table
  // exceeds the shared-memory limit get one in global memory, sized for the
  // longest possible list
  const int64_t need = pow2_at_least(4 * list_bound(INT64_MAX / 4, m));
  return need > tuning().smem_table_max ? need : 0;
}

}  // namespace ubt

using namespace ubt;

extern "C" ubt_status ubt_graph_workspace_size(int64_t n, int64_t m, int32_t flags, const ubt_graph_opts* opts,
                                               size_t* h_bytes) {
  if (!h_bytes || n < 0 || m < 0 || n >= 0xFFFFFFFFll || m >= 0xFFFFFFFFll) return UBT_ERR_INVALID_ARG;
  if (flags != UBT_GRAPH_FIXED && flags != UBT_GRAPH_REAL) return UBT_ERR_INVALID_ARG;
  if (opts && opts->d_vertex_offsets && opts->n_graphs < 1) return UBT_ERR_INVALID_ARG;
  BuildLayout L = layout(nullptr, 0, n, m, opts, device_sm_count(nullptr));
  *h_bytes = L.total;
  return UBT_OK;
}

extern "C" ubt_status ubt_create_graph(int64_t n, int64_t m, const uint32_t* d_src, const uint32_t* d_dst,
                                       const uint32_t* d_k, const float* d_p, int32_t flags,
                                       const ubt_graph_opts* opts, void* d_workspace, size_t ws_bytes,
                                       void* stream, ubt_graph** h_out) {
  UBT_RANGE("ubt_create_graph");
  if (!h_out) return UBT_ERR_INVALID_ARG;
  *h_out = nullptr;
  if (n < 0 || m < 0 || n >= 0xFFFFFFFFll || m >= 0xFFFFFFFFll) return UBT_ERR_INVALID_ARG;
  if (flags == UBT_GRAPH_FIXED) {
    if ((m > 0 && !d_k) || d_p) return UBT_ERR_INVALID_ARG;
  } else if (flags == UBT_GRAPH_REAL) {
    if ((m > 0 && !d_p) || d_k) return UBT_ERR_INVALID_ARG;
  } else {
    return UBT_ERR_INVALID_ARG;
  }
  if (m > 0 && (!d_src || !d_dst)) return UBT_ERR_INVALID_ARG;
  const bool und = opts && (opts->flags & UBT_OPT_UNDIRECTED);
  if (opts && (opts->flags & ~(int64_t)(UBT_OPT_UNDIRECTED | UBT_OPT_EDGE_INDEX))) return UBT_ERR_INVALID_ARG;
  if (opts && (opts->flags & UBT_OPT_EDGE_INDEX) && !und) return UBT_ERR_INVALID_ARG;
  if (und && flags != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
  if (!d_workspace || ((uintptr_t)d_workspace & 255)) return UBT_ERR_INVALID_ARG;
  const bool batch = opts && opts->d_vertex_offsets;
  if (batch && opts->n_graphs < 1) return UBT_ERR_INVALID_ARG;
  const int64_t ng = batch ? opts->n_graphs : 1;
  int dev = 0;
  const int sms = device_sm_count(&dev);
  BuildLayout L = layout(d_workspace, ws_bytes, n, m, opts, sms);
  if (ws_bytes < L.total) return UBT_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  const Tuning& T = tuning();
  const int64_t hub_thr = std::max<int64_t>(2, T.hub_threshold);
  const int64_t giant_thr = std::max<int64_t>(hub_thr, T.smem_table_max / 4);
  const int pull = T.pull ? 1 : 0;
  const int64_t block_work = std::max<int64_t>(1, T.block_work);

  UBT_CUDA(cudaMemsetAsync(L.scratch, 0, sizeof(Scratch), s));
  UBT_CUDA(cudaMemsetAsync(&L.scratch->err, 0xFF, sizeof(unsigned long long), s));
  UBT_CUDA(cudaMemsetAsync(L.deg, 0, sizeof(uint32_t) * (n + 1), s));
  UBT_CUDA(cudaMemsetAsync(L.fill, 0, sizeof(uint32_t) * (n + 1), s));
  UBT_CUDA(cudaMemsetAsync(L.stats, 0, sizeof(unsigned long long) * (2 * kStats + 4), s));
  const int thr = 256;
  const int grid_e = (int)std::min<int64_t>(std::max<int64_t>((m + thr - 1) / thr, 1), (int64_t)sms * 32);
  const int grid_v = (int)std::min<int64_t>(std::max<int64_t>((n + thr - 1) / thr, 1), (int64_t)sms * 32);
  const int grid_w = (int)std::min<int64_t>(std::max<int64_t>((n + 7) / 8, 1), (int64_t)sms * 32);

  if (batch) {
    k_vertex_graph<<<grid_v, thr, 0, s>>>(opts->d_vertex_offsets, opts->n_graphs, n, L.vgraph);
  }
  // 1. validate + degree
  NvtxPhases phase;
  phase.next("build: validate and degree");
  if (m > 0)
    k_validate_degree<<<grid_e, thr, 0, s>>>(n, m, d_src, d_dst, d_k, d_p, L.vgraph, L.deg, &L.scratch->err);
  unsigned long long err = 0;
  UBT_CUDA(cudaMemcpyAsync(&err, &L.scratch->err, sizeof(err), cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  ubt_status st = status_from_err(err);
  if (st != UBT_OK) return st;
  // 2. orientation + CSR offsets
  phase.next("build: orient, scatter, sort");
  if (m > 0) k_out_degree<<<grid_e, thr, 0, s>>>(m, d_src, d_dst, L.deg, L.fill);
  UBT_CUDA(exclusive_scan_u32(L.fill, L.row_ptr, n, L.scan_tmp, s));
  UBT_CUDA(cudaMemsetAsync(L.fill, 0, sizeof(uint32_t) * (n + 1), s));
  if (m > 0)
    k_scatter<<<grid_e, thr, 0, s>>>(m, d_src, d_dst, d_k, d_p, L.deg, L.row_ptr, L.fill, L.adj, L.eid,
                                     opts ? opts->d_edge_key : nullptr, L.ekey);
  // 3. sort every forward list
  const int fixed = flags == UBT_GRAPH_FIXED;
  const int mode = fixed ? kSortByAbsqChecked : kSortById;
  unsigned long long* lcount = L.stats + 2 * kStats;
  if (n > 0) {
    k_sort_short_rows<<<grid_w, thr, 0, s>>>(n, L.row_ptr, L.adj, L.eid, L.ekey, mode, &L.scratch->err);
    const uint32_t sort_smem = (uint32_t)tuning().sort_smem_max;
    const uint32_t warp_max = (uint32_t)tuning().warp_sort_max;
    k_collect_long<<<grid_v, thr, 0, s>>>(n, L.row_ptr, sort_smem, warp_max, L.mid_rows, L.huge_rows, lcount);
    unsigned long long lc[3] = {0, 0, 0};
    UBT_CUDA(cudaMemcpyAsync(lc, lcount, sizeof(lc), cudaMemcpyDeviceToHost, s));
    UBT_CUDA(cudaStreamSynchronize(s));
    if (lc[2]) {
      st = launch_mid_sorts(L.mid_rows + (n - (int64_t)lc[2]), (uint32_t)lc[2], L.row_ptr, L.adj, L.eid, L.ekey, mode,
                            &L.scratch->err, warp_max, sms, thr, s);
      if (st != UBT_OK) return st;
    }
    if (lc[0]) {
      st = launch_block_sorts(L.mid_rows, (uint32_t)lc[0], L.row_ptr, L.adj, L.eid, L.ekey, mode, &L.scratch->err,
                              warp_max, sort_smem, sms, s);
      if (st != UBT_OK) return st;
    }
    if (lc[1]) {
      const int64_t cap = pow2_at_least(list_bound(n, m));
      const int g = (int)std::min<unsigned long long>(lc[1], (unsigned long long)kSortHugeBlocks);
      k_sort_long_rows<true><<<g, 1024, 0, s>>>(L.huge_rows, (uint32_t)lc[1], L.row_ptr, L.adj, L.eid, L.ekey,
                                                fixed, &L.scratch->err, L.sort_tmp, cap);
    }
    UBT_CUDA(cudaGetLastError());
  }
  UBT_CUDA(cudaMemcpyAsync(&err, &L.scratch->err, sizeof(err), cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  st = status_from_err(err);
  if (st != UBT_OK) return st;
  // 4. pairs grouped by owner
  phase.next("build: pairs and work lists");
  UBT_CUDA(cudaMemsetAsync(L.pair_ptr, 0, sizeof(uint32_t) * (n + 1), s));
  if (n > 0) {
    UBT_CUDA(cudaMemsetAsync(L.fill, 0, sizeof(uint32_t) * (n + 1), s));
    // the row of every CSR position, in the (not yet used) adjoint accumulators
    uint32_t* rowid = (uint32_t*)L.gacc;
    k_row_ids<<<grid_v, thr, 0, s>>>(n, L.row_ptr, rowid);
    if (m > 0) k_pair_count<<<grid_e, thr, 0, s>>>(m, L.row_ptr, L.adj, rowid, pull, L.fill, &L.stats[0]);
    UBT_CUDA(exclusive_scan_u32(L.fill, L.pair_ptr, n, L.scan_tmp, s));
    UBT_CUDA(cudaMemsetAsync(L.fill, 0, sizeof(uint32_t) * (n + 1), s));
    UBT_CUDA(cudaMemsetAsync(L.work, 0, sizeof(unsigned long long) * n, s));
    if (m > 0)
      k_pair_fill<<<grid_e, thr, 0, s>>>(m, L.row_ptr, L.adj, rowid, pull, L.pair_ptr, L.fill, L.pairs, L.work);
    UBT_CUDA(cudaGetLastError());
  }
  // 5. work lists: giant | hub | medium tasks, each by decreasing work bucket
  unsigned long long stats[kStats];
  memset(stats, 0, sizeof(stats));
  if (n > 0) {
    k_row_stats<<<grid_v, thr, 0, s>>>(n, L.row_ptr, L.pair_ptr, L.work, (uint32_t)hub_thr, (uint32_t)giant_thr,
                                      (unsigned long long)block_work, L.bucket, L.stats);
    UBT_CUDA(cudaMemcpyAsync(stats, L.stats, sizeof(stats), cudaMemcpyDeviceToHost, s));
    UBT_CUDA(cudaStreamSynchronize(s));
  }
  unsigned long long cursor[4 * (kLgMax + 1)];
  int64_t count_cls[4] = {0, 0, 0, 0};
  for (int b = 0; b < 4 * (kLgMax + 1); b++) count_cls[b % 4] += (int64_t)stats[4 + b];
  int64_t run[4] = {0, 0, 0, 0};
  run[kClsGiant] = 0;
  run[kClsHub] = count_cls[kClsGiant];
  run[kClsMedium] = count_cls[kClsGiant] + count_cls[kClsHub];
  for (int lg = kLgMax; lg >= 0; lg--) {
    for (int cls = 1; cls < 4; cls++) {
      const int b = lg * 4 + cls;
      cursor[b] = (unsigned long long)run[cls];
      run[cls] += (int64_t)stats[4 + b];
    }
  }
  if (n > 0) {
    unsigned long long* dcur = L.stats + kStats;
    UBT_CUDA(cudaMemcpyAsync(dcur, cursor, sizeof(cursor), cudaMemcpyHostToDevice, s));
    k_fill_lists<<<grid_v, thr, 0, s>>>(n, L.bucket, dcur, L.lists);
    UBT_CUDA(cudaGetLastError());
    UBT_CUDA(cudaStreamSynchronize(s));
  }
  (void)ng;
  // 6. undirected adjacency in Absolute Edge Order, its mirror positions and
  //    the AEO pair partition (optional)
  int64_t n_aowners = 0, n_ablock = 0, max_udeg = 0;
  if (und && n > 0) {
    phase.next("build: undirected rows in Absolute Edge Order");
    UBT_CUDA(exclusive_scan_u32(L.deg, L.uptr, n, L.scan_tmp, s));
    UBT_CUDA(cudaMemsetAsync(L.fill, 0, sizeof(uint32_t) * (n + 1), s));
    if (m > 0) k_uscatter<<<grid_e, thr, 0, s>>>(m, d_src, d_dst, d_k, L.uptr, L.fill, L.uadj, L.ueid);
    k_sort_short_rows<<<grid_w, thr, 0, s>>>(n, L.uptr, L.uadj, L.ueid, nullptr, kSortByAbsq, &L.scratch->err);
    const uint32_t sort_smem = (uint32_t)tuning().sort_smem_max;
    UBT_CUDA(cudaMemsetAsync(lcount, 0, 3 * sizeof(unsigned long long), s));
    const uint32_t warp_max = (uint32_t)tuning().warp_sort_max;
    k_collect_long<<<grid_v, thr, 0, s>>>(n, L.uptr, sort_smem, warp_max, L.mid_rows, L.huge_rows, lcount);
    unsigned long long lc[3] = {0, 0, 0};
    UBT_CUDA(cudaMemcpyAsync(lc, lcount, sizeof(lc), cudaMemcpyDeviceToHost, s));
    UBT_CUDA(cudaStreamSynchronize(s));
    if (lc[2]) {
      st = launch_mid_sorts(L.mid_rows + (n - (int64_t)lc[2]), (uint32_t)lc[2], L.uptr, L.uadj, L.ueid, nullptr,
                            kSortByAbsq, &L.scratch->err, warp_max, sms, thr, s);
      if (st != UBT_OK) return st;
    }
    if (lc[0]) {
      st = launch_block_sorts(L.mid_rows, (uint32_t)lc[0], L.uptr, L.uadj, L.ueid, nullptr, kSortByAbsq,
                              &L.scratch->err, warp_max, sort_smem, sms, s);
      if (st != UBT_OK) return st;
    }
    if (lc[1]) {
      const int g2 = (int)std::min<unsigned long long>(lc[1], (unsigned long long)sms * 2);
      k_sort_rows_inplace<<<g2, 1024, 0, s>>>(L.huge_rows, (uint32_t)lc[1], L.uptr, L.uadj, L.ueid);
    }
    k_uepos<<<grid_w, thr, 0, s>>>(n, L.uptr, L.uadj, L.ueid, L.uepos);
    k_umirror<<<grid_w, thr, 0, s>>>(n, L.uptr, L.uadj, L.ueid, L.uepos, L.umir);
    if (L.eslots) {
      UBT_CUDA(cudaMemsetAsync(L.eslots, 0xFF, sizeof(uint4) * (size_t)L.eh_slots, s));
      int lg = 0;
      while ((1ll << lg) < L.eh_slots) lg++;
      k_edge_index<<<grid_w, thr, 0, s>>>(n, L.uptr, L.uadj, L.eslots, (uint64_t)L.eh_slots, 64 - lg,
                                          &L.scratch->err);
    }
    UBT_CUDA(cudaMemsetAsync(L.fill, 0, sizeof(uint32_t) * (n + 1), s));
    k_apair_count<<<grid_w, thr, 0, s>>>(n, L.uptr, L.uadj, L.fill);
    UBT_CUDA(exclusive_scan_u32(L.fill, L.apair_ptr, n, L.scan_tmp, s));
    k_apair_fill<<<grid_w, thr, 0, s>>>(n, L.uptr, L.uadj, L.apair_ptr, L.apairs, L.awork);
    unsigned long long* acur = L.stats;  // 2 (kLgMax + 1) cursors, then the longest row
    constexpr int kAB = 2 * (kLgMax + 1);
    UBT_CUDA(cudaMemsetAsync(acur, 0, sizeof(unsigned long long) * (kAB + 1), s));
    k_afill_lists<<<grid_v, thr, 0, s>>>(n, L.uptr, L.apair_ptr, L.awork, acur, L.alist, 1);
    unsigned long long acount[kAB + 1];
    UBT_CUDA(cudaMemcpyAsync(acount, acur, sizeof(acount), cudaMemcpyDeviceToHost, s));
    UBT_CUDA(cudaStreamSynchronize(s));
    unsigned long long run = 0;
    for (int cls = 1; cls >= 0; cls--) {  // block tasks, then warp tasks
      for (int lg = kLgMax; lg >= 0; lg--) {
        const unsigned long long c = acount[lg * 2 + cls];
        acount[lg * 2 + cls] = run;
        run += c;
      }
      if (cls == 1) n_ablock = (int64_t)run;
    }
    n_aowners = (int64_t)run;
    acount[kAB] = 0;
    UBT_CUDA(cudaMemcpyAsync(acur, acount, sizeof(acount), cudaMemcpyHostToDevice, s));
    k_afill_lists<<<grid_v, thr, 0, s>>>(n, L.uptr, L.apair_ptr, L.awork, acur, L.alist, 0);
    k_max_row<<<grid_v, thr, 0, s>>>(n, L.uptr, &acur[kAB]);
    unsigned long long mx = 0;
    UBT_CUDA(cudaMemcpyAsync(&mx, &acur[kAB], sizeof(mx), cudaMemcpyDeviceToHost, s));
    UBT_CUDA(cudaMemcpyAsync(&err, &L.scratch->err, sizeof(err), cudaMemcpyDeviceToHost, s));
    UBT_CUDA(cudaGetLastError());
    UBT_CUDA(cudaStreamSynchronize(s));
    max_udeg = (int64_t)mx;
    st = status_from_err(err);
    if (st != UBT_OK) return st;
  }

  ubt_graph* g = new (std::nothrow) ubt_graph();
  if (!g) return UBT_ERR_INVALID_ARG;
  g->n = n;
  g->m = m;
  g->kind = flags;
  g->n_graphs = ng;
  g->row_ptr = L.row_ptr;
  g->adj = L.adj;
  g->eid = L.eid;
  g->ekey = L.ekey ? L.ekey : L.eid;
  g->pair_ptr = L.pair_ptr;
  g->pairs = L.pairs;
  g->giant_list = L.lists;
  g->n_giant = count_cls[kClsGiant];
  g->hub_list = L.lists + count_cls[kClsGiant];
  g->n_hub = count_cls[kClsHub];
  g->med_list = L.lists + count_cls[kClsGiant] + count_cls[kClsHub];
  g->n_med = count_cls[kClsMedium];
  g->vgraph = L.vgraph;
  g->uptr = L.uptr;
  g->uadj = L.uadj;
  g->ueid = L.ueid;
  g->umir = L.umir;
  g->uepos = L.uepos;
  g->apair_ptr = L.apair_ptr;
  g->apairs = L.apairs;
  g->alist = L.alist;
  g->n_aowners = n_aowners;
  g->n_ablock = n_ablock;
  g->max_udeg = max_udeg;
  g->lqueue = L.lqueue;
  g->eslots = L.eslots;
  g->eh_slots = L.eh_slots;
  {
    int lg = 0;
    while ((1ll << lg) < L.eh_slots) lg++;
    g->eh_shift = 64 - lg;
  }
  g->gacc = L.gacc;
  g->bacc = L.bacc;
  g->gtab = L.gtab;
  g->gtab_slots = gtab_slots_for(m);
  g->gtab_blocks = L.gtab ? sms : 0;
  g->scratch = L.scratch;
  g->wedges = (int64_t)stats[0];
  g->max_out = (int64_t)stats[1];
  g->max_hub_len = (int64_t)stats[2];
  g->probes = (int64_t)stats[3];
  g->hub_threshold = hub_thr;
  g->giant_threshold = giant_thr;
  g->block_work = block_work;
  g->pull = pull;
  g->device = dev;
  g->sm_count = sms;
  *h_out = g;
  return UBT_OK;
}

extern "C" ubt_status ubt_destroy_graph(ubt_graph* g) {
  if (!g) return UBT_ERR_INVALID_ARG;
  delete g;
  return UBT_OK;
}

extern "C" ubt_status ubt_graph_get_info(const ubt_graph* g, ubt_graph_info* h_info) {
  if (!g || !h_info) return UBT_ERR_INVALID_ARG;
  h_info->n = g->n;
  h_info->m = g->m;
  h_info->max_out_degree = g->max_out;
  h_info->hub_vertices = g->n_hub + g->n_giant;
  h_info->wedges = g->wedges;
  h_info->kind = g->kind;
  h_info->probes = g->probes;
  return UBT_OK;
}

namespace ubt {
namespace {

// New edge values of a REAL graph: CSR position pos holds input edge eid[pos],
// so its value becomes s(p[eid[pos]]); the rows stay sorted (by neighbour id).
// A p outside [0, 1] (or NaN) leaves the entry as it was and records the
// first such input index in the self-check word (code 6).
__global__ void k_set_edge_values(int64_t m, const float* __restrict__ p, const uint32_t* __restrict__ eid,
                                  uint64_t* __restrict__ adj, unsigned long long* guard) {
  for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < m; pos += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = eid[pos];
    const float x = p[e];
    if (!(x >= 0.0f && x <= 1.0f)) {
      atomicCAS(guard, 0ull, (6ull << 56) | (unsigned long long)e);
      continue;
    }
    adj[pos] = adj_pack(adj_col(adj[pos]), real_valbits(x));
  }
}

}  // namespace
}  // namespace ubt

extern "C" ubt_status ubt_set_edge_values(ubt_graph* g, const float* d_p, void* stream) {
  UBT_RANGE("ubt_set_edge_values");
  if (!g || (!d_p && g->m > 0)) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_REAL) return UBT_ERR_UNSUPPORTED;
  if (g->m == 0) return UBT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = (int)std::min<int64_t>((g->m + 255) / 256, (int64_t)g->sm_count * 8);
  k_set_edge_values<<<grid, 256, 0, s>>>(g->m, d_p, g->eid, g->adj, &g->scratch->guard);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}
