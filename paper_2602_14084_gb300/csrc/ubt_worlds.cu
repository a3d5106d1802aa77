// ubt_worlds.cu -- Monte-Carlo sign worlds and batched per-graph queries.
//
// Sign worlds (not in the paper): world 64 w + j draws every edge sign with
// P(+) = k / 65536.  A triangle is balanced in a world iff it has an odd
// number of positive edges (Def. 3, Sec. 3), i.e. iff the XOR of its three
// sign bits is 1.  64 worlds share one 64-bit word per edge ("bit-sliced").
//
// Draws: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC'11) with key (seed, 0) and counter (K, w, c, 0),
// c = 0..3, gives 16 words r_0..r_15; bit j of r_b is bit b of world j's
// 16-bit uniform u_j, and the edge is positive iff u_j < k.  The comparison is
// evaluated for all 64 worlds at once on the bit planes (most significant
// plane first).
//
// Per-world counts are kept per lane as bit-sliced binary counters (plane t
// holds bit t of 64 counters), incremented by the XOR word of each triangle,
// and flushed to integer counts before they can overflow.
#include <algorithm>
#include <vector>

#include "ubt_traverse.cuh"

namespace ubt {

TravArgs make_trav_args(const ubt_graph* g, int64_t L, bool with_pos);

namespace {

// ------------------------------------------------------------ Philox4x64-10

struct U64x4 {
  unsigned long long x[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, unsigned long long k0, unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const unsigned long long lo0 = M0 * c.x[0], hi0 = __umul64hi(M0, c.x[0]);
    const unsigned long long lo1 = M1 * c.x[2], hi1 = __umul64hi(M1, c.x[2]);
    U64x4 n;
    n.x[0] = hi1 ^ c.x[1] ^ k0;
    n.x[1] = lo1;
    n.x[2] = hi0 ^ c.x[3] ^ k1;
    n.x[3] = lo0;
    c = n;
  }
  return c;
}

// 64 sign draws of one edge in world word w: bit j = 1 iff positive in world 64w+j
__device__ __forceinline__ unsigned long long sign_word(unsigned long long seed, uint32_t key, uint32_t w,
                                                        uint32_t k) {
  if (k >= 65536u) return ~0ull;
  if (k == 0u) return 0ull;
  // u < k on the 16 bit planes, most significant first: call c gives planes
  // 4c .. 4c + 3.  A world is decided at the first plane where u and k
  // differ; once every world of the word is decided (eq = 0) the lower planes
  // change nothing, so their calls are skipped (after two calls about 78 % of
  // the words are decided, after three 98 %).
  unsigned long long lt = 0, eq = ~0ull;
#pragma unroll 1
  for (int c = 3; c >= 0 && eq; c--) {
    U64x4 ctr;
    ctr.x[0] = key;
    ctr.x[1] = w;
    ctr.x[2] = (unsigned long long)c;
    ctr.x[3] = 0;
    const U64x4 o = philox4x64_10(ctr, seed, 0ull);
#pragma unroll
    for (int i = 3; i >= 0; i--) {
      const unsigned long long r = o.x[i];
      if ((k >> (4 * c + i)) & 1u) {
        lt |= eq & ~r;
        eq &= r;
      } else {
        eq &= ~r;
      }
    }
  }
  return lt;
}

// X[pos * wp + i] = sign word (w0 + i) of the edge at CSR position pos
__global__ void k_sign_table(int64_t m, const uint64_t* __restrict__ adj, const uint32_t* __restrict__ ekey,
                             unsigned long long seed, uint32_t w0, uint32_t wp, unsigned long long* __restrict__ X) {
  const int64_t total = m * (int64_t)wp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = i / wp;
    const uint32_t w = w0 + (uint32_t)(i - pos * wp);
    const int32_t q = adj_q(adj[pos]);
    const uint32_t k = (uint32_t)(32768 - q);
    X[i] = sign_word(seed, ekey[pos], w, k);
  }
}

// ------------------------------------------------------------ bit-sliced counters

template <int K>
struct Planes {
  unsigned long long c[K];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int t = 0; t < K; t++) c[t] = 0;
  }
  __device__ __forceinline__ void inc(unsigned long long b) {
#pragma unroll
    for (int t = 0; t < K; t++) {
      const unsigned long long carry = c[t] & b;
      c[t] ^= b;
      b = carry;
      if (!b) break;
    }
  }
  // two counters at once: one carry chain per counter, interleaved, ending
  // when both carries are spent
  __device__ __forceinline__ static void inc2(Planes& p0, Planes& p1, unsigned long long b0, unsigned long long b1) {
#pragma unroll
    for (int t = 0; t < K; t++) {
      const unsigned long long c0 = p0.c[t] & b0, c1 = p1.c[t] & b1;
      p0.c[t] ^= b0;
      p1.c[t] ^= b1;
      b0 = c0;
      b1 = c1;
      if (!(b0 | b1)) break;
    }
  }
  // per-lane count of world j
  __device__ __forceinline__ uint32_t count(int j) const {
    uint32_t v = 0;
#pragma unroll
    for (int t = 0; t < K; t++) v |= (uint32_t)((c[t] >> j) & 1ull) << t;
    return v;
  }
};

// ------------------------------------------------------------ sign-world visitor

struct WorldsP {
  const unsigned long long* X;  // sign table of this pass: m x wp words
  uint32_t wp;                  // words per pass (1..64, power of two)
  unsigned long long* out;      // counts of this pass's worlds: wp * 64
};

// SLOTS = words per lane: 1 when wp <= 32 (lanes grouped by word), 2 when wp = 64
template <int SLOTS>
struct Worlds {
  using P = WorldsP;
  static constexpr bool kPos = true;
  static constexpr bool kBatched = false;
  static constexpr int kRegCap = 128;
  static constexpr int K = SLOTS == 1 ? 14 : 12;      // planes per slot
  static constexpr uint32_t kLimit = (1u << K) - 1u;  // increments before a flush
  static constexpr int kQueue = 64;
  // counters + one queue per warp
  static __host__ __device__ int smem_bytes(int threads) { return 64 * 64 * 8 + (threads / 32) * kQueue * 12; }
  P p;
  unsigned long long* cnt;  // shared: wp * 64 counters
  uint32_t* q;              // this warp's queue: 3 x kQueue positions
  uint32_t qn = 0;
  uint32_t since = 0;
  Planes<K> pl[SLOTS];
  __device__ Worlds(const P& p_, char* smem) : p(p_) {
    cnt = (unsigned long long*)smem;
    q = (uint32_t*)(smem + 64 * 64 * 8) + (threadIdx.x >> 5) * 3 * kQueue;
#pragma unroll
    for (int s = 0; s < SLOTS; s++) pl[s].clear();
  }
  __device__ void block_init() {
    for (int i = threadIdx.x; i < (int)p.wp * 64; i += blockDim.x) cnt[i] = 0;
  }
  __device__ __forceinline__ uint32_t word_of(int s) const {
    const int lane = (int)lane_id();
    return SLOTS == 2 ? (uint32_t)(2 * lane + s) : (uint32_t)lane % p.wp;
  }
  __device__ void flush() {
#pragma unroll
    for (int s = 0; s < SLOTS; s++) {
      const uint32_t w = word_of(s);
#pragma unroll 1
      for (int j = 0; j < 64; j++) {
        const uint32_t v = pl[s].count(j);
        if (v) atomicAdd(&cnt[w * 64 + j], (unsigned long long)v);
      }
      pl[s].clear();
    }
    since = 0;
  }
  // The queued triangles one after another, with the next triangle's sign
  // words loaded before the current one's counters are updated, so that a
  // warp's loads overlap its counter updates.
  __device__ void drain() {
    __syncwarp();
    const int lane = (int)lane_id();
    const unsigned long long* X = p.X;
    const uint32_t wp = p.wp;
    if (SLOTS == 2) {
      // a row is 64 words = 32 16-byte pairs: lane l holds words 2l and 2l + 1
      const ulonglong2* __restrict__ X2 = reinterpret_cast<const ulonglong2*>(X);
      auto word2 = [&](uint32_t t) -> ulonglong2 {
        const ulonglong2 a = X2[(size_t)q[t] * 32 + lane], b = X2[(size_t)q[kQueue + t] * 32 + lane],
                         c = X2[(size_t)q[2 * kQueue + t] * 32 + lane];
        return make_ulonglong2(a.x ^ b.x ^ c.x, a.y ^ b.y ^ c.y);
      };
      ulonglong2 nx = make_ulonglong2(0ull, 0ull);  // the next triangle's XOR words
      if (qn) nx = word2(0);
      for (uint32_t t = 0; t < qn; t++) {
        const ulonglong2 cx = nx;
        if (t + 1 < qn) nx = word2(t + 1);  // the same for every lane (qn is)
        Planes<K>::inc2(pl[0], pl[1], cx.x, cx.y);
        if (++since == kLimit) flush();
      }
    } else {
      const uint32_t per = 32 / wp;  // triangles per iteration
      const uint32_t grp = (uint32_t)lane / wp, w = (uint32_t)lane % wp;
      auto word = [&](uint32_t t) -> unsigned long long {
        return t < qn ? X[(size_t)q[t] * wp + w] ^ X[(size_t)q[kQueue + t] * wp + w] ^
                            X[(size_t)q[2 * kQueue + t] * wp + w]
                      : 0ull;
      };
      unsigned long long nb = word(grp);
      for (uint32_t t0 = 0; t0 < qn; t0 += per) {
        const unsigned long long bw = nb;
        nb = word(t0 + per + grp);
        pl[0].inc(bw);
        if (++since == kLimit) flush();
      }
    }
    qn = 0;
    __syncwarp();
  }
  __device__ __forceinline__ void step(bool hit, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,
                                       uint32_t puv, uint32_t puw, uint32_t pvw) {
    const unsigned m = __ballot_sync(kFull, hit);
    if (!m) return;
    const int lane = (int)lane_id();
    if (hit) {
      const uint32_t at = qn + __popc(m & lanemask_lt());
      q[at] = puv;
      q[kQueue + at] = puw;
      q[2 * kQueue + at] = pvw;
    }
    qn += __popc(m);
    if (qn >= 32) drain();
  }
  __device__ void task_begin(uint32_t) {}
  __device__ void task_end(uint32_t) {}
  __device__ void block_end() {
    if (qn) drain();
    flush();
    __syncthreads();
    for (int i = threadIdx.x; i < (int)p.wp * 64; i += blockDim.x)
      if (cnt[i]) atomicAdd(&p.out[i], cnt[i]);
  }
};

__global__ void k_world_total(const unsigned long long* __restrict__ cnt, int64_t W, int64_t* total) {
  __shared__ unsigned long long s[1024];
  unsigned long long acc = 0;
  for (int64_t i = threadIdx.x; i < W; i += blockDim.x) acc += cnt[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int d = blockDim.x / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) s[threadIdx.x] += s[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = (int64_t)s[0];
}

// ------------------------------------------------------------ batch visitor

constexpr int kBatchTau = 8;

struct BatchP {
  int nt;
  int64_t B[kBatchTau];
  int64_t U[kBatchTau];
  const uint32_t* vgraph;
  const unsigned long long* X;  // one sign word per CSR position, or null
  unsigned long long* counts;   // per graph: 2 * nt
  unsigned long long* acc;      // per graph: T, sum_lo, sum_hi (or null)
  unsigned long long* worlds;   // per graph: 64 (or null)
};

// Per-graph answers; all tasks of a warp between two graph changes share
// their registers, which are flushed when the graph changes.
struct Batch {
  using P = BatchP;
  static constexpr bool kPos = true;
  static constexpr bool kBatched = false;
  static constexpr int kRegCap = 128;
  static __host__ __device__ int smem_bytes(int) { return 0; }
  static constexpr int K = 8;
  P p;
  uint32_t g = kEmpty;
  uint32_t bal[kBatchTau], unbal[kBatchTau];
  uint32_t tri = 0;
  unsigned long long lo = 0, hi = 0;
  Planes<K> pl;
  uint32_t since = 0;
  __device__ Batch(const P& p_, char*) : p(p_) { reset(); }
  __device__ void reset() {
#pragma unroll
    for (int i = 0; i < kBatchTau; i++) bal[i] = unbal[i] = 0;
    tri = 0;
    lo = hi = 0;
    pl.clear();
    since = 0;
  }
  __device__ void block_init() {}
  __device__ void flush() {
    const int lane = (int)lane_id();
    if (g == kEmpty) return;
#pragma unroll
    for (int i = 0; i < kBatchTau; i++) {
      if (i < p.nt) {
        const uint32_t b = __reduce_add_sync(kFull, bal[i]);
        const uint32_t u = __reduce_add_sync(kFull, unbal[i]);
        if (lane == 0) {
          if (b) atomicAdd(&p.counts[(size_t)g * 2 * p.nt + i], (unsigned long long)b);
          if (u) atomicAdd(&p.counts[(size_t)g * 2 * p.nt + p.nt + i], (unsigned long long)u);
        }
      }
    }
    if (p.acc) {
      const uint32_t t = __reduce_add_sync(kFull, tri);
      // 128-bit warp sum
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long l = __shfl_xor_sync(kFull, lo, d);
        const unsigned long long h = __shfl_xor_sync(kFull, hi, d);
        const unsigned long long o = lo;
        lo += l;
        hi += h + (lo < o ? 1ull : 0ull);
      }
      if (lane == 0 && t) {
        unsigned long long* a = p.acc + (size_t)g * 3;
        atomicAdd(&a[0], (unsigned long long)t);
        const unsigned long long o = atomicAdd(&a[1], lo);
        atomicAdd(&a[2], hi + ((o + lo < o) ? 1ull : 0ull));
      }
    }
    if (p.worlds) {
      for (int j = 0; j < 64; j++) {
        const uint32_t v = __reduce_add_sync(kFull, pl.count(j));
        if (lane == (j & 31) && v) atomicAdd(&p.worlds[(size_t)g * 64 + j], (unsigned long long)v);
      }
    }
    reset();
  }
  __device__ __forceinline__ void step(bool hit, uint32_t, uint32_t, uint32_t, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t puv, uint32_t puw, uint32_t pvw) {
    if (hit) {
      const int64_t P = (int64_t)((int32_t)quv * (int32_t)quw) * (int64_t)(int32_t)qvw;
#pragma unroll
      for (int i = 0; i < kBatchTau; i++) {
        if (i < p.nt) {
          bal[i] += (P <= p.B[i]);
          unbal[i] += (P > p.U[i]);
        }
      }
      tri++;
      const unsigned long long o = lo;
      lo += (unsigned long long)P;
      hi += (P < 0 ? ~0ull : 0ull) + (lo < o ? 1ull : 0ull);
      if (p.X) pl.inc(p.X[puv] ^ p.X[puw] ^ p.X[pvw]);
    }
    // a lane's counters grow by at most one per call that has any hit
    if (__any_sync(kFull, hit) && ++since == (1u << K) - 1u) {
      if (p.X) {
        const int lane = (int)lane_id();
        for (int j = 0; j < 64; j++) {
          const uint32_t v = __reduce_add_sync(kFull, pl.count(j));
          if (lane == (j & 31) && v && g != kEmpty) atomicAdd(&p.worlds[(size_t)g * 64 + j], (unsigned long long)v);
        }
        pl.clear();
      }
      since = 0;
    }
  }
  __device__ void task_begin(uint32_t u) {
    const uint32_t gu = p.vgraph[u];
    if (gu != g) {
      flush();
      g = gu;
    }
  }
  __device__ void task_end(uint32_t) {}
  __device__ void block_end() { flush(); }
};

__global__ void k_batch_finish(int64_t ng, int nt, const unsigned long long* __restrict__ acc, double* expect) {
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < ng; gi += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long T = acc[3 * gi], lo = acc[3 * gi + 1], hi = acc[3 * gi + 2];
    const bool small = (hi == 0ull && !(lo >> 63)) || (hi == ~0ull && (lo >> 63));
    const double sum = (small ? (double)(long long)lo : (double)(long long)hi * 18446744073709551616.0 + (double)lo) *
                       0x1p-45;
    expect[2 * gi] = ((double)T - sum) * 0.5;
    expect[2 * gi + 1] = ((double)T + sum) * 0.5;
  }
}

template <class V>
ubt_status launch_w(const ubt_graph* g, const typename V::P& p, cudaStream_t s) {
  return launch_traversal<V>(g, make_trav_args(g, 0, true), p, s);
}

size_t worlds_table_words(const ubt_graph* g, int64_t W) {
  const int64_t words = W / 64;
  const int64_t wp = std::min<int64_t>(words, tuning().world_words_per_pass);
  return (size_t)std::max<int64_t>(g->m, 1) * (size_t)wp;
}

// the workspace ubt_sample_worlds_workspace_size reports and ubt_sample_worlds requires
size_t worlds_workspace_bytes(const ubt_graph* g, int64_t W) { return worlds_table_words(g, W) * 8 + 256; }

}  // namespace
}  // namespace ubt

using namespace ubt;

extern "C" ubt_status ubt_sample_worlds_workspace_size(const ubt_graph* g, int64_t W, size_t* h_bytes) {
  if (!g || !h_bytes || W < 64 || W % 64) return UBT_ERR_INVALID_ARG;
  *h_bytes = worlds_workspace_bytes(g, W);
  return UBT_OK;
}

extern "C" ubt_status ubt_sample_worlds(ubt_graph* g, uint64_t seed, int64_t W, int64_t* d_bal_per_world,
                                        int64_t* d_total, void* d_workspace, size_t ws_bytes, void* stream) {
  UBT_RANGE("ubt_sample_worlds");
  if (!g || !d_bal_per_world || W < 64 || W % 64 || W / 64 > 0xFFFFFFFFll) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
  if (!d_workspace || ((uintptr_t)d_workspace & 255)) return UBT_ERR_INVALID_ARG;
  if (ws_bytes < worlds_workspace_bytes(g, W)) return UBT_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t words = W / 64;
  int64_t wp = std::min<int64_t>(words, tuning().world_words_per_pass);
  while (words % wp) wp >>= 1;  // passes of equal size
  unsigned long long* X = (unsigned long long*)d_workspace;
  UBT_CUDA(cudaMemsetAsync(d_bal_per_world, 0, sizeof(int64_t) * W, s));
  for (int64_t w0 = 0; w0 < words; w0 += wp) {
    if (g->m > 0) {
      const int grid = (int)std::min<int64_t>((g->m * wp + 255) / 256, (int64_t)g->sm_count * 32);
      k_sign_table<<<grid, 256, 0, s>>>(g->m, g->adj, g->ekey, seed, (uint32_t)w0, (uint32_t)wp, X);
      UBT_CUDA(cudaGetLastError());
    }
    WorldsP p{X, (uint32_t)wp, (unsigned long long*)(d_bal_per_world + w0 * 64)};
    const ubt_status st = wp == 64 ? launch_w<Worlds<2>>(g, p, s) : launch_w<Worlds<1>>(g, p, s);
    if (st != UBT_OK) return st;
  }
  if (d_total) {
    k_world_total<<<1, 1024, 0, s>>>((const unsigned long long*)d_bal_per_world, W, d_total);
    UBT_CUDA(cudaGetLastError());
  }
  return UBT_OK;
}

extern "C" ubt_status ubt_batch_query(ubt_graph* g, const double* h_tau, int32_t n_tau, uint64_t seed,
                                      int64_t* d_counts, double* d_expect, int64_t* d_worlds, void* stream) {
  UBT_RANGE("ubt_batch_query");
  if (!g || !h_tau || !d_counts || n_tau < 1 || n_tau > kBatchTau) return UBT_ERR_INVALID_ARG;
  if (!g->vgraph) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
  BatchP p;
  p.nt = n_tau;
  for (int i = 0; i < n_tau; i++) {
    Level lv;
    if (!tau_level(h_tau[i], &lv)) return UBT_ERR_TAU_OOB;
    p.B[i] = lv.B;
    p.U[i] = lv.U;
  }
  for (int i = n_tau; i < kBatchTau; i++) p.B[i] = p.U[i] = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ng = g->n_graphs;
  p.vgraph = g->vgraph;
  p.counts = (unsigned long long*)d_counts;
  p.acc = d_expect ? g->bacc : nullptr;
  p.worlds = (unsigned long long*)d_worlds;
  p.X = nullptr;
  UBT_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * ng * 2 * n_tau, s));
  if (d_expect) UBT_CUDA(cudaMemsetAsync(g->bacc, 0, sizeof(unsigned long long) * 3 * ng, s));
  if (d_worlds) {
    UBT_CUDA(cudaMemsetAsync(d_worlds, 0, sizeof(int64_t) * ng * 64, s));
    // one sign word per CSR position, kept in the backward accumulators
    if (g->m > 0) {
      const int grid = (int)std::min<int64_t>((g->m + 255) / 256, (int64_t)g->sm_count * 32);
      k_sign_table<<<grid, 256, 0, s>>>(g->m, g->adj, g->ekey, seed, 0u, 1u, g->gacc);
      UBT_CUDA(cudaGetLastError());
    }
    p.X = g->gacc;
  }
  ubt_status st = launch_w<Batch>(g, p, s);
  if (st != UBT_OK) return st;
  if (d_expect) {
    const int grid = (int)std::min<int64_t>((ng + 255) / 256, (int64_t)g->sm_count * 8);
    k_batch_finish<<<std::max(grid, 1), 256, 0, s>>>(ng, n_tau, g->bacc, d_expect);
    UBT_CUDA(cudaGetLastError());
  }
  return UBT_OK;
}
