// ubt_query.cu -- threshold counting, enumeration, expected counts and their
// adjoint: visitors fused into the traversal of ubt_traverse.cuh.
//
// Per triangle with edge values q_uv, q_uw, q_vw (FIXED: q = 32768 - k):
//   P = q_uv q_uw q_vw  (exact int64; P / 2^45 = (1-2p_uv)(1-2p_uw)(1-2p_vw))
//   P_bal = (1 - P/2^45) / 2     (the four-term sum of Sec. 3 in product form)
//   t-balanced   (Def. 4, P_bal >= t)   <=>  P <= B = -ceil((2t-1) 2^45)
//   t-unbalanced (Def. 5, P_unbal > t)  <=>  P >  U =  floor((2t-1) 2^45)
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "ubt_aeo.cuh"
#include "ubt_traverse.cuh"

namespace ubt {

namespace {

constexpr int kMaxTau = 64;

// register cap of the counting visitors' kernels (launch bounds)
#ifndef UBT_COUNT_REGCAP
#define UBT_COUNT_REGCAP 64
#endif

__device__ __forceinline__ int64_t tri_product(uint32_t a, uint32_t b, uint32_t c) {
  // |q| <= 2^15, so q_a q_b fits int32 (<= 2^30); the third factor widens to int64
  return (int64_t)((int32_t)a * (int32_t)b) * (int64_t)(int32_t)c;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
  return x;
}

// 128-bit two's-complement accumulator (lo, hi)
struct Acc128 {
  unsigned long long lo = 0, hi = 0;
  __device__ __forceinline__ void add(long long x) {
    const unsigned long long o = lo;
    lo += (unsigned long long)x;
    hi += (x < 0 ? ~0ull : 0ull) + (lo < o ? 1ull : 0ull);
  }
  __device__ __forceinline__ void add128(unsigned long long l, unsigned long long h) {
    const unsigned long long o = lo;
    lo += l;
    hi += h + (lo < o ? 1ull : 0ull);
  }
  __device__ void warp_reduce() {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const unsigned long long l = __shfl_xor_sync(kFull, lo, d);
      const unsigned long long h = __shfl_xor_sync(kFull, hi, d);
      add128(l, h);
    }
  }
  // exact 128-bit add into global (lo, hi) words: each add's own carry goes to hi
  __device__ void flush(unsigned long long* glo, unsigned long long* ghi) const {
    const unsigned long long o = atomicAdd(glo, lo);
    const unsigned long long c = (o + lo < o) ? 1ull : 0ull;
    atomicAdd(ghi, hi + c);
  }
};

// ------------------------------------------------------------ visitors

// Up to 8 thresholds: per-thread counters in registers, compared with every
// threshold (padding thresholds never match).  32-bit counters are flushed to
// the 64-bit globals before they can wrap.
constexpr int kRegTau = 8;
struct CountRegP {
  int64_t B[kRegTau], U[kRegTau];
  unsigned long long* out;  // [0, NT) balanced, [NT, 2 NT) unbalanced
};
// A warp collects the products P of its triangles in a shared-memory queue
// and counts them 32 at a time, so the counting runs on full warps.  The
// queue holds fewer than 32 between steps; a step adds at most 32 and a
// batched pair of steps at most 64.
constexpr int kHitQueue = 96;

// Appends the products of two probe steps' hits to a warp queue (q, qn); the
// caller drains it below 32 afterwards.  All lanes, converged.
__device__ __forceinline__ void enqueue_pair(long long* q, uint32_t& qn, bool h0, bool h1, uint32_t quv,
                                             uint32_t quw0, uint32_t qvw0, uint32_t quw1, uint32_t qvw1) {
  const unsigned lt = lanemask_lt();
  const unsigned m0 = __ballot_sync(kFull, h0);
  const unsigned m1 = __ballot_sync(kFull, h1);
  const uint32_t n0 = qn + __popc(m0);
  if (h0) q[qn + __popc(m0 & lt)] = tri_product(quv, quw0, qvw0);
  if (h1) q[n0 + __popc(m1 & lt)] = tri_product(quv, quw1, qvw1);
  qn = n0 + __popc(m1);
}

// Moves queue entries [32, qn) (fewer than 64) to the front.
__device__ __forceinline__ void queue_shift32(long long* q, uint32_t& qn) {
  const uint32_t lane = lane_id();
  const uint32_t rest = qn - 32;
  const long long a = lane < rest ? q[32 + lane] : 0;
  const long long b = lane + 32 < rest ? q[64 + lane] : 0;
  __syncwarp();
  if (lane < rest) q[lane] = a;
  if (lane + 32 < rest) q[32 + lane] = b;
  qn = rest;
  __syncwarp();
}

template <int NT>
struct CountReg {
  using P = CountRegP;
  static constexpr bool kPos = false;
  static constexpr bool kBatched = true;
  static constexpr int kRegCap = UBT_COUNT_REGCAP;
  static __host__ __device__ int smem_bytes(int threads) { return (threads / 32) * kHitQueue * 8; }
  int64_t B[NT], U[NT];
  unsigned long long* out;
  long long* q;  // this warp's queue of products
  uint32_t qn = 0;
  uint32_t bal[NT], unbal[NT];
  uint32_t since = 0;
  __device__ CountReg(const P& p, char* smem) : out(p.out) {
    q = (long long*)smem + (threadIdx.x >> 5) * kHitQueue;
#pragma unroll
    for (int i = 0; i < NT; i++) {
      B[i] = p.B[i];
      U[i] = p.U[i];
      bal[i] = unbal[i] = 0;
    }
  }
  __device__ void block_init() {}
  __device__ __forceinline__ void count(long long P) {
#pragma unroll
    for (int i = 0; i < NT; i++) {
      bal[i] += (P <= B[i]) ? 1u : 0u;
      unbal[i] += (P > U[i]) ? 1u : 0u;
    }
    since++;
  }
  // count the first 32 queued products, move the rest to the front
  __device__ void drain32() {
    const int lane = (int)lane_id();
    __syncwarp();
    const long long mine = q[lane];
    queue_shift32(q, qn);
    count(mine);
  }
  __device__ void drain_all() {
    const int lane = (int)lane_id();
    __syncwarp();
    if ((uint32_t)lane < qn) count(q[lane]);
    qn = 0;
    __syncwarp();
  }
  __device__ __forceinline__ void step(bool hit, uint32_t, uint32_t, uint32_t, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t, uint32_t, uint32_t) {
    const unsigned m = __ballot_sync(kFull, hit);
    if (!m) return;
    const int lane = (int)lane_id();
    if (hit) q[qn + __popc(m & lanemask_lt())] = tri_product(quv, quw, qvw);
    qn += __popc(m);
    if (qn >= 32) drain32();
  }
  template <int U>
  __device__ __forceinline__ void steps(const bool (&hit)[U], uint32_t quv, const uint32_t (&quw)[U],
                                        const uint32_t (&qvw)[U]) {
    static_assert(U % 2 == 0, "steps come in pairs");
#pragma unroll
    for (int s = 0; s < U; s += 2) {
      if (__any_sync(kFull, hit[s] || hit[s + 1])) {
        enqueue_pair(q, qn, hit[s], hit[s + 1], quv, quw[s], qvw[s], quw[s + 1], qvw[s + 1]);
        while (qn >= 32) drain32();
      }
    }
  }
  __device__ void task_begin(uint32_t) {}
  __device__ void flush() {
#pragma unroll
    for (int i = 0; i < NT; i++) {
      const uint32_t b = __reduce_add_sync(kFull, bal[i]);
      const uint32_t u = __reduce_add_sync(kFull, unbal[i]);
      if (lane_id() == 0) {
        if (b) atomicAdd(&out[i], (unsigned long long)b);
        if (u) atomicAdd(&out[NT + i], (unsigned long long)u);
      }
      bal[i] = unbal[i] = 0;
    }
    since = 0;
  }
  // a warp's 32 lanes sum to < 2^32 while every lane has counted fewer than 2^26
  __device__ void task_end(uint32_t) {
    if (__any_sync(kFull, since >= (1u << 26))) flush();
  }
  __device__ void block_end() {
    drain_all();
    flush();
  }
};

__global__ void k_finish_reg(const unsigned long long* __restrict__ acc, int nt, int NT, const int* perm_unused,
                             int64_t* __restrict__ out) {
  const int i = threadIdx.x;
  (void)perm_unused;
  if (i < nt) {
    out[i] = (int64_t)acc[i];
    out[nt + i] = (int64_t)acc[NT + i];
  }
}

// Many thresholds (up to 64), tested all at once.  The 2 nt levels -- every B
// and every U, sorted ascending (each B <= 0 <= each U) -- cut the integers
// into 2 nt + 1 intervals; a product P falls in interval r = #{levels < P}.
// Products are queued per warp as in CountReg; 32 at a time, each lane finds
// the interval of one product by binary search and adds 1 to that interval's
// bin (a block-wide shared histogram).  Then, with B_(k) and U_(k) the k-th
// smallest levels of each kind,
//   #{P <= B_(k)} = #{r <= k}           (P <= B_(k) iff fewer than k+1 B's are < P)
//   #{P >  U_(k)} = #{r > nt + k}       (P >  U_(k) iff at least k+1 U's are < P,
//                                        and then every B is < P too)
static_assert(UBT_LB_THREADS <= 512, "CountMulti's 32-bit bins assume at most 16 warps a block");
constexpr int kMultiLevels = 256;  // padded table of levels: 2^K > 2 kMaxTau
constexpr int kMultiBins = 2 * kMaxTau + 1;
struct CountMultiP {
  int nt;
  int half;                        // 2^(K-1), with 2^K the smallest power of two > 2 nt
  int64_t S[2 * kMaxTau];          // the 2 nt levels, ascending
  unsigned long long* out;         // global bins [0, 2 nt]
};
struct CountMulti {
  using P = CountMultiP;
  static constexpr bool kPos = false;
  static constexpr bool kBatched = true;
  static constexpr int kRegCap = UBT_COUNT_REGCAP;
  static __host__ __device__ int smem_bytes(int threads) {
    return kMultiLevels * 8 + ((kMultiBins * 4 + 15) / 16) * 16 + (threads / 32) * kHitQueue * 8;
  }
  unsigned long long* out;
  const long long* S;  // shared: levels, padded with INT64_MAX
  uint32_t* bins;      // shared: block histogram
  long long* q;        // shared: this warp's queue of products
  uint32_t qn = 0;
  uint32_t since = 0;  // products this warp binned since its last flush (warp-uniform)
  int nt, half;
  __device__ CountMulti(const P& p, char* smem) : out(p.out), nt(p.nt), half(p.half) {
    long long* s = (long long*)smem;
    S = s;
    bins = (uint32_t*)(smem + kMultiLevels * 8);
    q = (long long*)(smem + kMultiLevels * 8 + ((kMultiBins * 4 + 15) / 16) * 16) + (threadIdx.x >> 5) * kHitQueue;
    for (int i = threadIdx.x; i < kMultiLevels; i += blockDim.x) s[i] = i < 2 * p.nt ? p.S[i] : INT64_MAX;
    for (int i = threadIdx.x; i < kMultiBins; i += blockDim.x) bins[i] = 0;
  }
  __device__ void block_init() {}
  // interval of P: the largest r with S[r - 1] < P (S[-1] = -inf); the padding
  // is never < P, and 2^K > 2 nt, so r = #{levels < P}
  __device__ __forceinline__ void bin(long long P) {
    int r = 0;
    for (int b = half; b > 0; b >>= 1)
      if (S[r + b - 1] < P) r += b;
    atomicAdd(&bins[r], 1u);
  }
  // Bins are moved to the global counters with exchanges, so a flush by one
  // warp never loses another warp's increments.  A warp flushes once it has
  // binned 2^26 products, so a bin holds fewer than 16 x (2^26 + 32) < 2^32
  // (at most 16 warps a block).
  __device__ void flush() {
#pragma unroll 1
    for (int i = (int)lane_id(); i <= 2 * nt; i += 32) {
      const uint32_t v = atomicExch(&bins[i], 0u);
      if (v) atomicAdd(&out[i], (unsigned long long)v);
    }
    since = 0;
  }
  __device__ void drain32() {
    const int lane = (int)lane_id();
    __syncwarp();
    const long long mine = q[lane];
    queue_shift32(q, qn);
    bin(mine);
    since += 32;
    if (since >= (1u << 26)) flush();
  }
  __device__ void drain_all() {
    const int lane = (int)lane_id();
    __syncwarp();
    if ((uint32_t)lane < qn) bin(q[lane]);
    since += qn;
    qn = 0;
    __syncwarp();
  }
  __device__ __forceinline__ void step(bool hit, uint32_t, uint32_t, uint32_t, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t, uint32_t, uint32_t) {
    const unsigned m = __ballot_sync(kFull, hit);
    if (!m) return;
    if (hit) q[qn + __popc(m & lanemask_lt())] = tri_product(quv, quw, qvw);
    qn += __popc(m);
    if (qn >= 32) drain32();
  }
  template <int U>
  __device__ __forceinline__ void steps(const bool (&hit)[U], uint32_t quv, const uint32_t (&quw)[U],
                                        const uint32_t (&qvw)[U]) {
    static_assert(U % 2 == 0, "steps come in pairs");
#pragma unroll
    for (int s = 0; s < U; s += 2) {
      if (__any_sync(kFull, hit[s] || hit[s + 1])) {
        enqueue_pair(q, qn, hit[s], hit[s + 1], quv, quw[s], qvw[s], quw[s + 1], qvw[s + 1]);
        while (qn >= 32) drain32();
      }
    }
  }
  __device__ void task_begin(uint32_t) {}
  __device__ void task_end(uint32_t) {}
  __device__ void block_end() {
    drain_all();
    __syncthreads();
    if (threadIdx.x < 32) flush();
  }
};

// Any number of thresholds (up to 64), classified in the lane that found the
// triangle, without a queue.  The 2 nt levels S (every B and every U,
// ascending) cut the integers into 2 nt + 1 intervals; P falls in interval
// r = #{S_j < P}, counted in bin r (finished by k_finish_multi).  r is found
// with a slice table: P + 2^45 in [0, 2^46] is cut into 2049 slices of 2^35;
// slice i records b0 = #{S_j < its start} and the number c of levels inside
// it, so r = b0 + #{S_j < P, b0 <= j < b0 + c} (c is 0 or 1 unless two
// thresholds lie within 2^35 / 2^45 = 2^-10 of each other).  Bins 0 and 2 nt
// (P classified at every threshold, the common case for confident edges)
// are per-lane register counters; the others are 32-bit counters in shared
// memory, one set per warp, incremented without reading the old value.
//
// Overflow bound: a warp adds at most one per probed entry, and the bins are
// moved to the global bins (an atomic exchange with 0, then a 64-bit add;
// the exchange keeps adds made meanwhile) before a bin can reach 2^32:
//   * degree-ordered traversal (CountBins): the warp counts the entries
//     of each batch of pairs (probed(n); forward lists are shorter than
//     sqrt(2m) < 2^17, so a batch of 32 lists counts at most 2^23), and lane
//     0 moves the bins once the count reaches kWarpFlush = 2^31;
//   * Alg. 2 kernels (CountBinsAeo, rows of any length): every lane counts
//     the entries it was handed and moves the bins itself once its count
//     reaches kBinFlush, so a bin holds fewer than 32 x 2^27 adds.
constexpr int kSlices = 2049;
// moves bins [1, top) to the global bins: an atomic exchange with 0 keeps the
// adds other lanes make meanwhile (out of line: it runs at most once per
// kBinFlush entries of a lane or kWarpFlush entries of a warp)
static __device__ __noinline__ void count_bins_flush(uint32_t* bins, unsigned long long* out, int top) {
  for (int i = 1; i < top; i++) {
    const uint32_t v = atomicExch(&bins[i], 0u);
    if (v) atomicAdd(&out[i], (unsigned long long)v);
  }
}
constexpr int kBinStride = 144;                  // 32-bit words per warp's bins (>= 2 kMaxTau + 1)
constexpr uint32_t kBinFlush = (1u << 27) - 64;  // entries per lane between flushes (Alg. 2 kernels)
constexpr uint32_t kWarpFlush = 1u << 31;         // entries per warp between flushes (batch counts)
struct CountBinsP {
  int nt;
  int64_t S[2 * kMaxTau];   // the 2 nt levels, ascending
  unsigned long long* out;  // global bins [0, 2 nt]
};
struct CountBins {
  using P = CountBinsP;
  static constexpr bool kPos = false;
  static constexpr bool kBatched = true;
  static constexpr int kRegCap = UBT_COUNT_REGCAP;
  static constexpr int kTabBytes = ((kSlices * 2 + 15) / 16) * 16;
  static __host__ __device__ int smem_bytes(int threads) {
    return kTabBytes + 2 * kMaxTau * 8 + (threads / 32) * kBinStride * 4;
  }
  const uint16_t* tab;  // shared: slice table, b0 | c << 8
  const long long* S;   // shared: levels
  uint32_t* bins;       // shared: this warp's bins
  uint32_t* all;        // shared: every warp's bins, kBinStride words each
  unsigned long long* out;
  unsigned long long first = 0, last = 0;  // bins 0 and 2 nt of this lane
  uint32_t since = 0;                       // entries since the last flush (this lane's or the warp's)
  int top;                                  // 2 nt
  __device__ CountBins(const P& p, char* smem) : out(p.out), top(2 * p.nt) {
    uint16_t* t = (uint16_t*)smem;
    long long* sv = (long long*)(smem + kTabBytes);
    uint32_t* b = (uint32_t*)(smem + kTabBytes + 2 * kMaxTau * 8);
    tab = t;
    S = sv;
    all = b;
    bins = b + (threadIdx.x >> 5) * kBinStride;
    for (int i = threadIdx.x; i < 2 * p.nt; i += blockDim.x) sv[i] = p.S[i];
    for (int i = threadIdx.x; i < (int)(blockDim.x >> 5) * kBinStride; i += blockDim.x) b[i] = 0;
    for (int i = threadIdx.x; i < kSlices; i += blockDim.x) {
      const long long start = (long long)i * (1ll << 35) - (1ll << 45);
      const long long end = start + (1ll << 35);
      int b0 = 0, b1 = 0;  // #{S < start}, #{S < end}
      for (int j = 0; j < 2 * p.nt; j++) {
        b0 += p.S[j] < start ? 1 : 0;
        b1 += p.S[j] < end ? 1 : 0;
      }
      t[i] = (uint16_t)(b0 | ((b1 - b0) << 8));
    }
  }
  __device__ void block_init() {}
  __device__ __forceinline__ void count(long long P) {
    const uint32_t e = tab[(uint32_t)((unsigned long long)(P + (1ll << 45)) >> 35)];
    int r = (int)(e & 0xFFu);
    const int c = (int)(e >> 8);
    if (c) {
      const int b0 = r;
      for (int j = 0; j < c; j++) r += S[b0 + j] < P ? 1 : 0;
    }
    if (r == 0) {
      first++;
    } else if (r == top) {
      last++;
    } else {
      atomicAdd(&bins[r], 1u);
    }
  }
  __device__ __forceinline__ void step(bool hit, uint32_t, uint32_t, uint32_t, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t, uint32_t, uint32_t) {
    if (hit) count(tri_product(quv, quw, qvw));
  }
  template <int U>
  __device__ __forceinline__ void steps(const bool (&hit)[U], uint32_t quv, const uint32_t (&quw)[U],
                                        const uint32_t (&qvw)[U]) {
#pragma unroll
    for (int s = 0; s < U; s++)
      if (hit[s]) count(tri_product(quv, quw[s], qvw[s]));
  }
  // the degree-ordered traversal's batch count (all lanes, the same n)
  __device__ __forceinline__ void probed(uint32_t n) {
    since += n;
    if (since >= kWarpFlush) {
      if (lane_id() == 0) count_bins_flush(bins, out, top);
      since = 0;
    }
  }
  __device__ void task_begin(uint32_t) {}
  __device__ void task_end(uint32_t) {}
  __device__ void block_end() {
    const unsigned long long f = warp_sum(first), l = warp_sum(last);
    if (lane_id() == 0) {
      if (f) atomicAdd(&out[0], f);
      if (l) atomicAdd(&out[top], l);
    }
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    for (int i = threadIdx.x + 1; i < top; i += blockDim.x) {
      unsigned long long v = 0;
      for (int w = 0; w < nw; w++) v += all[w * kBinStride + i];
      if (v) atomicAdd(&out[i], v);
    }
  }
};

// CountBins for the Alg. 2 kernels, whose rows have any length: every lane
// counts the entries it was handed and moves its warp's bins itself
struct CountBinsAeo : CountBins {
  using CountBins::CountBins;
  __device__ __forceinline__ void step(bool hit, uint32_t u, uint32_t v, uint32_t w, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t puv, uint32_t puw, uint32_t pvw) {
    CountBins::step(hit, u, v, w, quv, quw, qvw, puv, puw, pvw);
    if (++since >= kBinFlush) {
      count_bins_flush(bins, out, top);
      since = 0;
    }
  }
};

struct FinishMulti {
  int nt;
  int perm[kMaxTau];  // caller index of the i-th smallest threshold
};

// bins -> counts: the i-th smallest t has the (nt-1-i)-th smallest B and the
// i-th smallest U
__global__ void k_finish_multi(const unsigned long long* __restrict__ bins, FinishMulti f, int64_t* __restrict__ out) {
  const int i = threadIdx.x;
  if (i < f.nt) {
    unsigned long long b = 0, u = 0;
    for (int r = 0; r <= f.nt - 1 - i; r++) b += bins[r];
    for (int r = f.nt + i + 1; r <= 2 * f.nt; r++) u += bins[r];
    out[f.perm[i]] = (int64_t)b;
    out[f.nt + f.perm[i]] = (int64_t)u;
  }
}

// balanced records: Blo < P <= B; unbalanced: U < P <= Uhi (top-k uses the
// extra bounds; the threshold queries pass INT64_MIN / INT64_MAX)
struct EnumP {
  int64_t B, U;
  int which;
  ubt_tri_rec* out;
  unsigned long long cap;
  unsigned long long* cursor;
  int64_t Blo = INT64_MIN, Uhi = INT64_MAX;
};
struct Enum {
  using P = EnumP;
  static constexpr bool kPos = false;
  static constexpr bool kBatched = false;
  static constexpr int kRegCap = 64;
  static __host__ __device__ int smem_bytes(int) { return 0; }
  P p;
  __device__ Enum(const P& p_, char*) : p(p_) {}
  __device__ void block_init() {}
  __device__ __forceinline__ void step(bool hit, uint32_t u, uint32_t v, uint32_t w, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t, uint32_t, uint32_t) {
    uint32_t cls = 0;
    int64_t P = 0;
    if (hit) {
      P = tri_product(quv, quw, qvw);
      if ((p.which & 1) && P <= p.B && P > p.Blo) cls = 1;
      else if ((p.which & 2) && P > p.U && P <= p.Uhi) cls = 2;
    }
    const unsigned m = __ballot_sync(kFull, cls != 0);
    if (!m) return;
    const int lane = (int)lane_id();
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(p.cursor, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (cls) {
      const unsigned long long idx = base + __popc(m & lanemask_lt());
      if (idx < p.cap) {
        uint32_t a = u, b = v, c = w, t;
        if (a > b) { t = a; a = b; b = t; }
        if (b > c) { t = b; b = c; c = t; }
        if (a > b) { t = a; a = b; b = t; }
        ubt_tri_rec r;
        r.u = a; r.v = b; r.w = c; r.cls = cls;
        // P_bal = (2^45 - P) / 2^46, exact in double (|numerator| <= 2^46)
        r.p_bal = (double)((1ll << 45) - P) * 0x1p-46;
        p.out[idx] = r;
      }
    }
  }
  __device__ void task_begin(uint32_t) {}
  __device__ void task_end(uint32_t) {}
  __device__ void block_end() {}
};

struct ExpectP {
  unsigned long long* tri;      // triangle count
  unsigned long long* sum_lo;   // 128-bit sum
  unsigned long long* sum_hi;
};
// FIXED: sum of P exactly.  REAL: sum of S = s_uv s_uw s_vw, each s a 2^-30
// fixed-point integer: s_uv s_uw is exact in int64 (2^-60), rounded to 2^-30,
// times s_vw exact (2^-60), rounded to 2^-32; summed in 128-bit integers.
template <bool kReal>
struct Expect {
  using P = ExpectP;
  static constexpr bool kPos = false;
  static constexpr bool kBatched = false;
  static constexpr int kRegCap = 64;
  static __host__ __device__ int smem_bytes(int) { return 0; }
  P p;
  Acc128 acc;
  unsigned long long cnt = 0;
  __device__ Expect(const P& p_, char*) : p(p_) {}
  __device__ void block_init() {}
  __device__ __forceinline__ void step(bool hit, uint32_t, uint32_t, uint32_t, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t, uint32_t, uint32_t) {
    if (!hit) return;
    cnt++;
    if (kReal) {
      const long long a = (long long)(int32_t)quv * (int32_t)quw;          // 2^-60
      const long long a30 = (a + (1ll << 29)) >> 30;                        // 2^-30
      const long long s60 = a30 * (long long)(int32_t)qvw;                  // 2^-60
      acc.add((s60 + (1ll << 27)) >> 28);                                   // 2^-32
    } else {
      acc.add(tri_product(quv, quw, qvw));
    }
  }
  __device__ void task_begin(uint32_t) {}
  __device__ void task_end(uint32_t) {}
  __device__ void block_end() {
    acc.warp_reduce();
    const unsigned long long c = warp_sum(cnt);
    if (lane_id() == 0 && c) {
      atomicAdd(p.tri, c);
      acc.flush(p.sum_lo, p.sum_hi);
    }
  }
};

__device__ double i128_to_double(unsigned long long lo, unsigned long long hi) {
  // value = hi * 2^64 + lo with hi signed; values that fit in int64 convert
  // with one rounding (the two-part sum would cancel for small negatives)
  if ((hi == 0ull && !(lo >> 63)) || (hi == ~0ull && (lo >> 63))) return (double)(long long)lo;
  return (double)(long long)hi * 18446744073709551616.0 + (double)lo;
}

__global__ void k_finish_expect(const Scratch* sc, int real, double* out, int64_t* exact) {
  const unsigned long long T = sc->tri_count, lo = sc->sum_lo, hi = sc->sum_hi;
  double sum;  // sum of S_t
  if (real) sum = i128_to_double(lo, hi) * 0x1p-32;
  else sum = i128_to_double(lo, hi) * 0x1p-45;
  if (out) {
    out[0] = ((double)T - sum) * 0.5;
    out[1] = ((double)T + sum) * 0.5;
  }
  if (exact) {
    exact[0] = (int64_t)T;
    exact[1] = (int64_t)lo;
    exact[2] = (int64_t)hi;
    exact[3] = 0;
  }
}

struct AdjointP {
  unsigned long long* acc;  // per CSR position
};
// d E_bal / d p_e = sum over triangles through e of s_f s_g (f, g the other edges)
template <bool kReal>
struct Adjoint {
  using P = AdjointP;
  static constexpr bool kPos = true;
  static constexpr bool kBatched = false;
  static constexpr int kRegCap = 64;
  static __host__ __device__ int smem_bytes(int) { return 0; }
  P p;
  __device__ Adjoint(const P& p_, char*) : p(p_) {}
  __device__ void block_init() {}
  __device__ __forceinline__ void step(bool hit, uint32_t, uint32_t, uint32_t, uint32_t quv, uint32_t quw,
                                       uint32_t qvw, uint32_t puv, uint32_t puw, uint32_t pvw) {
    if (!hit) return;
    long long a_uv, a_uw, a_vw;
    if (kReal) {
      // products of two 2^-30 fixed-point values are exact in int64 (2^-60);
      // rounded to 2^-40 for accumulation
      const long long su = (int32_t)quv, sw = (int32_t)quw, sv = (int32_t)qvw;
      a_uv = (sw * sv + (1ll << 19)) >> 20;
      a_uw = (su * sv + (1ll << 19)) >> 20;
      a_vw = (su * sw + (1ll << 19)) >> 20;
    } else {
      a_uv = (long long)((int32_t)quw * (int32_t)qvw);    // exact, scale 2^-30
      a_uw = (long long)((int32_t)quv * (int32_t)qvw);
      a_vw = (long long)((int32_t)quv * (int32_t)quw);
    }
    atomicAdd(&p.acc[puv], (unsigned long long)a_uv);
    atomicAdd(&p.acc[puw], (unsigned long long)a_uw);
    atomicAdd(&p.acc[pvw], (unsigned long long)a_vw);
  }
  __device__ void task_begin(uint32_t) {}
  __device__ void task_end(uint32_t) {}
  __device__ void block_end() {}
};

__global__ void k_finish_adjoint(int64_t m, const unsigned long long* __restrict__ acc, const uint32_t* __restrict__ eid,
                                 const double* __restrict__ gout, double scale, float* __restrict__ grad) {
  const double g = (gout[0] - gout[1]) * scale;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    grad[eid[i]] = (float)(g * (double)(long long)acc[i]);
}

// traversal sizes (same task and pruning rules as the traversal); one warp
// per owner.  out: [0] table entries, [1] pairs probed, [2] streamed
// entries, [3] tasks
__global__ void k_trav_stats(int64_t n, const uint32_t* __restrict__ row_ptr, const uint64_t* __restrict__ adj,
                             const uint32_t* __restrict__ pair_ptr, const uint64_t* __restrict__ pairs, int64_t L,
                             uint32_t light, unsigned long long* out) {
  const int lane = (int)lane_id();
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long tab = 0, npairs = 0, str = 0, tasks = 0;
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps) {
    const uint32_t rs = row_ptr[x];
    uint32_t len = row_ptr[x + 1] - rs;
    const uint32_t ps = pair_ptr[x], pe = pair_ptr[x + 1];
    if (len < 2 || pe == ps) continue;
    int64_t qmax = 0;
    if (L > 0) {
      qmax = qabs(adj_valbits(adj[rs]));
      len = prune_prefix(adj + rs, len, 1ll << 30, L);
    }
    if (len == 0) continue;
    if (lane == 0) {
      tab += len;
      tasks += 1;
    }
    for (uint32_t i = ps + lane; i < pe; i += 32) {
      const uint64_t d = pairs[i];
      const uint32_t sv = (uint32_t)d;
      const int64_t qe = qabs(adj_valbits(adj[(uint32_t)(d >> 32)]));
      if (L > 0 && qe * (1ll << 30) < L) continue;
      const uint32_t vs = row_ptr[sv];
      uint32_t dv = row_ptr[sv + 1] - vs;
      if (L > 0 && !light) dv = prune_prefix(adj + vs, dv, qe * qmax, L);
      npairs += 1;
      str += dv;
    }
  }
  tab = warp_sum(tab);
  npairs = warp_sum(npairs);
  str = warp_sum(str);
  tasks = warp_sum(tasks);
  if (lane == 0) {
    atomicAdd(&out[0], tab);
    atomicAdd(&out[1], npairs);
    atomicAdd(&out[2], str);
    atomicAdd(&out[3], tasks);
  }
}

// ------------------------------------------------------------ launching

}  // namespace

TravArgs make_trav_args(const ubt_graph* g, int64_t L, bool with_pos) {
  (void)with_pos;
  const Tuning& T = tuning();
  TravArgs a;
  a.row_ptr = g->row_ptr;
  a.adj = g->adj;
  a.pair_ptr = g->pair_ptr;
  a.pairs = g->pairs;
  a.giant_list = g->giant_list;
  a.hub_list = g->hub_list;
  a.med_list = g->med_list;
  a.n_giant = (uint32_t)g->n_giant;
  a.n_hub = (uint32_t)g->n_hub;
  a.n_med = (uint32_t)g->n_med;
  a.n = (uint32_t)g->n;
  a.m = (uint32_t)g->m;
  a.sc = g->scratch;
  a.gtab = g->gtab;
  a.gtab_slots = (uint32_t)g->gtab_slots;
  a.gtab_blocks = g->n_giant ? (uint32_t)g->gtab_blocks : 0u;
  a.hub_slots = g->n_hub ? (uint32_t)table_slots(g->max_hub_len) : 0u;
  // a warp table holds one medium task's list (at most hub_threshold entries)
  a.warp_slots = (uint32_t)table_slots(g->hub_threshold);
  a.unit = (uint32_t)std::min<int64_t>(32, std::max<int64_t>(1, T.block_unit));
  a.batch = (uint32_t)std::max<int64_t>(1, T.small_batch);
  a.long_min = (uint32_t)T.long_min;
  a.long_tail = (uint32_t)T.long_tail;
  a.L = L;
  a.light_prune = light_prune_for(L);
  return a;
}

template <class V>
ubt_status launch_traverse(const ubt_graph* g, const typename V::P& p, int64_t L, cudaStream_t s) {
  return launch_traversal<V>(g, make_trav_args(g, L, V::kPos), p, s);
}

// Threshold counts (at most kRegTau thresholds) whose per-call scratch -- the
// task counters and guard word (`sc`) and the 2 x kRegTau accumulators
// (`acc`) -- lives at the given device addresses instead of the graph's own
// scratch area.  Used by the no-allocation entry point.
ubt_status count_reg_at(const ubt_graph* g, const double* h_tau, int n_tau, int prune, int64_t* d_counts,
                        Scratch* sc, unsigned long long* acc, cudaStream_t s) {
  if (g->kind != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
  if (!h_tau || n_tau < 1 || n_tau > kRegTau) return UBT_ERR_INVALID_ARG;
  Level lv[kRegTau];
  int64_t L = INT64_MAX;
  for (int i = 0; i < n_tau; i++) {
    if (!tau_level(h_tau[i], &lv[i])) return UBT_ERR_TAU_OOB;
    L = std::min(L, lv[i].L);
  }
  if (!prune) L = 0;
  const int NT = n_tau <= 1 ? 1 : n_tau <= 2 ? 2 : n_tau <= 4 ? 4 : 8;
  CountRegP p;
  for (int i = 0; i < kRegTau; i++) {
    p.B[i] = i < n_tau ? lv[i].B : INT64_MIN;
    p.U[i] = i < n_tau ? lv[i].U : INT64_MAX;
  }
  p.out = acc;
  TravArgs a = make_trav_args(g, L, false);
  a.sc = sc;
  ubt_status st = UBT_OK;
  switch (NT) {
    case 1: st = launch_traversal<CountReg<1>>(g, a, p, s); break;
    case 2: st = launch_traversal<CountReg<2>>(g, a, p, s); break;
    case 4: st = launch_traversal<CountReg<4>>(g, a, p, s); break;
    default: st = launch_traversal<CountReg<8>>(g, a, p, s); break;
  }
  if (st != UBT_OK) return st;
  k_finish_reg<<<1, kRegTau, 0, s>>>(acc, n_tau, NT, nullptr, d_counts);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}

}  // namespace ubt

using namespace ubt;

namespace {

ubt_status check_taus(const double* h_tau, int n_tau, std::vector<Level>& lv) {
  if (!h_tau || n_tau < 1 || n_tau > kMaxTau) return UBT_ERR_INVALID_ARG;
  lv.resize(n_tau);
  for (int i = 0; i < n_tau; i++)
    if (!tau_level(h_tau[i], &lv[i])) return UBT_ERR_TAU_OOB;
  return UBT_OK;
}

}  // namespace

namespace {

// Threshold counts through the degree-ordered traversal, or through the edge
// iteration in Absolute Edge Order (aeo).
template <class V>
ubt_status launch_count(const ubt_graph* g, const typename V::P& p, int64_t L, bool aeo, cudaStream_t s) {
  return aeo ? launch_aeo<V>(g, L, p, s) : launch_traverse<V>(g, p, L, s);
}

ubt_status count_impl(ubt_graph* g, const double* h_tau, int32_t n_tau, int32_t prune, int64_t* d_counts,
                      bool aeo, cudaStream_t s) {
  if (!g || !d_counts) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
  if (aeo && !g->uptr) return UBT_ERR_UNSUPPORTED;
  std::vector<Level> lv;
  ubt_status st = check_taus(h_tau, n_tau, lv);
  if (st != UBT_OK) return st;
  // thresholds in ascending t: B descending, U ascending
  std::vector<int> order(n_tau);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lv[x].L < lv[y].L; });
  const int64_t L = prune ? lv[order[0]].L : 0;
  const int64_t visitor = tuning().count_visitor;
  if (visitor == 0) {
    CountBinsP p;
    p.nt = n_tau;
    for (int i = 0; i < n_tau; i++) {
      p.S[i] = lv[order[n_tau - 1 - i]].B;  // B ascending: t descending
      p.S[n_tau + i] = lv[order[i]].U;      // U ascending: t ascending
    }
    p.out = g->scratch->hist;
    UBT_CUDA(cudaMemsetAsync(g->scratch->hist, 0, sizeof(g->scratch->hist), s));
    st = aeo ? launch_aeo<CountBinsAeo>(g, L, p, s) : launch_traverse<CountBins>(g, p, L, s);
    if (st != UBT_OK) return st;
    FinishMulti f;
    f.nt = n_tau;
    for (int i = 0; i < n_tau; i++) f.perm[i] = order[i];
    k_finish_multi<<<1, kMaxTau, 0, s>>>(g->scratch->hist, f, d_counts);
    UBT_CUDA(cudaGetLastError());
    return UBT_OK;
  }
  if (n_tau <= kRegTau) {
    const int NT = n_tau <= 1 ? 1 : n_tau <= 2 ? 2 : n_tau <= 4 ? 4 : 8;
    CountRegP p;
    for (int i = 0; i < kRegTau; i++) {
      p.B[i] = i < n_tau ? lv[i].B : INT64_MIN;  // padding: never balanced
      p.U[i] = i < n_tau ? lv[i].U : INT64_MAX;  // padding: never unbalanced
    }
    unsigned long long* acc = g->scratch->hist;
    p.out = acc;
    UBT_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 2 * NT, s));
    switch (NT) {
      case 1: st = launch_count<CountReg<1>>(g, p, L, aeo, s); break;
      case 2: st = launch_count<CountReg<2>>(g, p, L, aeo, s); break;
      case 4: st = launch_count<CountReg<4>>(g, p, L, aeo, s); break;
      default: st = launch_count<CountReg<8>>(g, p, L, aeo, s); break;
    }
    if (st != UBT_OK) return st;
    k_finish_reg<<<1, kRegTau, 0, s>>>(acc, n_tau, NT, nullptr, d_counts);
    UBT_CUDA(cudaGetLastError());
    return UBT_OK;
  }
  CountMultiP p;
  p.nt = n_tau;
  p.half = 1;
  while (2 * p.half <= 2 * n_tau) p.half *= 2;  // 2 half > 2 nt
  for (int i = 0; i < n_tau; i++) {
    p.S[i] = lv[order[n_tau - 1 - i]].B;  // B ascending: t descending
    p.S[n_tau + i] = lv[order[i]].U;      // U ascending: t ascending
  }
  p.out = g->scratch->hist;
  UBT_CUDA(cudaMemsetAsync(g->scratch->hist, 0, sizeof(g->scratch->hist), s));
  st = launch_count<CountMulti>(g, p, L, aeo, s);
  if (st != UBT_OK) return st;
  FinishMulti f;
  f.nt = n_tau;
  for (int i = 0; i < n_tau; i++) f.perm[i] = order[i];
  k_finish_multi<<<1, kMaxTau, 0, s>>>(g->scratch->hist, f, d_counts);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}

}  // namespace

extern "C" ubt_status ubt_count_threshold(ubt_graph* g, const double* h_tau, int32_t n_tau, int32_t prune,
                                          int64_t* d_counts, void* stream) {
  UBT_RANGE("ubt_count_threshold");
  return count_impl(g, h_tau, n_tau, prune, d_counts, false, (cudaStream_t)stream);
}

extern "C" ubt_status ubt_count_aeo(ubt_graph* g, const double* h_tau, int32_t n_tau, int64_t* d_counts,
                                    void* stream) {
  UBT_RANGE("ubt_count_aeo");
  return count_impl(g, h_tau, n_tau, 1, d_counts, true, (cudaStream_t)stream);
}

namespace {

ubt_status enumerate_impl(ubt_graph* g, double tau, int32_t which, int32_t prune, ubt_tri_rec* d_out,
                          int64_t capacity, int64_t* h_n_found, bool aeo, cudaStream_t s) {
  if (!g || !h_n_found || capacity < 0 || (capacity > 0 && !d_out)) return UBT_ERR_INVALID_ARG;
  if (which < 1 || which > 3) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
  if (aeo && !g->uptr) return UBT_ERR_UNSUPPORTED;
  Level lv;
  if (!tau_level(tau, &lv)) return UBT_ERR_TAU_OOB;
  EnumP p{lv.B, lv.U, which, d_out, (unsigned long long)capacity, &g->scratch->enum_cursor};
  ubt_status st = aeo ? launch_aeo<Enum>(g, lv.L, p, s) : launch_traverse<Enum>(g, p, prune ? lv.L : 0, s);
  if (st != UBT_OK) return st;
  unsigned long long found = 0;
  UBT_CUDA(cudaMemcpyAsync(&found, &g->scratch->enum_cursor, sizeof(found), cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  *h_n_found = (int64_t)found;
  return found > (unsigned long long)capacity ? UBT_ERR_CAPACITY : UBT_OK;
}

}  // namespace

extern "C" ubt_status ubt_enumerate(ubt_graph* g, double tau, int32_t which, int32_t prune, ubt_tri_rec* d_out,
                                    int64_t capacity, int64_t* h_n_found, void* stream) {
  UBT_RANGE("ubt_enumerate");
  return enumerate_impl(g, tau, which, prune, d_out, capacity, h_n_found, false, (cudaStream_t)stream);
}

extern "C" ubt_status ubt_enumerate_aeo(ubt_graph* g, double tau, int32_t which, ubt_tri_rec* d_out,
                                        int64_t capacity, int64_t* h_n_found, void* stream) {
  UBT_RANGE("ubt_enumerate_aeo");
  return enumerate_impl(g, tau, which, 1, d_out, capacity, h_n_found, true, (cudaStream_t)stream);
}

extern "C" ubt_status ubt_expected_counts(ubt_graph* g, double* d_out, int64_t* d_exact, void* stream) {
  UBT_RANGE("ubt_expected_counts");
  if (!g || (!d_out && !d_exact)) return UBT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ExpectP p{&g->scratch->tri_count, &g->scratch->sum_lo, &g->scratch->sum_hi};
  ubt_status st = g->kind == UBT_GRAPH_REAL ? launch_traverse<Expect<true>>(g, p, 0, s)
                                            : launch_traverse<Expect<false>>(g, p, 0, s);
  if (st != UBT_OK) return st;
  k_finish_expect<<<1, 1, 0, s>>>(g->scratch, g->kind == UBT_GRAPH_REAL, d_out, d_exact);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}

extern "C" ubt_status ubt_expected_counts_backward(ubt_graph* g, const double* d_gout, float* d_grad_p,
                                                   void* stream) {
  UBT_RANGE("ubt_expected_counts_backward");
  if (!g || !d_gout || (!d_grad_p && g->m > 0)) return UBT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (g->m == 0) return UBT_OK;
  UBT_CUDA(cudaMemsetAsync(g->gacc, 0, sizeof(unsigned long long) * g->m, s));
  AdjointP p{g->gacc};
  const bool real = g->kind == UBT_GRAPH_REAL;
  ubt_status st = real ? launch_traverse<Adjoint<true>>(g, p, 0, s) : launch_traverse<Adjoint<false>>(g, p, 0, s);
  if (st != UBT_OK) return st;
  const int grid = (int)std::min<int64_t>((g->m + 255) / 256, (int64_t)g->sm_count * 16);
  k_finish_adjoint<<<grid, 256, 0, s>>>(g->m, g->gacc, g->eid, d_gout, real ? 0x1p-40 : 0x1p-30, d_grad_p);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}

extern "C" ubt_status ubt_traversal_stats(ubt_graph* g, const double* h_tau, int32_t n_tau, int32_t prune,
                                          int64_t* h_out, void* stream) {
  if (!g || !h_out) return UBT_ERR_INVALID_ARG;
  int64_t L = 0;
  if (prune) {
    if (g->kind != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
    std::vector<Level> lv;
    ubt_status st = check_taus(h_tau, n_tau, lv);
    if (st != UBT_OK) return st;
    L = lv[0].L;
    for (const Level& x : lv) L = std::min(L, x.L);
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* d = &g->scratch->hist[0];
  UBT_CUDA(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), s));
  if (g->n > 0) {
    const int grid = (int)std::min<int64_t>((g->n + 7) / 8, (int64_t)g->sm_count * 16);
    k_trav_stats<<<grid, 256, 0, s>>>(g->n, g->row_ptr, g->adj, g->pair_ptr, g->pairs, L, light_prune_for(L), d);
    UBT_CUDA(cudaGetLastError());
  }
  unsigned long long h[4];
  UBT_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < 4; i++) h_out[i] = (int64_t)h[i];
  return UBT_OK;
}

extern "C" ubt_status ubt_query_guard(ubt_graph* g, int64_t* h_word, void* stream) {
  if (!g || !h_word) return UBT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long w = 0;
  UBT_CUDA(cudaMemcpyAsync(&w, &g->scratch->guard, sizeof(w), cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaMemsetAsync(&g->scratch->guard, 0, sizeof(w), s));
  UBT_CUDA(cudaStreamSynchronize(s));
  *h_word = (int64_t)w;
  return UBT_OK;
}

extern "C" ubt_status ubt_graph_export(const ubt_graph* g, uint32_t* h_row_ptr, uint64_t* h_adj, uint32_t* h_eid,
                                       uint32_t* h_lists, int64_t* h_list_sizes, void* stream) {
  if (!g) return UBT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (h_row_ptr)
    UBT_CUDA(cudaMemcpyAsync(h_row_ptr, g->row_ptr, sizeof(uint32_t) * (g->n + 1), cudaMemcpyDeviceToHost, s));
  if (h_adj && g->m)
    UBT_CUDA(cudaMemcpyAsync(h_adj, g->adj, sizeof(uint64_t) * g->m, cudaMemcpyDeviceToHost, s));
  if (h_eid && g->m)
    UBT_CUDA(cudaMemcpyAsync(h_eid, g->eid, sizeof(uint32_t) * g->m, cudaMemcpyDeviceToHost, s));
  const int64_t tasks = g->n_giant + g->n_hub + g->n_med;
  if (h_lists && tasks)
    UBT_CUDA(cudaMemcpyAsync(h_lists, g->giant_list, sizeof(uint32_t) * tasks, cudaMemcpyDeviceToHost, s));
  if (h_list_sizes) {
    h_list_sizes[0] = g->n_giant;
    h_list_sizes[1] = g->n_hub;
    h_list_sizes[2] = g->n_med;
    h_list_sizes[3] = 0;
  }
  UBT_CUDA(cudaStreamSynchronize(s));
  return UBT_OK;
}

// ------------------------------------------------------------ top-k

namespace ubt {
namespace {

// record order of a top-k answer: P_bal descending (balanced) or ascending
// (unbalanced), then (u, v, w)
__device__ __forceinline__ bool rec_before(const ubt_tri_rec& a, const ubt_tri_rec& b, bool desc) {
  if (a.p_bal != b.p_bal) return desc ? a.p_bal > b.p_bal : a.p_bal < b.p_bal;
  if (a.u != b.u) return a.u < b.u;
  if (a.v != b.v) return a.v < b.v;
  return a.w < b.w;
}

// one step of a bitonic network whose comparators all put the earlier record
// first (the first step of every merge pairs i with its mirror); positions
// >= n act as records after every record and are skipped
__global__ void k_sort_recs_step(ubt_tri_rec* r, uint32_t n, uint32_t kk, uint32_t j, int desc) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t ixj = (j == (kk >> 1)) ? (i ^ (kk - 1)) : (i ^ j);
    if (ixj > i && ixj < n) {
      const ubt_tri_rec a = r[i], b = r[ixj];
      if (rec_before(b, a, desc != 0)) {
        r[i] = b;
        r[ixj] = a;
      }
    }
  }
}

ubt_status sort_records(ubt_tri_rec* r, uint32_t n, bool desc, int sms, cudaStream_t s) {
  uint32_t cap = 2;
  while (cap < n) cap <<= 1;
  const int grid = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sms * 8);
  for (uint32_t kk = 2; kk <= cap; kk <<= 1)
    for (uint32_t j = kk >> 1; j > 0; j >>= 1)
      k_sort_recs_step<<<std::max(grid, 1), 256, 0, s>>>(r, n, kk, j, desc ? 1 : 0);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}

// Counts of the triangle products P among up to 128 sorted levels in one
// pruned traversal: h_bins[r] = #{P : #{levels < P} = r}.
ubt_status count_levels(const ubt_graph* g, const std::vector<int64_t>& lev, int64_t L, unsigned long long* h_bins,
                        cudaStream_t s) {
  CountBinsP p;
  p.nt = (int)lev.size() / 2;
  for (size_t i = 0; i < lev.size(); i++) p.S[i] = lev[i];
  p.out = g->scratch->hist;
  UBT_CUDA(cudaMemsetAsync(g->scratch->hist, 0, sizeof(g->scratch->hist), s));
  ubt_status st = launch_traverse<CountBins>(g, p, L, s);
  if (st != UBT_OK) return st;
  UBT_CUDA(cudaMemcpyAsync(h_bins, g->scratch->hist, sizeof(unsigned long long) * (lev.size() + 1),
                           cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  return UBT_OK;
}

// records with P in the given bounds appended to r[at, cap): returns how many
// exist (all of them, even past cap)
ubt_status enum_range(const ubt_graph* g, int which, int64_t B, int64_t Blo, int64_t U, int64_t Uhi, int64_t L,
                      ubt_tri_rec* r, int64_t cap, int64_t* found, cudaStream_t s) {
  EnumP p{B, U, which, r, (unsigned long long)std::max<int64_t>(cap, 0), &g->scratch->enum_cursor, Blo, Uhi};
  ubt_status st = launch_traverse<Enum>(g, p, L, s);
  if (st != UBT_OK) return st;
  unsigned long long f = 0;
  UBT_CUDA(cudaMemcpyAsync(&f, &g->scratch->enum_cursor, sizeof(f), cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  *found = (int64_t)f;
  return UBT_OK;
}

int64_t topk_capacity(int64_t K) {
  int64_t c = 1;
  while (c < std::max<int64_t>(2 * K, K + 4096)) c <<= 1;
  return c;
}

constexpr int64_t kP1 = 1ll << 45;  // |P| <= 2^45

}  // namespace
}  // namespace ubt

extern "C" ubt_status ubt_topk_workspace_size(int64_t K, size_t* h_bytes) {
  if (!h_bytes || K < 1 || K > (1ll << 26)) return UBT_ERR_INVALID_ARG;
  *h_bytes = (size_t)topk_capacity(K) * sizeof(ubt_tri_rec);
  return UBT_OK;
}

extern "C" ubt_status ubt_topk(ubt_graph* g, int64_t K, int32_t which, ubt_tri_rec* d_out, int64_t* h_n_out,
                               void* d_work, size_t work_bytes, void* stream) {
  UBT_RANGE("ubt_topk");
  if (!g || !d_out || !h_n_out || !d_work || K < 1 || K > (1ll << 26)) return UBT_ERR_INVALID_ARG;
  if (which != 1 && which != 2) return UBT_ERR_INVALID_ARG;
  if (g->kind != UBT_GRAPH_FIXED) return UBT_ERR_UNSUPPORTED;
  const int64_t cap = topk_capacity(K);
  if (work_bytes < (size_t)cap * sizeof(ubt_tri_rec)) return UBT_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  ubt_tri_rec* cand = (ubt_tri_rec*)d_work;
  const bool bal = which == 1;
  // Balanced: the K largest P_bal are the K smallest P.  Keep lo < hi with
  // #{P <= lo} < K <= #{P <= hi}, and narrow (lo, hi] 64-fold per pass by
  // counting P at 64 cuts, until the triangles up to hi fit the candidate
  // buffer or hi = lo + 1.  Each pass prunes at the level its interval
  // allows (the raised threshold of Sec. 5's top-k adaptation): a triangle
  // with |P| below max(0, -hi) cannot have P <= hi.  Unbalanced mirrors it
  // with #{P >= x}: keep #{P >= hi} < K <= #{P >= lo}.
  int64_t lo = bal ? -kP1 - 1 : -kP1, hi = bal ? kP1 : kP1 + 1;
  int64_t n_in = -1;  // triangles in the final range
  for (int pass = 0; pass < 16; pass++) {
    // 64 cuts, non-decreasing (strictly increasing when the range allows):
    // balanced in (lo, hi] ending at hi, unbalanced in [lo, hi) starting at lo
    std::vector<int64_t> cuts(64);
    const __int128 span = (__int128)hi - lo;
    for (int j = 0; j < 64; j++) cuts[j] = lo + (int64_t)((span * (bal ? j + 1 : j) + 63) / 64);
    std::vector<int64_t> lev(64);
    for (int j = 0; j < 64; j++) lev[j] = bal ? cuts[j] : cuts[j] - 1;  // P <= c  |  P >= c  <=>  P > c - 1
    std::sort(lev.begin(), lev.end());
    unsigned long long bins[129];
    const int64_t L = bal ? std::max<int64_t>(0, -hi) : std::max<int64_t>(0, lo);
    ubt_status st = count_levels(g, lev, L, bins, s);
    if (st != UBT_OK) return st;
    int64_t cum[64];
    if (bal) {
      int64_t acc = 0;
      for (int j = 0; j < 64; j++) { acc += (int64_t)bins[j]; cum[j] = acc; }  // #{P <= cuts[j]}
      int jj = 0;
      while (jj < 63 && cum[jj] < K) jj++;
      if (cum[jj] < K) {  // fewer than K triangles in all: take them all
        n_in = cum[jj];
        hi = cuts[jj];
        break;
      }
      const int64_t nlo = jj > 0 ? cuts[jj - 1] : lo;
      hi = cuts[jj];
      lo = nlo;
      n_in = cum[jj];
    } else {
      int64_t acc = 0;
      for (int j = 63; j >= 0; j--) { acc += (int64_t)bins[j + 1]; cum[j] = acc; }  // #{P >= cuts[j]}
      if (cum[0] < K) {  // cuts[0] = lo: fewer than K triangles in all: take them all
        n_in = cum[0];
        break;
      }
      int jj = 63;
      while (cum[jj] < K) jj--;
      hi = jj < 63 ? cuts[jj + 1] : hi;
      lo = cuts[jj];
      n_in = cum[jj];
    }
    if (n_in <= cap || hi - lo <= 1) break;
  }
  // candidates: every triangle strictly inside the answer (fewer than K), then
  // the triangles of the last range, as many as fit
  int64_t n1 = 0, n2 = 0;
  ubt_status st;
  if (bal) {
    st = enum_range(g, 1, lo, INT64_MIN, 0, 0, std::max<int64_t>(0, -lo), cand, cap, &n1, s);
    if (st != UBT_OK) return st;
    st = enum_range(g, 1, hi, lo, 0, 0, std::max<int64_t>(0, -hi), cand + std::min(n1, cap), cap - std::min(n1, cap),
                    &n2, s);
  } else {
    st = enum_range(g, 2, 0, 0, hi - 1, INT64_MAX, std::max<int64_t>(0, hi), cand, cap, &n1, s);
    if (st != UBT_OK) return st;
    st = enum_range(g, 2, 0, 0, lo - 1, hi - 1, std::max<int64_t>(0, lo), cand + std::min(n1, cap),
                    cap - std::min(n1, cap), &n2, s);
  }
  if (st != UBT_OK) return st;
  const int64_t have = std::min(n1 + n2, cap);
  st = sort_records(cand, (uint32_t)have, bal, g->sm_count, s);
  if (st != UBT_OK) return st;
  const int64_t nout = std::min(have, K);
  if (nout > 0)
    UBT_CUDA(cudaMemcpyAsync(d_out, cand, sizeof(ubt_tri_rec) * nout, cudaMemcpyDeviceToDevice, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  *h_n_out = nout;
  return UBT_OK;
}

extern "C" ubt_status ubt_graph_export_undirected(const ubt_graph* g, uint32_t* h_uptr, uint64_t* h_uadj,
                                                  uint32_t* h_ueid, uint32_t* h_umir, uint32_t* h_apair_ptr,
                                                  uint64_t* h_apairs, void* stream) {
  if (!g) return UBT_ERR_INVALID_ARG;
  if (!g->uptr) return UBT_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t m2 = (size_t)(2 * g->m);
  if (h_uptr) UBT_CUDA(cudaMemcpyAsync(h_uptr, g->uptr, sizeof(uint32_t) * (g->n + 1), cudaMemcpyDeviceToHost, s));
  if (h_uadj && m2) UBT_CUDA(cudaMemcpyAsync(h_uadj, g->uadj, sizeof(uint64_t) * m2, cudaMemcpyDeviceToHost, s));
  if (h_ueid && m2) UBT_CUDA(cudaMemcpyAsync(h_ueid, g->ueid, sizeof(uint32_t) * m2, cudaMemcpyDeviceToHost, s));
  if (h_umir && m2) UBT_CUDA(cudaMemcpyAsync(h_umir, g->umir, sizeof(uint32_t) * m2, cudaMemcpyDeviceToHost, s));
  if (h_apair_ptr)
    UBT_CUDA(cudaMemcpyAsync(h_apair_ptr, g->apair_ptr, sizeof(uint32_t) * (g->n + 1), cudaMemcpyDeviceToHost, s));
  if (h_apairs && g->m)
    UBT_CUDA(cudaMemcpyAsync(h_apairs, g->apairs, sizeof(uint64_t) * g->m, cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  return UBT_OK;
}

extern "C" ubt_status ubt_graph_export_pairs(const ubt_graph* g, uint32_t* h_pair_ptr, uint64_t* h_pairs,
                                             void* stream) {
  if (!g) return UBT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (h_pair_ptr)
    UBT_CUDA(cudaMemcpyAsync(h_pair_ptr, g->pair_ptr, sizeof(uint32_t) * (g->n + 1), cudaMemcpyDeviceToHost, s));
  if (h_pairs && g->m)
    UBT_CUDA(cudaMemcpyAsync(h_pairs, g->pairs, sizeof(uint64_t) * g->m, cudaMemcpyDeviceToHost, s));
  UBT_CUDA(cudaStreamSynchronize(s));
  return UBT_OK;
}
