// ubt_internal.cuh -- data layout and device helpers shared by the libubt
// CUDA sources.  Not part of the public ABI (include/ubt.h is).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/ubt.h"

namespace ubt {

// ---------------------------------------------------------------- layout
//
// Forward CSR under Node Order (Def. Node Order, Sec. 4): row u holds N>(u),
// the neighbours later than u in (degree, id) order.  Each entry is one
// 64-bit word: low 32 bits the neighbour id, high 32 bits the edge value:
//   FIXED graphs: q = 32768 - k as int32 (1 - 2 P+ = q / 2^15)
//   REAL graphs:  s = 1 - 2 p as int32 fixed point, s * 2^30 rounded
// FIXED rows are sorted by |q| descending, ties by neighbour id, so the
// entries a pruning level removes form a suffix of the row (Lemma 2); REAL
// rows by neighbour id.
// eid[pos] is the input index of the edge stored at CSR position pos.
//
// Pairs: every forward edge x-s is one pair of the traversal, owned by the
// endpoint whose list becomes the hash table (the other endpoint's list is
// streamed through it).  pair_ptr / pairs group the pairs by owner; a pair
// word holds the streamed vertex s (low 32 bits) and the CSR position of the
// edge (high 32 bits).

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kWarp = 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

#ifdef __CUDACC__
// lane index and mask of the lower lanes; not volatile, so the compiler keeps
// them in registers instead of re-reading special registers in loops
__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
#endif

__host__ __device__ inline uint32_t adj_col(uint64_t e) { return (uint32_t)e; }
__host__ __device__ inline int32_t adj_q(uint64_t e) { return (int32_t)(uint32_t)(e >> 32); }
__host__ __device__ inline uint32_t adj_valbits(uint64_t e) { return (uint32_t)(e >> 32); }
__host__ __device__ inline uint64_t adj_pack(uint32_t col, uint32_t valbits) {
  return ((uint64_t)valbits << 32) | col;
}

// Edge index (UBT_OPT_EDGE_INDEX): open addressing with linear probing over
// a power-of-two number of 16-byte slots (at least 4m, so at most a quarter
// are used and a miss rarely leaves its first 32-byte sector) -- key min(u, w) << 32 | max(u, w) in the first 8 bytes, the edge
// value in the next 4, so that one 16-byte load reads both; empty slots hold
// the key ~0.
constexpr uint64_t kEdgeIndexEmpty = ~0ull;
__host__ __device__ inline uint64_t edge_index_key(uint32_t a, uint32_t b) {
  return a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
}
__host__ __device__ inline uint64_t edge_index_home(uint64_t key, int shift) {
  return (key * 0x9E3779B97F4A7C15ull) >> shift;  // Fibonacci hashing: the top bits
}
#ifdef __CUDACC__
// 1: edge a-b found (its value in val); 0: absent; -1: the probe bound was
// reached (a self-check: a table at most a quarter full never reaches it)
__device__ __forceinline__ int edge_index_lookup(const uint4* __restrict__ slots, uint64_t mask, int shift, uint32_t a,
                                                 uint32_t b, uint32_t& val) {
  const uint64_t k = edge_index_key(a, b);
  uint64_t h = edge_index_home(k, shift);
  for (uint64_t it = 0; it <= mask; it++) {
    const uint4 sl = slots[h];
    const uint64_t key = ((uint64_t)sl.y << 32) | sl.x;
    if (key == k) {
      val = sl.z;
      return 1;
    }
    if (key == kEdgeIndexEmpty) return 0;
    h = (h + 1) & mask;
  }
  return -1;
}
#endif

#ifdef __CUDACC__
// The stored value of a REAL edge: s = 1 - 2p as a 2^-30 fixed-point int32.
// 1 - 2p is exact in double for float32 p >= 2^-29, and the rounding to the
// 2^-30 grid is exact for p >= 2^-7.
__device__ __forceinline__ uint32_t real_valbits(float p) {
  return (uint32_t)(int32_t)__double2ll_rn((1.0 - 2.0 * (double)p) * 1073741824.0);
}
#endif

// Entries of the queue of long vertex samples (ubt_graph::lqueue).
constexpr int kLongQueue = 1024;

// Query scratch carved from the graph workspace (one per graph).
struct Scratch {
  unsigned long long task[4];       // next giant / hub / small task, spare
  unsigned long long enum_cursor;   // enumeration append cursor
  unsigned long long tri_count;     // triangles seen (expected counts)
  unsigned long long sum_lo;        // 128-bit two's-complement sum, low word
  unsigned long long sum_hi;        // high word
  unsigned long long err;           // device-side error word (build)
  unsigned long long guard;         // first failed self-check of a query (0 = none)
  unsigned long long pad[6];
  unsigned long long hist[2 * 65];  // per-threshold accumulators (bal [0,64), unbal [64,128))
};
constexpr size_t kScratchHeader = 16 * sizeof(unsigned long long);  // zeroed per query

}  // namespace ubt

// The opaque handle of the public ABI.
struct ubt_graph {
  int64_t n = 0, m = 0;
  int32_t kind = 0;
  int64_t n_graphs = 1;
  // device arrays (inside the caller's workspace)
  uint32_t* row_ptr = nullptr;      // n + 1
  uint64_t* adj = nullptr;          // m
  uint32_t* eid = nullptr;          // m: input edge index per CSR position
  uint32_t* ekey = nullptr;         // m: Philox key per CSR position
  uint32_t* pair_ptr = nullptr;     // n + 1: pairs of owner x are [pair_ptr[x], pair_ptr[x+1])
  uint64_t* pairs = nullptr;        // m: streamed vertex | CSR position << 32
  uint32_t* giant_list = nullptr;   // owners whose list is too long for a shared-memory table
  uint32_t* hub_list = nullptr;     // long lists or heavy owners: whole-block tasks
  uint32_t* med_list = nullptr;     // the other owners: one-warp tasks
  uint32_t* vgraph = nullptr;       // batch: graph id of every vertex (or null)
  // undirected adjacency in Absolute Edge Order (UBT_OPT_UNDIRECTED; else null):
  // row x holds every edge at x, |q| descending then neighbour id (Def. AEO
  // restricted to the edges at x), packed like adj
  uint32_t* uptr = nullptr;         // n + 1
  uint64_t* uadj = nullptr;         // 2m
  uint32_t* ueid = nullptr;         // 2m: input edge index
  uint32_t* umir = nullptr;         // 2m: position of the same edge in the other endpoint's row
  uint32_t* uepos = nullptr;        // 2m: [2e + side] position of input edge e in the row of its
                                    //     smaller-id (side 0) / larger-id (side 1) endpoint
  uint32_t* apair_ptr = nullptr;    // n + 1: edges owned by x in the AEO traversal
  uint64_t* apairs = nullptr;       // m: streamed endpoint | position of the edge in x's row << 32
  uint32_t* alist = nullptr;        // owners, by decreasing streamed work
  int64_t n_aowners = 0, n_ablock = 0, max_udeg = 0;  // owners; the first n_ablock are block tasks
  unsigned long long* lqueue = nullptr;  // with the undirected rows: 2 + kLongQueue words, the vertex
                                         // samples a local-count call spreads over all blocks
  uint4* eslots = nullptr;          // edge index (UBT_OPT_EDGE_INDEX; else null): eh_slots slots of
                                    // 16 bytes, key in the first 8, edge value (valbits) in the next 4
  int64_t eh_slots = 0;             // power of two >= max(4m, 64)
  int eh_shift = 64;                // 64 - log2(eh_slots)
  unsigned long long* gacc = nullptr;   // m: backward accumulators
  unsigned long long* bacc = nullptr;   // batch accumulators
  uint32_t* gtab = nullptr;         // global hash tables for very long lists
  int64_t gtab_slots = 0;           // slots per block
  int64_t gtab_blocks = 0;          // blocks that have one
  ubt::Scratch* scratch = nullptr;
  // sizes recorded at build time
  int64_t n_giant = 0, n_hub = 0, n_med = 0;
  int64_t max_out = 0, max_hub_len = 0, wedges = 0, probes = 0;
  int64_t hub_threshold = 0, giant_threshold = 0, block_work = 0, pull = 1;
  int device = 0, sm_count = 0;
};

namespace ubt {

// ---------------------------------------------------------------- tuning

struct Tuning {
  int64_t pull = 1;               // 1: each pair streams the shorter list; 0: always N>(v) (Alg. 1)
  int64_t count_visitor = 0;      // threshold counts: 0 binned in the finding lane, 1 queued per warp
  int64_t block_work = 1 << 14;   // owners streaming more entries are whole-block tasks
  int64_t hub_threshold = 128;    // owners with longer lists are whole-block tasks
  int64_t block_threads = 512;    // threads of the block-task kernel
  int64_t warp_threads = 128;     // threads of the warp-task kernel (at most 128)
  int64_t blocks_per_sm = 32;     // cap on resident blocks (occupancy decides below it)
  int64_t smem_table_max = 8192;  // hash slots of a shared-memory table
  int64_t world_words_per_pass = 8;
  int64_t small_batch = 4;        // warp tasks taken per grab
  int64_t block_unit = 16;        // pairs per warp step in block tasks
  int64_t long_min = 64;          // streamed lists this long are streamed by the whole warp
  int64_t long_tail = 1;          // 1: the last < 64 entries of such a list join the short lists
  int64_t edge_index = 1;         // vertex queries: 0 never look pairs up in the edge index, 1 when cheaper, 2 always
  int64_t vertex_split = 64;      // vertex samples with longer pruned rows are spread over all blocks (edge index)
  int64_t sort_smem_max = 4096;   // longer forward lists are sorted in global memory
  int64_t warp_sort_max = 256;    // lists up to this long are sorted by one warp in registers
};
Tuning& tuning();

// ---------------------------------------------------------------- host helpers

#define UBT_CUDA(call)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      ubt::set_last_cuda_error(e_, #call, __FILE__, __LINE__); \
      return UBT_ERR_CUDA;                                \
    }                                                     \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// An NVTX range over a host scope (the build's phases, each query's launch
// and finish), so that a timeline profiler shows where the library's calls
// begin and end.  Costs nothing measurable when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// Consecutive phases of one scope: next() closes the open range and opens
// the next; the last closes with the scope.
struct NvtxPhases {
  bool open = false;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhases() {
    if (open) nvtxRangePop();
  }
};
#define UBT_RANGE_CAT2(a, b) a##b
#define UBT_RANGE_CAT(a, b) UBT_RANGE_CAT2(a, b)
#define UBT_RANGE(name) ::ubt::NvtxRange UBT_RANGE_CAT(ubt_range_, __LINE__)(name)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over the caller's workspace.
struct Carver {
  char* base;
  size_t off = 0;
  size_t cap;
  Carver(void* b, size_t c) : base((char*)b), cap(c) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = (T*)(base ? base + off : nullptr);
    off += sizeof(T) * count;
    return p;
  }
};

// thresholds of one t (exact): c = 2t - 1, X = c * 2^45;
//   balanced   <=> P <= B = -ceil(X)
//   unbalanced <=> P >  U =  floor(X)
//   prune level L = ceil(X): a triangle with |P| < L is neither
struct Level {
  int64_t B, U, L;
};
bool tau_level(double tau, Level* out);

// device workspace needed for the global hash tables of a graph
int64_t gtab_slots_for(int64_t m);

// hash-table slots for a list of `entries` entries: a power of two >= 4x (min 32)
inline int64_t table_slots(int64_t entries) {
  int64_t s = 32;
  while (s < 4 * entries) s <<= 1;
  return s;
}

// launch helpers implemented in ubt_scan.cu
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp,
                               cudaStream_t s);
size_t scan_tmp_words(int64_t n);

}  // namespace ubt
