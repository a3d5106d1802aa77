// ubt_noalloc.cu -- a threshold-count entry point that needs no device memory
// from its caller beyond the graph, the thresholds and the output.
//
// Some callers cannot allocate device memory at the point where they query:
// code running where the process's allocator belongs to another framework
// (a plugin that may only use the buffers it is handed), real-time loops that
// must not call into an allocator, or code that only receives pre-built
// objects.  ubt_count_threshold itself uses the scratch area inside the
// graph's workspace; this variant instead keeps its per-call scratch (task
// counters, self-check word, per-threshold accumulators) in a fixed array in
// the library's own device memory.
#include <mutex>

#include "ubt_internal.cuh"

namespace ubt {
ubt_status count_reg_at(const ubt_graph* g, const double* h_tau, int n_tau, int prune, int64_t* d_counts,
                        Scratch* sc, unsigned long long* acc, cudaStream_t s);
}

using namespace ubt;

namespace {

// The fixed scratch: a Scratch header followed by 2 x 8 64-bit accumulators.
// Every GPU that loads the library holds these bytes until the process exits.
constexpr size_t kNoallocBytes = 2048;
constexpr int kNoallocMaxTau = 8;
static_assert(sizeof(Scratch) + 2 * kNoallocMaxTau * sizeof(unsigned long long) <= kNoallocBytes,
              "fixed scratch too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The array's device address on each device, taken once per device with that
// device current.  In host code the array's name is only a host-side stand-in,
// so the address must come from cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];

// The array of the graph's device; that device must be the current one, as
// every launch of the call goes to the current device.
ubt_status scratch_address(const ubt_graph* g, void** out) {
  int dev = 0;
  UBT_CUDA(cudaGetDevice(&dev));
  if (dev != g->device || dev < 0 || dev >= kMaxDevices) return UBT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    UBT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return UBT_OK;
}

// The fixed array's self-check word goes to the graph's own (first failure
// wins there too), so that ubt_query_guard reports a failed check of this
// call although the next call clears the array.
__global__ void k_merge_guard(const Scratch* from, Scratch* to) {
  const unsigned long long w = from->guard;
  if (w) atomicCAS(&to->guard, 0ull, w);
}

}  // namespace

extern "C" ubt_status ubt_count_threshold_noalloc(ubt_graph* g, const double* h_tau, int32_t n_tau, int32_t prune,
                                                  int64_t* d_counts, void* stream) {
  UBT_RANGE("ubt_count_threshold_noalloc");
  if (!g || !d_counts || !h_tau) return UBT_ERR_INVALID_ARG;
  if (n_tau < 1 || n_tau > kNoallocMaxTau) return UBT_ERR_SCRATCH_LIMIT;
  void* base = nullptr;
  ubt_status st = scratch_address(g, &base);
  if (st != UBT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear counters and accumulators
  UBT_CUDA(cudaMemsetAsync(base, 0, kNoallocBytes, s));
  Scratch* sc = (Scratch*)base;
  unsigned long long* acc = (unsigned long long*)((char*)base + sizeof(Scratch));
  st = count_reg_at(g, h_tau, n_tau, prune, d_counts, sc, acc, s);
  if (st != UBT_OK) return st;
  k_merge_guard<<<1, 1, 0, s>>>(sc, g->scratch);
  UBT_CUDA(cudaGetLastError());
  return UBT_OK;
}
