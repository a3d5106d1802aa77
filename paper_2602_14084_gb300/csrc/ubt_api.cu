// ubt_api.cu -- status strings, tuning knobs, exact thresholds and the
// end-to-end host-memory entry point of libubt.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "ubt_internal.cuh"

namespace ubt {

Tuning& tuning() {
  static Tuning t;
  return t;
}

static char g_last_error[512];

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

// Thresholds of one t, exactly (Defs. 4-5 with P = q_uv q_uw q_vw, P/2^45 = S):
//   P_bal >= t   <=>  (1 - P/2^45)/2 >= t  <=>  P <= -(2t-1) 2^45  <=>  P <= -ceil(X)
//   P_unbal > t  <=>  (1 + P/2^45)/2 >  t  <=>  P >   (2t-1) 2^45  <=>  P >  floor(X)
// with X = (2t-1) 2^45.  For t in [0.5, 1], 2t-1 is exact (Sterbenz) and so is
// the scaling by 2^45.  Any classified triangle has |P| >= ceil(X) = L.
bool tau_level(double tau, Level* out) {
  if (!(tau >= 0.5 && tau <= 1.0)) return false;
  const double X = ldexp(2.0 * tau - 1.0, 45);
  out->B = -(int64_t)ceil(X);
  out->U = (int64_t)floor(X);
  out->L = (int64_t)ceil(X);
  return true;
}

}  // namespace ubt

using namespace ubt;

extern "C" const char* ubt_status_str(ubt_status s) {
  switch (s) {
    case UBT_OK: return "ok";
    case UBT_ERR_INVALID_ARG: return "invalid argument";
    case UBT_ERR_SELF_LOOP: return "self-loop in edge list";
    case UBT_ERR_DUPLICATE_EDGE: return "duplicate edge in edge list";
    case UBT_ERR_VERTEX_OOB: return "vertex id out of range";
    case UBT_ERR_PROB_OOB: return "edge probability out of range";
    case UBT_ERR_TAU_OOB: return "threshold outside [0.5, 1]";
    case UBT_ERR_CAPACITY: return "enumeration output capacity too small";
    case UBT_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case UBT_ERR_TIMEOUT: return "device wait timed out";
    case UBT_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA runtime error";
    case UBT_ERR_UNSUPPORTED: return "operation not supported for this graph kind";
    case UBT_ERR_SCRATCH_LIMIT: return "request exceeds the fixed scratch array of this entry point";
    default: return "unknown status";
  }
}

extern "C" int32_t ubt_version(void) { return 1 * 10000 + 0 * 100 + 0; }

extern "C" ubt_status ubt_set_tuning(const char* name, int64_t value) {
  if (!name) return UBT_ERR_INVALID_ARG;
  Tuning& t = tuning();
  if (!strcmp(name, "hub_threshold")) {
    if (value < 2 || value > 4096) return UBT_ERR_INVALID_ARG;
    t.hub_threshold = value;
  } else if (!strcmp(name, "block_threads")) {
    if (value < 64 || value > 512 || value % 32) return UBT_ERR_INVALID_ARG;
    t.block_threads = value;
  } else if (!strcmp(name, "warp_threads")) {
    if (value < 64 || value > 512 || value % 32) return UBT_ERR_INVALID_ARG;
    t.warp_threads = value;
  } else if (!strcmp(name, "blocks_per_sm")) {
    if (value < 1 || value > 32) return UBT_ERR_INVALID_ARG;
    t.blocks_per_sm = value;
  } else if (!strcmp(name, "smem_table_max")) {
    if (value < 64 || value > (1 << 20) || (value & (value - 1))) return UBT_ERR_INVALID_ARG;
    t.smem_table_max = value;
  } else if (!strcmp(name, "world_words_per_pass")) {
    if (value < 1 || value > 64 || (value & (value - 1))) return UBT_ERR_INVALID_ARG;
    t.world_words_per_pass = value;
  } else if (!strcmp(name, "small_batch")) {
    if (value < 1 || value > 1024) return UBT_ERR_INVALID_ARG;
    t.small_batch = value;
  } else if (!strcmp(name, "count_visitor")) {
    if (value < 0 || value > 1) return UBT_ERR_INVALID_ARG;
    t.count_visitor = value;
  } else if (!strcmp(name, "pull")) {
    if (value < 0 || value > 1) return UBT_ERR_INVALID_ARG;
    t.pull = value;
  } else if (!strcmp(name, "block_work")) {
    if (value < 1 || value > (1ll << 40)) return UBT_ERR_INVALID_ARG;
    t.block_work = value;
  } else if (!strcmp(name, "block_unit")) {
    if (value < 1 || value > 32) return UBT_ERR_INVALID_ARG;
    t.block_unit = value;
  } else if (!strcmp(name, "long_min")) {
    if (value < 1 || value > (1 << 20)) return UBT_ERR_INVALID_ARG;
    t.long_min = value;
  } else if (!strcmp(name, "long_tail")) {
    if (value < 0 || value > 1) return UBT_ERR_INVALID_ARG;
    t.long_tail = value;
  } else if (!strcmp(name, "vertex_split")) {
    if (value < 1 || value > (1ll << 32)) return UBT_ERR_INVALID_ARG;
    t.vertex_split = value;
  } else if (!strcmp(name, "edge_index")) {
    if (value < 0 || value > 2) return UBT_ERR_INVALID_ARG;
    t.edge_index = value;
  } else if (!strcmp(name, "sort_smem_max")) {
    if (value < 64 || value > 4096 || (value & (value - 1))) return UBT_ERR_INVALID_ARG;
    t.sort_smem_max = value;
  } else if (!strcmp(name, "warp_sort_max")) {
    if (value != 128 && value != 256 && value != 512) return UBT_ERR_INVALID_ARG;
    t.warp_sort_max = value;
  } else {
    return UBT_ERR_INVALID_ARG;
  }
  return UBT_OK;
}

extern "C" ubt_status ubt_get_tuning(const char* name, int64_t* h_value) {
  if (!name || !h_value) return UBT_ERR_INVALID_ARG;
  const Tuning& t = tuning();
  if (!strcmp(name, "hub_threshold")) *h_value = t.hub_threshold;
  else if (!strcmp(name, "block_threads")) *h_value = t.block_threads;
  else if (!strcmp(name, "warp_threads")) *h_value = t.warp_threads;
  else if (!strcmp(name, "blocks_per_sm")) *h_value = t.blocks_per_sm;
  else if (!strcmp(name, "smem_table_max")) *h_value = t.smem_table_max;
  else if (!strcmp(name, "world_words_per_pass")) *h_value = t.world_words_per_pass;
  else if (!strcmp(name, "small_batch")) *h_value = t.small_batch;
  else if (!strcmp(name, "sort_smem_max")) *h_value = t.sort_smem_max;
  else if (!strcmp(name, "warp_sort_max")) *h_value = t.warp_sort_max;
  else if (!strcmp(name, "pull")) *h_value = t.pull;
  else if (!strcmp(name, "count_visitor")) *h_value = t.count_visitor;
  else if (!strcmp(name, "block_work")) *h_value = t.block_work;
  else if (!strcmp(name, "block_unit")) *h_value = t.block_unit;
  else if (!strcmp(name, "long_min")) *h_value = t.long_min;
  else if (!strcmp(name, "long_tail")) *h_value = t.long_tail;
  else if (!strcmp(name, "edge_index")) *h_value = t.edge_index;
  else if (!strcmp(name, "vertex_split")) *h_value = t.vertex_split;
  else return UBT_ERR_INVALID_ARG;
  return UBT_OK;
}

// ---------------------------------------------------------------- end to end

namespace {
struct HostLayout {
  uint32_t* src;
  uint32_t* dst;
  uint32_t* k;
  int64_t* counts;
  char* graph_ws;
  size_t graph_bytes;
  size_t total;
};

bool host_layout(int64_t n, int64_t m, void* ws, HostLayout* L) {
  size_t gb = 0;
  if (ubt_graph_workspace_size(n, m, UBT_GRAPH_FIXED, nullptr, &gb) != UBT_OK) return false;
  Carver c(ws, 0);
  L->src = c.take<uint32_t>(std::max<int64_t>(m, 1));
  L->dst = c.take<uint32_t>(std::max<int64_t>(m, 1));
  L->k = c.take<uint32_t>(std::max<int64_t>(m, 1));
  L->counts = c.take<int64_t>(128);
  L->graph_ws = c.take<char>(gb);
  L->graph_bytes = gb;
  L->total = c.off + 256;
  return true;
}
}  // namespace

extern "C" ubt_status ubt_count_host_workspace_size(int64_t n, int64_t m, size_t* h_bytes) {
  if (!h_bytes) return UBT_ERR_INVALID_ARG;
  HostLayout L;
  if (!host_layout(n, m, nullptr, &L)) return UBT_ERR_INVALID_ARG;
  *h_bytes = L.total;
  return UBT_OK;
}

extern "C" ubt_status ubt_count_host(int64_t n, int64_t m, const uint32_t* h_src, const uint32_t* h_dst,
                                     const uint32_t* h_k, const double* h_tau, int32_t n_tau, int32_t prune,
                                     int64_t* h_counts, void* d_workspace, size_t ws_bytes, void* stream) {
  UBT_RANGE("ubt_count_host");
  if (!h_counts || !d_workspace || ((uintptr_t)d_workspace & 255)) return UBT_ERR_INVALID_ARG;
  if (m > 0 && (!h_src || !h_dst || !h_k)) return UBT_ERR_INVALID_ARG;
  if (n_tau < 1 || n_tau > 64) return UBT_ERR_INVALID_ARG;
  HostLayout L;
  if (!host_layout(n, m, d_workspace, &L)) return UBT_ERR_INVALID_ARG;
  if (ws_bytes < L.total) return UBT_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  if (m > 0) {
    UBT_CUDA(cudaMemcpyAsync(L.src, h_src, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, s));
    UBT_CUDA(cudaMemcpyAsync(L.dst, h_dst, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, s));
    UBT_CUDA(cudaMemcpyAsync(L.k, h_k, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, s));
  }
  ubt_graph* g = nullptr;
  ubt_status st = ubt_create_graph(n, m, L.src, L.dst, L.k, nullptr, UBT_GRAPH_FIXED, nullptr, L.graph_ws,
                                   L.graph_bytes, stream, &g);
  if (st != UBT_OK) return st;
  st = ubt_count_threshold(g, h_tau, n_tau, prune, L.counts, stream);
  if (st == UBT_OK) {
    cudaError_t e = cudaMemcpyAsync(h_counts, L.counts, sizeof(int64_t) * 2 * n_tau, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_last_cuda_error(e, "copy counts to host", __FILE__, __LINE__);
      st = UBT_ERR_CUDA;
    }
  }
  ubt_destroy_graph(g);
  return st;
}
