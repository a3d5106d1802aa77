// ubt_scan.cu -- exclusive prefix sum of uint32 counts (CSR offsets, list
// offsets).  Three passes over tiles of 4096 values: tile totals, a scan of
// the totals by one block, then a rescan of every tile with its offset.
#include "ubt_internal.cuh"

namespace ubt {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* excl) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  __shared__ uint32_t total_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = wsum[lane];
    uint32_t ti = t;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, ti, d);
      if (lane >= d) ti += y;
    }
    wsum[lane] = ti - t;
    if (lane == 31) total_s = ti;
  }
  __syncthreads();
  *excl = wsum[wid] + inc - x;
  const uint32_t total = total_s;
  __syncthreads();
  return total;
}

__global__ void k_tile_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ tile_sum) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++)
    if (base + i < n) s += in[base + i];
  uint32_t ex;
  uint32_t tot = block_exclusive_scan(s, &ex);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// One block: exclusive scan of the tile totals in place, total at [ntiles].
__global__ void k_scan_tiles(uint32_t* tile_sum, int64_t ntiles) {
  uint32_t carry = 0;
  for (int64_t start = 0; start < ntiles; start += kTile) {
    const int64_t base = start + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
      v[i] = (base + i < ntiles) ? tile_sum[base + i] : 0;
      s += v[i];
    }
    uint32_t ex;
    uint32_t tot = block_exclusive_scan(s, &ex);
    uint32_t run = carry + ex;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
      if (base + i < ntiles) tile_sum[base + i] = run;
      run += v[i];
    }
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_sum[ntiles] = carry;
}

__global__ void k_tile_apply(const uint32_t* in, int64_t n, const uint32_t* __restrict__ tile_off,
                             uint32_t* out) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  uint32_t ex;
  block_exclusive_scan(s, &ex);
  uint32_t run = tile_off[blockIdx.x] + ex;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

__global__ void k_write_total(const uint32_t* tile_off, int64_t ntiles, uint32_t* out, int64_t n) {
  out[n] = tile_off[ntiles];
}

}  // namespace

size_t scan_tmp_words(int64_t n) { return (size_t)((n + kTile - 1) / kTile) + 2; }

// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.  `in` and
// `out` may alias.  tmp holds scan_tmp_words(n) words.
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s) {
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (ntiles > 0) {
    k_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_tiles<<<1, kScanThreads, 0, s>>>(tmp, ntiles);
    k_tile_apply<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp, out);
  } else {
    cudaMemsetAsync(tmp, 0, sizeof(uint32_t), s);
  }
  k_write_total<<<1, 1, 0, s>>>(tmp, ntiles, out, n);
  return cudaGetLastError();
}

}  // namespace ubt
