// scan.cu -- device prefix sums and the output sort of the bridge list.
//
// The bridges are emitted as unique packed keys (a << k) | b with a < b and k the bit width of
// V-1; sorting the keys sorts the pairs lexicographically.  Small lists (<= kRankMax keys) are
// sorted by rank: a key's position is the number of smaller keys, computed by all-pairs
// comparison in one launch (exact because keys are unique).  Larger lists use a stable LSD radix
// sort with 8-bit digits: per pass a tile histogram, an exclusive scan of the digit-major
// histogram, and a stable scatter ranked with warp match/ballot.
#include <algorithm>

#include "common.cuh"

namespace bridges {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048
constexpr int64_t kRankMax = 16384;
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 2048

// Block-wide exclusive scan of one 2048-element tile; returns the tile total to every thread.
__device__ int32_t block_scan_tile(int32_t* sm /* kScanTile */, int32_t* warp_tot /* 8 */) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = sm[tid * kScanItems + k];
    s += v[k];
  }
  int32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int32_t wbase = 0, total = 0;
  for (int w = 0; w < kScanThreads / 32; w++) {
    int32_t t = warp_tot[w];
    if (w < warp) wbase += t;
    total += t;
  }
  int32_t run = wbase + incl - s;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    sm[tid * kScanItems + k] = run;
    run += v[k];
  }
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kScanThreads) tile_sum_kernel(const int32_t* in, int64_t n, int32_t* sums) {
  __shared__ int32_t red[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t s = 0;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int64_t i = base + k;
    if (i < n) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; w++) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// Scans each tile and adds its offset (offsets == null: a single tile).
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const int32_t* in, int32_t* out, int64_t n,
                                                                const int32_t* offsets, int32_t* total_out) {
  __shared__ int32_t sm[kScanTile];
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int64_t i = base + k;
    sm[k] = i < n ? in[i] : 0;
  }
  __syncthreads();
  int32_t total = block_scan_tile(sm, warp_tot);
  const int32_t off = offsets ? offsets[blockIdx.x] : 0;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int64_t i = base + k;
    if (i < n) out[i] = sm[k] + off;
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = off + total;
}

// ---- sort ----
__global__ void rank_sort_kernel(const uint64_t* keys, const int32_t* d_n, int32_t cap, int kbits, int32_t* out) {
  __shared__ uint64_t tile[2048];
  const int32_t n = min(*d_n, cap);
  if (n > kRankMax) return;  // the caller never asks; guards the quadratic loop
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((int64_t)blockIdx.x * blockDim.x >= n) return;  // whole block idle
  const uint64_t mine = i < n ? keys[i] : ~0ULL;
  int32_t rank = 0;
  for (int32_t t0 = 0; t0 < n; t0 += 2048) {
    __syncthreads();
    for (int k = threadIdx.x; k < 2048; k += blockDim.x) tile[k] = (t0 + k < n) ? keys[t0 + k] : ~0ULL;
    __syncthreads();
    const int lim = min(2048, n - t0);
    for (int k = 0; k < lim; k++) rank += tile[k] < mine;
  }
  if (i < n) {
    const uint64_t mask = (1ULL << kbits) - 1;
    out[2 * (int64_t)rank] = (int32_t)(mine >> kbits);
    out[2 * (int64_t)rank + 1] = (int32_t)(mine & mask);
  }
}

__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(const uint64_t* keys, const int32_t* d_n, int32_t cap,
                                                                  int shift, uint32_t* hist, int nblocks) {
  __shared__ uint32_t h[256];
  const int32_t n = min(*d_n, cap);
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int k = threadIdx.x; k < kRadixTile; k += kRadixThreads) {
    int64_t i = base + k;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: keys of the tile are taken in index order (sub-round, warp, lane).
__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(const uint64_t* keys, uint64_t* keys_out,
                                                                     const int32_t* d_n, int32_t cap, int shift,
                                                                     const uint32_t* offs, int nblocks, int kbits,
                                                                     int32_t* pairs_out) {
  __shared__ uint32_t wcnt[kRadixThreads / 32][256];
  __shared__ uint32_t run[256];
  const int32_t n = min(*d_n, cap);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int w = 0; w < kRadixThreads / 32; w++) wcnt[w][tid] = 0;
  run[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixItems; r++) {
    const int64_t i = base + (int64_t)r * kRadixThreads + tid;
    const bool valid = i < n;
    const uint64_t key = valid ? keys[i] : 0;
    const unsigned d = valid ? (unsigned)((key >> shift) & 255) : 256u + lane;
    const unsigned peers = __match_any_sync(kFull, d);
    const unsigned rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = run[tid];
      for (int w = 0; w < kRadixThreads / 32; w++) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      run[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wcnt[warp][d] + rank;
      if (pairs_out) {
        const uint64_t mask = (1ULL << kbits) - 1;
        pairs_out[2 * (int64_t)pos] = (int32_t)(key >> kbits);
        pairs_out[2 * (int64_t)pos + 1] = (int32_t)(key & mask);
      } else {
        keys_out[pos] = key;
      }
    }
    __syncthreads();
    for (int w = 0; w < kRadixThreads / 32; w++) wcnt[w][tid] = 0;
    __syncthreads();
  }
}

}  // namespace

size_t scan_tmp_elems(int64_t n) {
  int64_t nb = ceil_div(std::max<int64_t>(n, 1), kScanTile);
  if (nb <= 1) return 8;
  return (size_t)align_up((size_t)nb, 64) + scan_tmp_elems(nb);
}

void exclusive_scan_i32(const Launch& L, const int32_t* in, int32_t* out, int64_t n, bool write_total, int32_t* tmp) {
  if (n <= 0) {
    if (write_total) cudaMemsetAsync(out, 0, sizeof(int32_t), L.stream);
    return;
  }
  const int64_t nb = ceil_div(n, kScanTile);
  int32_t* total = write_total ? out + n : nullptr;
  if (nb == 1) {
    tile_scan_kernel<<<1, kScanThreads, 0, L.stream>>>(in, out, n, nullptr, total);
    *L.launches += 1;
    return;
  }
  int32_t* sums = tmp;
  int32_t* rest = tmp + align_up((size_t)nb, 64);
  tile_sum_kernel<<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, n, sums);
  exclusive_scan_i32(L, sums, sums, nb, false, rest);
  tile_scan_kernel<<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, out, n, sums, total);
  *L.launches += 2;
}

size_t sort_hist_elems(int64_t cap) {
  int64_t nb = ceil_div(std::max<int64_t>(cap, 1), kRadixTile);
  return (size_t)nb * 256;
}

void sort_pairs(const Launch& L, uint64_t* keys, uint64_t* keys2, const int32_t* d_n, int64_t cap, int key_bits,
                int32_t* out, uint32_t* hist, size_t hist_elems, int32_t* scan_tmp) {
  const int kbits = key_bits / 2;
  const int32_t ncap = (int32_t)std::min<int64_t>(cap, INT32_MAX);  // keys beyond cap are never read
  if (cap <= kRankMax) {
    const int bs = 256;
    rank_sort_kernel<<<(unsigned)ceil_div(std::max<int64_t>(cap, 1), bs), bs, 0, L.stream>>>(keys, d_n, ncap, kbits,
                                                                                              out);
    *L.launches += 1;
    return;
  }
  const int nblocks = (int)ceil_div(cap, kRadixTile);
  const int passes = std::max(1, (key_bits + 7) / 8);
  uint64_t* src = keys;
  uint64_t* dst = keys2;
  for (int p = 0; p < passes; p++) {
    const int shift = 8 * p;
    radix_hist_kernel<<<nblocks, kRadixThreads, 0, L.stream>>>(src, d_n, ncap, shift, hist, nblocks);
    exclusive_scan_i32(L, reinterpret_cast<int32_t*>(hist), reinterpret_cast<int32_t*>(hist), (int64_t)256 * nblocks,
                       false, scan_tmp);
    const bool last = p == passes - 1;
    radix_scatter_kernel<<<nblocks, kRadixThreads, 0, L.stream>>>(src, dst, d_n, ncap, shift, hist, nblocks, kbits,
                                                                    last ? out : nullptr);
    *L.launches += 2;
    std::swap(src, dst);
  }
}

}  // namespace bridges
