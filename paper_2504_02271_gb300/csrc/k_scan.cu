// Exclusive prefix sums and small reductions used to lay out the CSR arrays.
#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// Exclusive scan over the block's threads; returns this thread's prefix, *total = block sum.
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = warp_incl_scan(v);
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t x = lane < kScanThreads / 32 ? wsum[lane] : 0;
    x = warp_incl_scan(x);
    if (lane < kScanThreads / 32) wsum[lane] = x;
  }
  __syncthreads();
  int64_t before = (w > 0 ? wsum[w - 1] : 0) + incl - v;
  *total = wsum[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const T* __restrict__ in, int64_t n,
                                                            int64_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kTile;
  int64_t s = 0;
  for (int k = threadIdx.x; k < kTile; k += kScanThreads) {
    int64_t idx = base + k;
    if (idx < n) s += (int64_t)in[idx];
  }
  int64_t total;
  (void)block_excl_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[idx] = offs[block] + exclusive prefix inside the tile; the last tile writes out[n].
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T* __restrict__ in, int64_t n,
                                                            const int64_t* __restrict__ offs,
                                                            int64_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + k;
    v[k] = idx < n ? (int64_t)in[idx] : 0;
    s += v[k];
  }
  int64_t total;
  int64_t run = block_excl_scan(s, &total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + k;
    if (idx < n) out[idx] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
}

size_t level_bytes(int64_t n) {
  int64_t nb = (n + kTile - 1) / kTile;
  return (size_t)(2 * nb + 1) * sizeof(int64_t) + 256;
}

template <typename T>
void scan_impl(const T* in, int64_t* out, int64_t n, char* tmp, cudaStream_t s) {
  if (n <= kTile) {
    note_launch();
    k_tile_scan<T><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
    return;
  }
  const int64_t nb = (n + kTile - 1) / kTile;
  int64_t* sums = reinterpret_cast<int64_t*>(tmp);
  int64_t* sums_scan = sums + nb;
  char* next = tmp + (((size_t)(2 * nb + 1) * sizeof(int64_t) + 255) / 256) * 256;
  note_launch(2);
  k_tile_sums<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  scan_impl<int64_t>(sums, sums_scan, nb, next, s);
  k_tile_scan<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums_scan, out);
}

__global__ void k_deg_stats(const int32_t* __restrict__ a, int64_t n,
                            unsigned long long* __restrict__ acc) {
  unsigned long long c2 = 0, mx = 0, sum = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long x = (unsigned long long)a[i];
    c2 += x * (x - (x ? 1ull : 0ull)) / 2ull;
    sum += x;
    mx = x > mx ? x : mx;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    c2 += __shfl_down_sync(0xffffffffu, c2, d);
    sum += __shfl_down_sync(0xffffffffu, sum, d);
    unsigned long long o = __shfl_down_sync(0xffffffffu, mx, d);
    mx = o > mx ? o : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], c2);
    atomicMax(&acc[1], mx);
    atomicAdd(&acc[2], sum);
  }
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) {
  size_t b = 0;
  while (n > kTile) {
    b += level_bytes(n);
    n = (n + kTile - 1) / kTile;
  }
  return b + 256;
}

void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s) {
  scan_impl<int32_t>(in, out, n, static_cast<char*>(tmp), s);
}

void scan_i64_to_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s) {
  scan_impl<int64_t>(in, out, n, static_cast<char*>(tmp), s);
}

void reduce_deg_stats(const int32_t* a, int64_t n, unsigned long long* acc, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  note_launch();
  k_deg_stats<<<(unsigned)blocks, 256, 0, s>>>(a, n, acc);
}

}  // namespace hg
