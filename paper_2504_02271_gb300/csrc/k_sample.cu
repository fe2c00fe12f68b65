// Hyperwedge-sampling estimate (Sec. 4.1, Algorithm 6, Appro-bs) on the GPU.
//
// The hyperwedges are numbered in the order O of Sec. 2: by i, then by j, i < j.
// The "upper" lists hold, for each hyperedge i, its neighbours j > i with
// omega_ij, sorted by j (built once per handle: emitted by the hyperwedge pass,
// then each row sorted here).  Sample n takes the Philox4x32-10 block of counter
// (n lo, n hi, 0, 0) under key (seed lo, seed hi) (Salmon et al., SC'11), forms
// r = x1 << 32 | x0 and draws hyperwedge m = floor(r * W / 2^64).  For the drawn
// (i, j) every k > j in both upper(i) and upper(j) closes the hyper-triangle
// {i, j, k} whose smallest hyperwedge in O is (i, j); it is classified from its
// seven Venn regions (g by a 3-way merge of the vertex lists) and counted.
#include <mutex>

#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 512;
constexpr int kSampleWarps = 8;

__constant__ uint8_t c_sample_lut[128];

// one Philox4x32-10 block: 10 rounds of two 32x32 -> 64 products, Weyl key bumps
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Sort each upper row in shared memory (bitonic network on 64-bit keys
// j << 32 | omega, padded to a power of two).  Rows longer than max_len set err.
__global__ void __launch_bounds__(kSortThreads)
    k_sort_upper(const int64_t* __restrict__ up_ptr, int32_t ne, Oriented up, int packed,
                 int max_len_log2, int* __restrict__ err) {
  extern __shared__ unsigned long long keys[];
  for (int32_t i = blockIdx.x; i < ne; i += gridDim.x) {
    const int64_t b = up_ptr[i];
    const int32_t len = (int32_t)(up_ptr[i + 1] - b);
    if (len <= 1) continue;
    if (len > (1 << max_len_log2)) {
      if (threadIdx.x == 0) dev_fail(err, DE_LIMIT);
      continue;
    }
    int n = 1;
    while (n < len) n <<= 1;
    for (int t = threadIdx.x; t < n; t += kSortThreads) {
      unsigned long long key = ~0ull;
      if (t < len) {
        if (packed) {
          const uint32_t x = up.packed[b + t];
          key = ((unsigned long long)(x >> 8) << 32) | (x & 0xffu);
        } else {
          key = ((unsigned long long)(uint32_t)up.nbr[b + t] << 32) | (uint32_t)up.omega[b + t];
        }
      }
      keys[t] = key;
    }
    __syncthreads();
    for (int k = 2; k <= n; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < n; t += kSortThreads) {
          const int p = t ^ j;
          if (p > t) {
            const unsigned long long a = keys[t], c = keys[p];
            const bool up_dir = (t & k) == 0;
            if ((a > c) == up_dir) {
              keys[t] = c;
              keys[p] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int t = threadIdx.x; t < len; t += kSortThreads) {
      const unsigned long long key = keys[t];
      if (packed) {
        up.packed[b + t] = ((uint32_t)(key >> 32) << 8) | (uint32_t)(key & 0xffu);
      } else {
        up.nbr[b + t] = (int32_t)(key >> 32);
        up.omega[b + t] = (int32_t)(key & 0xffffffffu);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void up_entry(const Oriented& up, int packed, int64_t at, int32_t& j,
                                         int32_t& om) {
  if (packed) {
    const uint32_t x = __ldg(up.packed + at);
    j = (int32_t)(x >> 8);
    om = (int32_t)(x & 0xffu);
  } else {
    j = __ldg(up.nbr + at);
    om = __ldg(up.omega + at);
  }
}

// |a cap b cap c| of three ascending vertex lists
__device__ int triple_common(const int32_t* a, int na, const int32_t* b, int nb, const int32_t* c,
                            int nc) {
  int i = 0, j = 0, k = 0, n = 0;
  while (i < na && j < nb && k < nc) {
    const int32_t x = __ldg(a + i), y = __ldg(b + j), z = __ldg(c + k);
    if (x == y && y == z) {
      ++n;
      ++i;
      ++j;
      ++k;
    } else {
      const int32_t m = max(x, max(y, z));
      if (x < m) ++i;
      if (y < m) ++j;
      if (z < m) ++k;
    }
  }
  return n;
}

// One warp per sample (grid-stride).  raw[0..23] += per-pattern counts.
__global__ void __launch_bounds__(kSampleWarps * 32)
    k_sample(DevGraph g, const int64_t* __restrict__ up_ptr, Oriented up, int packed, uint64_t W,
             uint64_t seed, uint64_t first, uint64_t num, unsigned long long* __restrict__ raw) {
  __shared__ uint32_t hist[kSampleWarps][24];
  __shared__ uint8_t lut[128];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < 128; k += blockDim.x) lut[k] = c_sample_lut[k];
  for (int k = lane; k < 24; k += 32) hist[w][k] = 0;
  __syncthreads();
  const uint64_t warps = (uint64_t)gridDim.x * kSampleWarps;
  for (uint64_t s = (uint64_t)blockIdx.x * kSampleWarps + w; s < num; s += warps) {
    const uint64_t n = first + s;
    uint32_t c[4] = {(uint32_t)n, (uint32_t)(n >> 32), 0u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t r = ((uint64_t)c[1] << 32) | c[0];
    const uint64_t m = __umul64hi(r, W);
    // row i: last i with up_ptr[i] <= m
    int32_t lo = 0, hi = g.ne - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (__ldg(up_ptr + mid) <= (int64_t)m) lo = mid; else hi = mid - 1;
    }
    const int32_t i = lo;
    const int64_t ib = (int64_t)m, ie = __ldg(up_ptr + i + 1);
    int32_t j, wij;
    up_entry(up, packed, ib, j, wij);
    const int64_t jb = __ldg(up_ptr + j), je = __ldg(up_ptr + j + 1);
    const int64_t ei = g.e_ptr[i], ej = g.e_ptr[j];
    const int szi = (int)(g.e_ptr[i + 1] - ei), szj = (int)(g.e_ptr[j + 1] - ej);
    // k > j in upper(i) (entries after m) and in upper(j): binary search each in upper(j)
    for (int64_t a = ib + 1 + lane; a < ie; a += 32) {
      int32_t k, wik;
      up_entry(up, packed, a, k, wik);
      int64_t l = jb, h = je;
      while (l < h) {
        const int64_t mid = (l + h) >> 1;
        int32_t x, om;
        up_entry(up, packed, mid, x, om);
        if (x < k) l = mid + 1; else h = mid;
      }
      if (l >= je) continue;
      int32_t x, wjk;
      up_entry(up, packed, l, x, wjk);
      if (x != k) continue;
      const int64_t ek = g.e_ptr[k];
      const int szk = (int)(g.e_ptr[k + 1] - ek);
      const int gg = triple_common(g.e_idx + ei, szi, g.e_idx + ej, szj, g.e_idx + ek, szk);
      const int ra = szi - wij - wik + gg, rb = szj - wij - wjk + gg, rc = szk - wik - wjk + gg;
      const int bits = (ra > 0) | ((rb > 0) << 1) | ((rc > 0) << 2) | ((wij > gg) << 3) |
                       ((wjk > gg) << 4) | ((wik > gg) << 5) | ((gg > 0) << 6);
      atomicAdd(&hist[w][lut[bits]], 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 24; k += blockDim.x) {
    unsigned long long x = 0;
    for (int ww = 0; ww < kSampleWarps; ++ww) x += hist[ww][k];
    if (x) atomicAdd(&raw[k], x);
  }
}

}  // namespace

constexpr int kSortMaxLog2 = 14;   // rows of up to 16,384 neighbours sort in shared memory

int sample_sort_max_log2() { return kSortMaxLog2; }

// Written once per device, synchronously (see close_set_lut).
void sample_set_lut(const uint8_t lut[128], cudaStream_t s) {
  (void)s;
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done >> dev & 1) return;
  if (cudaMemcpyToSymbol(c_sample_lut, lut, 128, 0, cudaMemcpyHostToDevice) == cudaSuccess)
    done |= uint64_t(1) << dev;
}

cudaError_t launch_sort_upper(const int64_t* up_ptr, int32_t ne, const Oriented& up, int packed,
                              int* err, cudaStream_t s, int nsm) {
  if (ne == 0) return cudaSuccess;
  const int smem = (int)(sizeof(unsigned long long) << kSortMaxLog2);
  cudaError_t e = cudaFuncSetAttribute(k_sort_upper, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  note_launch();
  k_sort_upper<<<nsm, kSortThreads, smem, s>>>(up_ptr, ne, up, packed, kSortMaxLog2, err);
  return cudaGetLastError();
}

void launch_sample(const DevGraph& g, const int64_t* up_ptr, const Oriented& up, int packed,
                   uint64_t W, uint64_t seed, uint64_t first, uint64_t num,
                   unsigned long long* raw, cudaStream_t s, int nsm) {
  if (num == 0 || W == 0) return;
  uint64_t blocks = (num + kSampleWarps - 1) / kSampleWarps;
  if (blocks > (uint64_t)nsm * 16) blocks = (uint64_t)nsm * 16;
  note_launch();
  k_sample<<<(unsigned)blocks, kSampleWarps * 32, 0, s>>>(g, up_ptr, up, packed, W, seed, first,
                                                          num, raw);
}

}  // namespace hg
