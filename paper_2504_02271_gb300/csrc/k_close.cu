// K3/K4/K5: hyper-triangle closure, classification and per-pattern reduction
// (step two of the two-step framework, Sec. 3.2-3.3).
//
// Every hyper-triangle {e_u, e_v, e_w} (Def. 2.4) is found exactly once, from
// its lowest-ranked hyperedge u in the degree order: v and w are both
// out-neighbours of u, and w is an out-neighbour of v.  The team that owns u
//   1. inserts out(u) into a hash table (key w -> slot),
//   2. records for every out-neighbour x the set Omega_ux = e_u cap e_x as a bit
//      mask over the positions of e_u (scanning E_y for each vertex y of e_u),
//   3. streams out(v) for every v in out(u) and probes each w in the table.
// A hit is a hyper-triangle.  With m_uv, m_uw the masks,
//   g = |e_u cap e_v cap e_w| = popc(m_uv & m_uw),  omega_uv = popc(m_uv),
//   omega_uw = popc(m_uw),  omega_vw from the entry of out(v),
// and the seven Venn regions of Sec. 2 follow by inclusion-exclusion:
//   a = |e_u| - omega_uv - omega_uw + g, b = |e_v| - omega_uv - omega_vw + g,
//   c = |e_w| - omega_uw - omega_vw + g, d = omega_uv - g, e = omega_vw - g,
//   f = omega_uw - g, and g itself.
// Their non-emptiness bits index a 128-entry table giving the pattern 1..20; a
// block-local histogram is flushed to 64-bit global counters.
#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBins = 24;      // pattern 0 (invalid) .. 20, padded
constexpr int kHistCopies = 4; // spread same-pattern increments of one warp
constexpr int kWideThreads = 256;

__constant__ uint8_t c_lut[128];

__device__ __forceinline__ uint32_t slot_of(uint32_t key, int cap_log2) {
  return (key * 0x9E3779B1u) >> (32 - cap_log2);
}

template <bool PACKED>
__device__ __forceinline__ void get_entry(const Oriented& o, int64_t at, int32_t& nbr, int32_t& om) {
  if (PACKED) {
    const uint32_t x = __ldg(o.packed + at);
    nbr = (int32_t)(x >> 8);
    om = (int32_t)(x & 0xffu);
  } else {
    nbr = __ldg(o.nbr + at);
    om = __ldg(o.omega + at);
  }
}

__device__ __forceinline__ int region_bits(int szu, int szv, int szw, int wuv, int wuw, int wvw,
                                           int g) {
  const int a = szu - wuv - wuw + g, b = szv - wuv - wvw + g, c = szw - wuw - wvw + g;
  return (a > 0) | ((b > 0) << 1) | ((c > 0) << 2) | ((wuv > g) << 3) | ((wvw > g) << 4) |
         ((wuw > g) << 5) | ((g > 0) << 6);
}

// ------------------------------------------------------------------ warp per u

template <int CAP_LOG2>
struct WarpTables {
  static constexpr int CAP = 1 << CAP_LOG2;
  static constexpr int DMAX = CAP / 4;   // load factor <= 1/4
  int32_t key[CAP];
  uint32_t mask[CAP];
  int32_t size[CAP];
  uint16_t kslot[DMAX];
  int32_t kcnt[DMAX];
  int64_t kbeg[DMAX];
};

template <int CAP_LOG2, int WARPS, bool PACKED>
__global__ void __launch_bounds__(WARPS * 32)
    k_close_warp(DevGraph g, Oriented o, const int32_t* __restrict__ list,
                 const int32_t* __restrict__ n_p, unsigned long long* __restrict__ hist_out,
                 unsigned long long* __restrict__ work, int32_t* __restrict__ counter) {
  using TT = WarpTables<CAP_LOG2>;
  constexpr int CAP = TT::CAP;
  __shared__ TT tabs[WARPS];
  __shared__ uint32_t hist[WARPS][kHistCopies][kBins];
  __shared__ uint8_t lut[128];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  TT& t = tabs[w];
  for (int k = threadIdx.x; k < 128; k += blockDim.x) lut[k] = c_lut[k];
  for (int k = lane; k < kHistCopies * kBins; k += 32) (&hist[w][0][0])[k] = 0;
  __syncthreads();
  const int32_t n = *n_p;
  uint32_t* my_hist = hist[w][lane & (kHistCopies - 1)];
  uint64_t since_flush = 0;
  unsigned long long probes = 0, gathers = 0;

  while (true) {
    int r = 0;
    if (lane == 0) r = atomicAdd(counter, 1);
    r = __shfl_sync(kFull, r, 0);
    if (r >= n) break;
    const int32_t u = list[r];
    const int32_t du = o.dplus[u];
    const int64_t bu = o.row_ptr[u];
    const int64_t eb = g.e_ptr[u];
    const int32_t szu = (int32_t)(g.e_ptr[u + 1] - eb);

    for (int s = lane; s < CAP; s += 32) t.key[s] = -1;
    __syncwarp();
    // 1. out(u) into the table
    for (int k = lane; k < du; k += 32) {
      int32_t x, om;
      get_entry<PACKED>(o, bu + k, x, om);
      uint32_t s = slot_of((uint32_t)x, CAP_LOG2);
      while (atomicCAS(&t.key[s], -1, x) != -1) s = (s + 1) & (CAP - 1);
      t.mask[s] = 0;
      t.size[s] = __ldg(g.esize + x);
      t.kslot[k] = (uint16_t)s;
      t.kbeg[k] = __ldg(o.row_ptr + x);
      t.kcnt[k] = __ldg(o.dplus + x);
    }
    __syncwarp();
    // 2. Omega_ux masks: for vertex y at position p of e_u, every x in E_y that is in out(u)
    for (int p = 0; p < szu; ++p) {
      const int32_t y = __ldg(g.e_idx + eb + p);
      const int64_t yb = __ldg(g.v_ptr + y), ye = __ldg(g.v_ptr + y + 1);
      gathers += (unsigned long long)(ye - yb);
      for (int64_t q = yb + lane; q < ye; q += 32) {
        const int32_t x = __ldg(g.v_idx + q);
        uint32_t s = slot_of((uint32_t)x, CAP_LOG2);
        int32_t kk;
        while ((kk = t.key[s]) != x && kk != -1) s = (s + 1) & (CAP - 1);
        if (kk == x) atomicOr(&t.mask[s], 1u << p);  // lanes may be at different p
      }
    }
    __syncwarp();
    // 3. close: for v in out(u), probe every w in out(v)
    for (int k = 0; k < du; ++k) {
      const int sv = t.kslot[k];
      const uint32_t muv = t.mask[sv];
      const int szv = t.size[sv];
      const int wuv = __popc(muv);
      const int64_t vb = t.kbeg[k];
      const int32_t cnt = t.kcnt[k];
      since_flush += (uint64_t)cnt;
      probes += (unsigned long long)cnt;
      for (int32_t j0 = 0; j0 < cnt; j0 += 4 * 32) {
        int32_t wv[4], om[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int32_t j = j0 + q * 32 + lane;
          wv[q] = -2;
          om[q] = 0;
          if (j < cnt) get_entry<PACKED>(o, vb + j, wv[q], om[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (wv[q] < 0) continue;
          uint32_t s = slot_of((uint32_t)wv[q], CAP_LOG2);
          int32_t kk;
          while ((kk = t.key[s]) != wv[q] && kk != -1) s = (s + 1) & (CAP - 1);
          if (kk != wv[q]) continue;
          const uint32_t muw = t.mask[s];
          const int szw = t.size[s];
          const int gg = __popc(muv & muw);
          const int bits = region_bits(szu, szv, szw, wuv, __popc(muw), om[q], gg);
          atomicAdd(&my_hist[lut[bits]], 1u);
        }
      }
    }
    if (since_flush > (1ull << 30)) {  // keep the 32-bit bins far from overflow
      __syncwarp();
      for (int k = lane; k < kHistCopies * kBins; k += 32) {
        const uint32_t x = (&hist[w][0][0])[k];
        if (x) atomicAdd(&hist_out[k % kBins], (unsigned long long)x);
        (&hist[w][0][0])[k] = 0;
      }
      since_flush = 0;
    }
    __syncwarp();
  }
  __syncwarp();
  for (int k = lane; k < kHistCopies * kBins; k += 32) {
    const uint32_t x = (&hist[w][0][0])[k];
    if (x) atomicAdd(&hist_out[k % kBins], (unsigned long long)x);
  }
  if (lane == 0) {  // warp-uniform totals
    atomicAdd(&work[0], probes);
    atomicAdd(&work[1], gathers);
  }
}

// ------------------------------------------------------------------ block per u (wide)
// Any |e_u| (masks of `words` 32-bit words) and any out-degree; tables in global scratch.

struct WideScratch {
  int32_t* key;     // [cap]
  int32_t* size;    // [cap]
  uint32_t* mask;   // [cap * words]
  int32_t* kslot;   // [dmax]
  int32_t* kcnt;    // [dmax]
  int64_t* kbeg;    // [dmax]
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline size_t wide_block_bytes(int64_t cap, int64_t words, int64_t dmax) {
  return align256(cap * 4) * 2 + align256(cap * words * 4) + align256(dmax * 4) * 2 +
         align256(dmax * 8);
}

__device__ WideScratch wide_carve(char* base, int64_t cap, int64_t words, int64_t dmax) {
  WideScratch w;
  w.key = (int32_t*)base;
  base += align256(cap * 4);
  w.size = (int32_t*)base;
  base += align256(cap * 4);
  w.mask = (uint32_t*)base;
  base += align256(cap * words * 4);
  w.kslot = (int32_t*)base;
  base += align256(dmax * 4);
  w.kcnt = (int32_t*)base;
  base += align256(dmax * 4);
  w.kbeg = (int64_t*)base;
  return w;
}

template <bool PACKED>
__global__ void __launch_bounds__(kWideThreads)
    k_close_wide(DevGraph g, Oriented o, const int32_t* __restrict__ list,
                 const int32_t* __restrict__ n_p, int64_t cap_max, int64_t words_max,
                 int64_t dmax, char* __restrict__ scratch, unsigned long long* __restrict__ hist_out,
                 unsigned long long* __restrict__ work, int32_t* __restrict__ counter) {
  __shared__ uint32_t hist[kHistCopies][kBins];
  __shared__ uint8_t lut[128];
  __shared__ int32_t s_r;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kW = kWideThreads / 32;
  WideScratch t = wide_carve(scratch + wide_block_bytes(cap_max, words_max, dmax) * blockIdx.x,
                             cap_max, words_max, dmax);
  for (int k = threadIdx.x; k < 128; k += blockDim.x) lut[k] = c_lut[k];
  for (int k = threadIdx.x; k < kHistCopies * kBins; k += blockDim.x) (&hist[0][0])[k] = 0;
  const int32_t n = *n_p;
  uint32_t* my_hist = hist[lane & (kHistCopies - 1)];
  uint64_t since_flush = 0;
  unsigned long long probes = 0, gathers = 0;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_r = atomicAdd(counter, 1);
    __syncthreads();
    const int32_t r = s_r;
    if (r >= n) break;
    const int32_t u = list[r];
    const int32_t du = o.dplus[u];
    const int64_t bu = o.row_ptr[u];
    const int64_t eb = g.e_ptr[u];
    const int32_t szu = (int32_t)(g.e_ptr[u + 1] - eb);
    const int32_t words = (szu + 31) / 32;
    int cl = 4;
    while ((int64_t(1) << cl) < 4 * (int64_t)du) ++cl;
    const uint32_t cap = 1u << cl;
    for (uint32_t s = threadIdx.x; s < cap; s += kWideThreads) t.key[s] = -1;
    for (uint32_t s = threadIdx.x; s < cap * (uint32_t)words; s += kWideThreads) t.mask[s] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < du; k += kWideThreads) {
      int32_t x, om;
      get_entry<PACKED>(o, bu + k, x, om);
      uint32_t s = slot_of((uint32_t)x, cl);
      while (atomicCAS(&t.key[s], -1, x) != -1) s = (s + 1) & (cap - 1);
      t.size[s] = __ldg(g.esize + x);
      t.kslot[k] = (int32_t)s;
      t.kbeg[k] = __ldg(o.row_ptr + x);
      t.kcnt[k] = __ldg(o.dplus + x);
    }
    __syncthreads();
    for (int p = w; p < szu; p += kW) {
      const int32_t y = __ldg(g.e_idx + eb + p);
      const int64_t yb = __ldg(g.v_ptr + y), ye = __ldg(g.v_ptr + y + 1);
      if (lane == 0) gathers += (unsigned long long)(ye - yb);
      for (int64_t q = yb + lane; q < ye; q += 32) {
        const int32_t x = __ldg(g.v_idx + q);
        uint32_t s = slot_of((uint32_t)x, cl);
        int32_t kk;
        while ((kk = *((volatile int32_t*)&t.key[s])) != x && kk != -1) s = (s + 1) & (cap - 1);
        if (kk == x) atomicOr(&t.mask[(size_t)s * words + (p >> 5)], 1u << (p & 31));
      }
    }
    __syncthreads();
    for (int k = w; k < du; k += kW) {
      const int sv = t.kslot[k];
      const uint32_t* muv = t.mask + (size_t)sv * words;
      const int szv = t.size[sv];
      int wuv = 0;
      for (int q = 0; q < words; ++q) wuv += __popc(muv[q]);
      const int64_t vb = t.kbeg[k];
      const int32_t cnt = t.kcnt[k];
      since_flush += (uint64_t)cnt;
      if (lane == 0) probes += (unsigned long long)cnt;
      for (int32_t j = lane; j < cnt; j += 32) {
        int32_t wv, om;
        get_entry<PACKED>(o, vb + j, wv, om);
        uint32_t s = slot_of((uint32_t)wv, cl);
        int32_t kk;
        while ((kk = t.key[s]) != wv && kk != -1) s = (s + 1) & (cap - 1);
        if (kk != wv) continue;
        const uint32_t* muw = t.mask + (size_t)s * words;
        int wuw = 0, gg = 0;
        for (int q = 0; q < words; ++q) {
          wuw += __popc(muw[q]);
          gg += __popc(muw[q] & muv[q]);
        }
        const int bits = region_bits(szu, szv, t.size[s], wuv, wuw, om, gg);
        atomicAdd(&my_hist[lut[bits]], 1u);
      }
    }
    if (since_flush > (1ull << 28)) {
      __syncthreads();
      if (threadIdx.x < kHistCopies * kBins) {
        const uint32_t x = (&hist[0][0])[threadIdx.x];
        if (x) atomicAdd(&hist_out[threadIdx.x % kBins], (unsigned long long)x);
        (&hist[0][0])[threadIdx.x] = 0;
      }
      since_flush = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x < kHistCopies * kBins) {
    const uint32_t x = (&hist[0][0])[threadIdx.x];
    if (x) atomicAdd(&hist_out[threadIdx.x % kBins], (unsigned long long)x);
  }
  if (lane == 0) {
    atomicAdd(&work[0], probes);
    atomicAdd(&work[1], gathers);
  }
}

// ------------------------------------------------------------------ bucketing

constexpr int kWarpMaskBits = 32;

__global__ void k_bucket_close(DevGraph g, Oriented o, CloseBuckets b,
                               unsigned long long* __restrict__ wide_max) {
  const int lane = threadIdx.x & 31;
  unsigned long long my_d = 0, my_s = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.ne;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = base + threadIdx.x;
    int bucket = -1;
    if (u < g.ne) {
      const int32_t d = o.dplus[u];
      const int32_t sz = g.esize[u];
      if (d >= 2) {
        if (sz <= kWarpMaskBits && d <= 64) bucket = 0;
        else if (sz <= kWarpMaskBits && d <= 128) bucket = 1;
        else if (sz <= kWarpMaskBits && d <= 256) bucket = 2;
        else {
          bucket = 3;
          my_d = (unsigned long long)d > my_d ? (unsigned long long)d : my_d;
          my_s = (unsigned long long)sz > my_s ? (unsigned long long)sz : my_s;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned bal = __ballot_sync(kFull, bucket == k);
      if (!bal) continue;
      int32_t at = 0;
      const int leader = __ffs(bal) - 1;
      if (lane == leader) at = atomicAdd(&b.count[k], __popc(bal));
      at = __shfl_sync(kFull, at, leader);
      if (bucket == k) b.lists[k][at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)u;
    }
  }
  atomicMax(&wide_max[0], my_d);
  atomicMax(&wide_max[1], my_s);
}

template <int CAP_LOG2, int WARPS>
void launch_warp(const DevGraph& g, const Oriented& o, int packed, const int32_t* list, int32_t n,
                 const int32_t* n_p, unsigned long long* hist, unsigned long long* work,
                 int32_t* counter, cudaStream_t s, int nsm) {
  int per_sm = 0;
  if (packed) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_close_warp<CAP_LOG2, WARPS, true>,
                                                  WARPS * 32, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_close_warp<CAP_LOG2, WARPS, false>,
                                                  WARPS * 32, 0);
  }
  if (per_sm < 1) per_sm = 1;
  int blocks = (n + WARPS - 1) / WARPS;
  if (blocks > per_sm * nsm) blocks = per_sm * nsm;
  note_launch();
  if (packed)
    k_close_warp<CAP_LOG2, WARPS, true>
        <<<blocks, WARPS * 32, 0, s>>>(g, o, list, n_p, hist, work, counter);
  else
    k_close_warp<CAP_LOG2, WARPS, false>
        <<<blocks, WARPS * 32, 0, s>>>(g, o, list, n_p, hist, work, counter);
}

}  // namespace

void close_set_lut(const uint8_t lut[128], cudaStream_t s) {
  cudaMemcpyToSymbolAsync(c_lut, lut, 128, 0, cudaMemcpyHostToDevice, s);
}

void launch_bucket_close(const DevGraph& g, const Oriented& o, CloseBuckets b,
                         unsigned long long* wide_max, cudaStream_t s) {
  if (g.ne == 0) return;
  int64_t blocks = (g.ne + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  note_launch();
  k_bucket_close<<<(unsigned)blocks, 256, 0, s>>>(g, o, b, wide_max);
}

size_t close_wide_scratch_bytes(int64_t cap, int64_t words, int64_t dmax, int nsm) {
  if (cap <= 0) return 0;
  return wide_block_bytes(cap, words, dmax) * (size_t)(nsm * 2);
}

void launch_close(int bucket, const DevGraph& g, const Oriented& o, int packed,
                  const int32_t* list, int32_t n, const int32_t* n_p, int64_t wide_cap,
                  int64_t wide_words, int64_t wide_dmax, void* scratch, unsigned long long* hist,
                  unsigned long long* work, int32_t* counter, cudaStream_t s, int nsm) {
  if (n <= 0) return;
  switch (bucket) {
    case 0: launch_warp<8, 8>(g, o, packed, list, n, n_p, hist, work, counter, s, nsm); break;
    case 1: launch_warp<9, 4>(g, o, packed, list, n, n_p, hist, work, counter, s, nsm); break;
    case 2: launch_warp<10, 2>(g, o, packed, list, n, n_p, hist, work, counter, s, nsm); break;
    default: {
      int blocks = n < nsm * 2 ? n : nsm * 2;
      note_launch();
      if (packed)
        k_close_wide<true><<<blocks, kWideThreads, 0, s>>>(g, o, list, n_p, wide_cap, wide_words,
                                                           wide_dmax, (char*)scratch, hist, work,
                                                           counter);
      else
        k_close_wide<false><<<blocks, kWideThreads, 0, s>>>(g, o, list, n_p, wide_cap, wide_words,
                                                            wide_dmax, (char*)scratch, hist, work,
                                                            counter);
    }
  }
}

}  // namespace hg
