// K1/K2: hyperwedge construction and degree-ordered orientation (step one,
// Sec. 3.1, Algorithm 2).
//
// For each hyperedge e_i the kernels gather, for every vertex v of e_i, the
// hyperedges j != i of E_v, and accumulate omega_ij = |e_i cap e_j| (the number
// of shared vertices, Def. 2.2) in a hash table keyed by j.  That is row i of
// the sparse product H * H^T without its diagonal.  One gather pass per row
// yields deg(i) (the number of distinct j), the inclusion-type counts (omega_ij =
// min(|e_i|, |e_j|), Def. 2.3), the duplicate-hyperedge check (omega_ij = |e_i| =
// |e_j|), and writes every (j, omega_ij) of the row into a capacity layout (room
// for min(gathered incidences, |E| - 1) entries per row).  Once every deg(j) is
// known, a streaming row filter keeps the j ranked above i in the order (deg, id)
// (the oriented line graph, exact layout), or the j > i (the sampler's rows), or
// copies the row.  Algorithm 2 merges the sorted E_v lists one id at a time on a
// CPU; here the accumulation is a hash table in shared memory (one warp per light
// row, one block per medium row) or in global scratch (one block per heavy row).
// In the packed layout (|E| < 2^24, every |e| < 256, so omega < 256) a slot is one
// 32-bit word (j << 8) | count; otherwise a 64-bit word (j << 32) | count.  A slot
// is claimed with one compare-and-swap that also seeds the count, so a new key costs
// one shared atomic and a repeated key two.
#include <type_traits>

#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Hash-table slot of the gather pass: 32-bit (j << 8) | count in the packed layout,
// 64-bit (j << 32) | count otherwise; all ones = empty.
template <bool PACKED>
struct GatherSlot {
  using T = typename std::conditional<PACKED, uint32_t, unsigned long long>::type;
  static constexpr int kShift = PACKED ? 8 : 32;
  static constexpr T kEmpty = ~(T)0;
  __device__ static uint32_t key(T x) { return (uint32_t)(x >> kShift); }
  __device__ static uint32_t count(T x) {
    return PACKED ? (uint32_t)(x & 0xffu) : (uint32_t)(x & 0xffffffffu);
  }
};

// One-warp rows: a shared table of up to 2^light_cap_log2 slots (32 KB per 8-warp
// block in both layouts), for rows gathering at most half of that: 1,024 slots in the
// packed layout (rows of up to 512 incidences), 512 64-bit slots otherwise.  On the
// co-authorship workload 1,024 slots and 8 resident blocks per SM took the gather pass
// from 1.44 to 1.24 ms (512 slots: 1.44 ms; 1,024 slots alone 1.33 ms; 8 blocks alone
// 1.29 ms).
#ifndef HG_LIGHT_CAP_LOG2
#define HG_LIGHT_CAP_LOG2 10
#endif
template <bool PACKED>
__host__ __device__ constexpr int light_cap_log2() { return PACKED ? HG_LIGHT_CAP_LOG2 : 9; }
constexpr int kLightWarps = 8;
constexpr int kMediumCapLog2 = 13;   // 8192 slots (32 KiB packed, 64 KiB wide), rows with cand <= 4096
constexpr int kBlockThreads = 256;

__device__ __forceinline__ uint32_t slot_of(uint32_t key, int cap_log2) {
  return (key * 0x9E3779B1u) >> (32 - cap_log2);
}

// omega accumulation: add n to the count of key j (linear probing).  The claiming
// compare-and-swap writes the key with its first count; a slot that already holds j
// takes an atomic add.  Counts never exceed the smaller hyperedge, which fits the
// count field (8 bits packed, 32 bits otherwise).
template <bool PACKED>
__device__ __forceinline__ void ht_add(typename GatherSlot<PACKED>::T* T, int cap_log2, uint32_t j,
                                       uint32_t n = 1) {
  using S = GatherSlot<PACKED>;
  using W = typename S::T;
  const uint32_t mask = (1u << cap_log2) - 1u;
  uint32_t s = slot_of(j, cap_log2);
  const W item = ((W)j << S::kShift) | (W)n;
  while (true) {
    const W cur = atomicCAS(&T[s], S::kEmpty, item);
    if (cur == S::kEmpty) return;
    if (S::key(cur) == j) {
      atomicAdd(&T[s], (W)n);
      return;
    }
    s = (s + 1u) & mask;
  }
}

// Row i of a heavy hyperedge: its heavy neighbours come from the dense tiles, so the
// gather skips them; light rows (and a graph without a dense path) gather everything.
__device__ __forceinline__ bool gather_pair(const DenseInfo& dn, int32_t hi, int32_t j) {
  return hi < 0 || dn.heavy_idx[j] < 0;
}

// Table size of a row: the smallest power of two >= 2 * (its gathered incidences), so the
// load factor stays <= 1/2, clamped to [2^lo, 2^hi].
__device__ __forceinline__ int row_cap_log2(int64_t cand, int lo, int hi) {
  int l = lo;
  while (l < hi && (int64_t(1) << l) < 2 * cand) ++l;
  return l;
}

__device__ __forceinline__ bool ranked_above(int32_t di, int32_t i, int32_t dj, int32_t j) {
  return di < dj || (di == dj && i < j);
}

template <bool PACKED>
__device__ __forceinline__ void put_entry(const Oriented& o, int64_t at, uint32_t j, uint32_t om) {
  if (PACKED) {
    o.packed[at] = (j << 8) | om;
  } else {
    o.nbr[at] = (int32_t)j;
    o.omega[at] = (int32_t)om;
  }
}

// One warp per row; the table lives in shared memory.
#ifndef HG_LIGHT_MIN_BLOCKS
#define HG_LIGHT_MIN_BLOCKS 8
#endif
template <bool PACKED>
__global__ void __launch_bounds__(kLightWarps * 32, HG_LIGHT_MIN_BLOCKS)
    k_wedge_light(DevGraph g, const int32_t* __restrict__ rows, const int32_t* __restrict__ nrows_p,
                  const int64_t* __restrict__ cand, int32_t* __restrict__ deg,
                  unsigned long long* __restrict__ wc, Oriented o, int* __restrict__ err,
                  int32_t* __restrict__ counter, DenseInfo dn, RowCounts rc) {
  using S = GatherSlot<PACKED>;
  using W = typename S::T;
  constexpr int kLightCapLog2 = light_cap_log2<PACKED>();
  constexpr int CAP = 1 << kLightCapLog2;
  __shared__ W tab[kLightWarps][CAP];
  __shared__ unsigned long long blk_wc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  W* T = tab[w];
  const int32_t nrows = *nrows_p;
  if (threadIdx.x == 0) blk_wc = 0;
  __syncthreads();
  unsigned long long my_wc = 0;
  while (true) {
    int r = 0;
    if (lane == 0) r = atomicAdd(counter, 1);
    r = __shfl_sync(kFull, r, 0);
    if (r >= nrows) break;
    const int32_t i = rows[r];
    const int cl = row_cap_log2(cand[i], 5, kLightCapLog2);   // this row's table: 2^cl slots
    const int cap = 1 << cl;
    for (int s = lane; s < cap; s += 32) T[s] = S::kEmpty;
    __syncwarp();
    const int32_t hi = dn.heavy_idx ? dn.heavy_idx[i] : -1;
    const int64_t b = g.e_ptr[i], e = g.e_ptr[i + 1];
    // 32 vertices of e_i at a time: their E_v ranges in one round trip (lane l holds
    // vertex p0 + l), then the concatenated lists as one flat range, 32 entries per step.
    // A light row gathers at most 2^kLightCapLog2 incidences, so the prefix sums are
    // 32-bit; each lane keeps the 64-bit start of its list minus its exclusive prefix.
    for (int64_t p0 = b; p0 < e; p0 += 32) {
      int64_t yb = 0;
      int32_t len = 0;
      if (p0 + lane < e) {
        const int32_t v = g.e_idx[p0 + lane];
        yb = g.v_ptr[v];
        len = (int32_t)(g.v_ptr[v + 1] - yb);
      }
      int32_t incl = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t o2 = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += o2;
      }
      const int64_t base = yb - (incl - len);   // flat position f of this list: v_idx[base + f]
      const int32_t total = __shfl_sync(kFull, incl, 31);
      for (int32_t f0 = 0; f0 < total; f0 += 32) {   // warp-uniform: all lanes shuffle
        const int32_t f = f0 + lane;
        int lo = 0, hi2 = 31;   // owner: first lane whose inclusive prefix exceeds f
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const int mid = (lo + hi2) >> 1;
          if (__shfl_sync(kFull, incl, mid) > f) hi2 = mid; else lo = mid + 1;
        }
        const int64_t start = __shfl_sync(kFull, base, lo);
        if (f >= total) continue;
        const int32_t j = g.v_idx[start + f];
        if (j != i && gather_pair(dn, hi, j)) ht_add<PACKED>(T, cl, (uint32_t)j);
      }
    }
    if (hi >= 0) {
      for (int32_t h = lane; h < dn.nh; h += 32) {
        const uint32_t om = dn.omega[(int64_t)hi * dn.ld + h];
        if (om && h != hi) ht_add<PACKED>(T, cl, (uint32_t)dn.ids[h], om);
      }
    }
    __syncwarp();
    const int32_t szi = (int32_t)(e - b);
    const int64_t base = o.row_ptr[i];
    int written = 0, up = 0, incl = 0;
    for (int s0 = 0; s0 < cap; s0 += 32) {
      const W x = T[s0 + lane];
      const bool valid = x != S::kEmpty;
      uint32_t j = 0, om = 0;
      if (valid) {
        j = S::key(x);
        om = S::count(x);
        if ((int32_t)j > i) {
          ++up;
          const int32_t szj = g.esize[j];
          if ((int32_t)om == szi && (int32_t)om == szj) dev_fail(err, DE_DUPEDGE);
          if ((int32_t)om == min(szi, szj)) ++incl;
        }
      }
      const unsigned bal = __ballot_sync(kFull, valid);
      if (valid) put_entry<PACKED>(o, base + written + __popc(bal & ((1u << lane) - 1u)), j, om);
      written += __popc(bal);
    }
    my_wc += (unsigned long long)incl;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      up += __shfl_down_sync(kFull, up, d);
      incl += __shfl_down_sync(kFull, incl, d);
    }
    if (lane == 0) {
      deg[i] = written;
      if (rc.upc) rc.upc[i] = up;
      if (rc.wcr) rc.wcr[i] = incl;
    }
    __syncwarp();
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) my_wc += __shfl_down_sync(kFull, my_wc, d);
  if (lane == 0) atomicAdd(&blk_wc, my_wc);
  __syncthreads();
  if (threadIdx.x == 0 && blk_wc) atomicAdd(wc, blk_wc);
}

// One block per row; the table is in dynamic shared memory (SMEM) or in a
// per-block slice of global scratch.
template <bool PACKED, bool SMEM>
__global__ void __launch_bounds__(kBlockThreads)
    k_wedge_block(DevGraph g, const int32_t* __restrict__ rows, const int32_t* __restrict__ nrows_p,
                  const int64_t* __restrict__ cand, int cap_log2,
                  unsigned long long* __restrict__ gscratch, int32_t* __restrict__ deg,
                  unsigned long long* __restrict__ wc, Oriented o, int* __restrict__ err,
                  int32_t* __restrict__ counter, DenseInfo dn, RowCounts rc) {
  using S = GatherSlot<PACKED>;
  using W = typename S::T;
  extern __shared__ unsigned long long dyn[];
  W* T = SMEM ? reinterpret_cast<W*>(dyn)
              : reinterpret_cast<W*>(gscratch) + ((size_t)blockIdx.x << cap_log2);
  __shared__ int32_t s_row;
  __shared__ int32_t s_cnt, s_up, s_incl;
  __shared__ unsigned long long s_wc;
  __shared__ int64_t s_ybeg[32];
  __shared__ int32_t s_yincl[32];   // a row gathers fewer than 2^30 incidences (host check)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t nrows = *nrows_p;
  if (threadIdx.x == 0) s_wc = 0;
  unsigned long long my_wc = 0;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_row = atomicAdd(counter, 1);
      s_cnt = 0;
      s_up = 0;
      s_incl = 0;
    }
    __syncthreads();
    const int32_t r = s_row;
    if (r >= nrows) break;
    const int32_t i = rows[r];
    const int cl = row_cap_log2(cand[i], 8, cap_log2);   // this row's table: 2^cl slots
    const uint32_t CAP = 1u << cl;
    for (uint32_t s = threadIdx.x; s < CAP; s += kBlockThreads) T[s] = S::kEmpty;
    __syncthreads();
    const int32_t hi = dn.heavy_idx ? dn.heavy_idx[i] : -1;
    const int64_t b = g.e_ptr[i], e = g.e_ptr[i + 1];
    // 32 vertices of e_i at a time: warp 0 puts their E_v ranges and prefix sums in
    // shared memory, then every thread takes flat positions of the concatenated lists
    for (int64_t p0 = b; p0 < e; p0 += 32) {   // block-uniform
      if (w == 0) {
        int64_t yb = 0;
        int32_t len = 0;
        if (p0 + lane < e) {
          const int32_t v = g.e_idx[p0 + lane];
          yb = g.v_ptr[v];
          len = (int32_t)(g.v_ptr[v + 1] - yb);
        }
        int32_t incl = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int32_t o2 = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += o2;
        }
        s_ybeg[lane] = yb - (incl - len);   // flat position f of this list maps to s_ybeg + f
        s_yincl[lane] = incl;
      }
      __syncthreads();
      const int32_t total = s_yincl[31];
      for (int32_t f = threadIdx.x; f < total; f += kBlockThreads) {
        int lo = 0, hi2 = 31;   // owner: first vertex whose inclusive prefix exceeds f
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const int mid = (lo + hi2) >> 1;
          if (s_yincl[mid] > f) hi2 = mid; else lo = mid + 1;
        }
        const int32_t j = g.v_idx[s_ybeg[lo] + f];
        if (j != i && gather_pair(dn, hi, j)) ht_add<PACKED>(T, cl, (uint32_t)j);
      }
      __syncthreads();   // the next chunk rewrites the ranges
    }
    if (hi >= 0) {
      for (int32_t h = threadIdx.x; h < dn.nh; h += kBlockThreads) {
        const uint32_t om = dn.omega[(int64_t)hi * dn.ld + h];
        if (om && h != hi) ht_add<PACKED>(T, cl, (uint32_t)dn.ids[h], om);
      }
    }
    __syncthreads();
    const int32_t szi = (int32_t)(e - b);
    const int64_t base = o.row_ptr[i];
    int up = 0, incl = 0;
    for (uint32_t s = threadIdx.x; s < CAP; s += kBlockThreads) {
      const W x = T[s];
      if (x == S::kEmpty) continue;
      const uint32_t j = S::key(x), om = S::count(x);
      if ((int32_t)j > i) {
        ++up;
        const int32_t szj = g.esize[j];
        if ((int32_t)om == szi && (int32_t)om == szj) dev_fail(err, DE_DUPEDGE);
        if ((int32_t)om == min(szi, szj)) ++incl;
      }
      put_entry<PACKED>(o, base + atomicAdd(&s_cnt, 1), j, om);
    }
    my_wc += (unsigned long long)incl;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      up += __shfl_down_sync(kFull, up, d);
      incl += __shfl_down_sync(kFull, incl, d);
    }
    if (lane == 0) {
      atomicAdd(&s_up, up);
      atomicAdd(&s_incl, incl);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      deg[i] = s_cnt;
      if (rc.upc) rc.upc[i] = s_up;
      if (rc.wcr) rc.wcr[i] = s_incl;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) my_wc += __shfl_down_sync(kFull, my_wc, d);
  if (lane == 0) atomicAdd(&s_wc, my_wc);
  __syncthreads();
  if (threadIdx.x == 0 && s_wc) atomicAdd(wc, s_wc);
}

// Row capacity of the gather pass: min(gathered incidences, |E| - 1) distinct neighbours.
__global__ void k_cap_rows(const int64_t* __restrict__ cand, int32_t ne, int32_t* __restrict__ cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cand[i];
    cap[i] = (int32_t)(c < (int64_t)ne - 1 ? c : (int64_t)ne - 1);
  }
}

template <bool PACKED>
__device__ __forceinline__ void get_row_entry(const Oriented& o, int64_t at, uint32_t& j,
                                              uint32_t& om) {
  if (PACKED) {
    const uint32_t x = o.packed[at];
    j = x >> 8;
    om = x & 0xffu;
  } else {
    j = (uint32_t)o.nbr[at];
    om = (uint32_t)o.omega[at];
  }
}

// One warp per row: row i of the capacity layout (len[i] entries from src_ptr[i]) filtered
// into row i of an exact layout (from dst_ptr[i]), order kept.  KEEP 0: j ranked above i in
// (deg, id) (the oriented line graph); 1: j > i; 2: every entry.  COUNT: only the number
// kept, into cnt[i]; otherwise the rows, and the number kept into cnt[i] when cnt is set.
template <int KEEP, bool PACKED, bool COUNT>
__global__ void k_filter_rows(const int64_t* __restrict__ src_ptr, const int32_t* __restrict__ len,
                              Oriented src, const int32_t* __restrict__ deg, int32_t ne,
                              const int64_t* __restrict__ dst_ptr, Oriented dst,
                              int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < ne; i += warps) {
    const int64_t b = src_ptr[i];
    const int32_t n = len[i];
    const int32_t di = KEEP == 0 ? deg[i] : 0;
    const int64_t out = COUNT ? 0 : dst_ptr[i];
    int32_t kept = 0;
    for (int32_t t0 = 0; t0 < n; t0 += 32) {
      const int32_t t = t0 + lane;
      bool keep = false;
      uint32_t j = 0, om = 0;
      if (t < n) {
        get_row_entry<PACKED>(src, b + t, j, om);
        keep = KEEP == 0 ? ranked_above(di, i, deg[j], (int32_t)j)
                         : (KEEP == 1 ? (int32_t)j > i : true);
      }
      const unsigned bal = __ballot_sync(kFull, keep);
      if (!COUNT && keep) put_entry<PACKED>(dst, out + kept + __popc(bal & ((1u << lane) - 1u)), j, om);
      kept += __popc(bal);
    }
    if (lane == 0 && cnt) cnt[i] = kept;
  }
}

// Sort rows into the three buckets by their gather count.
__global__ void k_bucket_rows(const int64_t* __restrict__ cand, int32_t ne, WedgeBuckets b,
                              int64_t light_max, int64_t medium_max) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ne;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int bucket = -1;
    if (i < ne) {
      const int64_t c = cand[i];
      if (c > 0) bucket = c <= light_max ? 0 : (c <= medium_max ? 1 : 2);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const unsigned bal = __ballot_sync(kFull, bucket == k);
      if (!bal) continue;
      int32_t at = 0;
      const int leader = __ffs(bal) - 1;
      if (lane == leader) at = atomicAdd(&b.count[k], __popc(bal));
      at = __shfl_sync(kFull, at, leader);
      if (bucket == k) b.rows[k][at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
}

int cap_log2_for(int64_t cand) {
  int l = 4;
  while ((int64_t(1) << l) < 2 * cand) ++l;
  return l;
}

template <bool PACKED>
void launch_all(const DevGraph& g, const WedgeBuckets& b, const int32_t* nb, int64_t heavy_max,
                const int64_t* cand, int32_t* deg, unsigned long long* wc, const Oriented& o,
                unsigned long long* scratch, int* err, int32_t* counters, const DenseInfo& dn,
                RowCounts rc, cudaStream_t s, int nsm) {
  // counters[0..2] are zeroed by the caller
  if (nb[0] > 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wedge_light<PACKED>,
                                                  kLightWarps * 32, 0);
    if (per_sm < 1) per_sm = 1;
    int blocks = (nb[0] + kLightWarps - 1) / kLightWarps;
    blocks = blocks < nsm * per_sm ? blocks : nsm * per_sm;
    note_launch();
    k_wedge_light<PACKED><<<blocks, kLightWarps * 32, 0, s>>>(g, b.rows[0], b.count + 0, cand,
                                                              deg, wc, o, err, counters + 0, dn,
                                                              rc);
  }
  if (nb[1] > 0) {
    const size_t smem = sizeof(typename GatherSlot<PACKED>::T) << kMediumCapLog2;
    cudaFuncSetAttribute(k_wedge_block<PACKED, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wedge_block<PACKED, true>,
                                                  kBlockThreads, smem);
    if (per_sm < 1) per_sm = 1;
    int blocks = nb[1] < nsm * per_sm ? nb[1] : nsm * per_sm;
    note_launch();
    k_wedge_block<PACKED, true><<<blocks, kBlockThreads, smem, s>>>(
        g, b.rows[1], b.count + 1, cand, kMediumCapLog2, nullptr, deg, wc, o, err, counters + 1,
        dn, rc);
  }
  if (nb[2] > 0) {
    int blocks = nb[2] < nsm * 2 ? nb[2] : nsm * 2;
    note_launch();
    k_wedge_block<PACKED, false><<<blocks, kBlockThreads, 0, s>>>(
        g, b.rows[2], b.count + 2, cand, cap_log2_for(heavy_max), scratch, deg, wc, o, err,
        counters + 2, dn, rc);
  }
}

int grid_rows(int64_t rows, int per_block) {
  int64_t b = (rows + per_block - 1) / per_block;
  if (b > 65535) b = 65535;
  if (b < 1) b = 1;
  return (int)b;
}

template <int KEEP, bool PACKED>
void launch_filter_t(bool count_only, const int64_t* src_ptr, const int32_t* len,
                     const Oriented& src, const int32_t* deg, int32_t ne, const int64_t* dst_ptr,
                     const Oriented& dst, int32_t* cnt, cudaStream_t s) {
  note_launch();
  if (count_only)
    k_filter_rows<KEEP, PACKED, true><<<grid_rows(ne, 8), 256, 0, s>>>(src_ptr, len, src, deg, ne,
                                                                        dst_ptr, dst, cnt);
  else
    k_filter_rows<KEEP, PACKED, false><<<grid_rows(ne, 8), 256, 0, s>>>(src_ptr, len, src, deg,
                                                                         ne, dst_ptr, dst, cnt);
}

}  // namespace

int wedge_light_max_cand(int packed) {
  return (1 << (packed ? light_cap_log2<true>() : light_cap_log2<false>())) / 2;
}
int wedge_medium_max_cand() { return (1 << kMediumCapLog2) / 2; }

size_t wedge_heavy_scratch_bytes(int64_t heavy_max_cand, int nsm) {
  if (heavy_max_cand <= 0) return 0;
  return (sizeof(unsigned long long) << cap_log2_for(heavy_max_cand)) * (size_t)(nsm * 2);
}

void launch_bucket_rows(const int64_t* cand, int32_t ne, WedgeBuckets b, int light_max,
                        cudaStream_t s) {
  if (ne == 0) return;
  int64_t blocks = (ne + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  note_launch();
  k_bucket_rows<<<(unsigned)blocks, 256, 0, s>>>(cand, ne, b, light_max, wedge_medium_max_cand());
}

void launch_wedge_rows(const DevGraph& g, const WedgeBuckets& b, const int32_t* nb,
                       int64_t heavy_max_cand, const int64_t* cand, int32_t* deg,
                       unsigned long long* wc, const Oriented& rows, int packed,
                       unsigned long long* scratch, int* err, int32_t* work_counter,
                       const DenseInfo& dn, RowCounts rc, cudaStream_t s, int nsm) {
  if (packed)
    launch_all<true>(g, b, nb, heavy_max_cand, cand, deg, wc, rows, scratch, err, work_counter, dn,
                     rc, s, nsm);
  else
    launch_all<false>(g, b, nb, heavy_max_cand, cand, deg, wc, rows, scratch, err, work_counter,
                      dn, rc, s, nsm);
}

void launch_cap_rows(const int64_t* cand, int32_t ne, int32_t* cap, cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_cap_rows<<<grid_rows(ne, 256), 256, 0, s>>>(cand, ne, cap);
}

void launch_filter_rows(int keep, bool count_only, const int64_t* src_ptr, const int32_t* len,
                        const Oriented& src, const int32_t* deg, int32_t ne, int packed,
                        const int64_t* dst_ptr, const Oriented& dst, int32_t* cnt,
                        cudaStream_t s) {
  if (ne == 0) return;
#define HG_FILTER(K)                                                                        \
  if (packed)                                                                              \
    launch_filter_t<K, true>(count_only, src_ptr, len, src, deg, ne, dst_ptr, dst, cnt, s); \
  else                                                                                     \
    launch_filter_t<K, false>(count_only, src_ptr, len, src, deg, ne, dst_ptr, dst, cnt, s);
  if (keep == 0) {
    HG_FILTER(0)
  } else if (keep == 1) {
    HG_FILTER(1)
  } else {
    HG_FILTER(2)
  }
#undef HG_FILTER
}

}  // namespace hg
