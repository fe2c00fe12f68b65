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
// seven Venn regions (g = |e_i cap e_j cap e_k| from the staged e_i cap e_j) and
// counted.
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

// ------------------------------------------------------------------ warp routines
//
// A draw (i, j) closes its triangles by probing each candidate k in a sorted row of
// j, and computes g = |e_i cap e_j cap e_k| for each.  Both are served from the warp's
// shared memory when they fit: the searched row is staged once per draw (a binary
// search then costs shared loads, not dependent global ones), and e_i cap e_j (of
// size omega_ij, known from the entry) is staged once, so that g needs omega_ij
// binary searches in e_k instead of a 3-way merge.

constexpr int kCacheEntries = 384;   // searched rows up to this long go to shared memory
constexpr int kCommonMax = 64;       // e_i cap e_j up to this large goes to shared memory

struct WarpCache {
  int32_t key[kCacheEntries];
  int32_t om[kCacheEntries];
  int32_t common[kCommonMax];
};

// Reads made by a warp, for roofline accounting: [0] row pointers, [1] row entries,
// [2] vertex ids.  Lanes count their own; reduced at exit.
struct ReadCount {
  unsigned long long ptr = 0, ent = 0, vtx = 0;
  __device__ void flush(unsigned long long* work, int lane) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      ptr += __shfl_down_sync(kFull, ptr, d);
      ent += __shfl_down_sync(kFull, ent, d);
      vtx += __shfl_down_sync(kFull, vtx, d);
    }
    if (lane == 0 && work) {
      atomicAdd(&work[0], ptr);
      atomicAdd(&work[1], ent);
      atomicAdd(&work[2], vtx);
    }
  }
};

// Copy row [b, e) into the cache when it fits (warp-uniform; all lanes).
__device__ __forceinline__ bool stage_row(WarpCache& c, const Oriented& rows, int packed,
                                          int64_t b, int64_t e, int lane, ReadCount& rc) {
  const int64_t len = e - b;
  if (len > kCacheEntries) return false;
  for (int64_t t = lane; t < len; t += 32) {
    int32_t x, om;
    up_entry(rows, packed, b + t, x, om);
    c.key[t] = x;
    c.om[t] = om;
    ++rc.ent;
  }
  __syncwarp();
  return true;
}

// omega of key k in row [b, e) (sorted), -1 when absent.
__device__ __forceinline__ int find_in_row(const WarpCache& c, bool cached, const Oriented& rows,
                                           int packed, int64_t b, int64_t e, int32_t k,
                                           ReadCount& rc) {
  if (cached) {
    int l = 0, h = (int)(e - b);
    while (l < h) {
      const int mid = (l + h) >> 1;
      if (c.key[mid] < k) l = mid + 1; else h = mid;
    }
    return (l < (int)(e - b) && c.key[l] == k) ? c.om[l] : -1;
  }
  int64_t l = b, h = e;
  while (l < h) {
    const int64_t mid = (l + h) >> 1;
    int32_t x, om;
    up_entry(rows, packed, mid, x, om);
    ++rc.ent;
    if (x < k) l = mid + 1; else h = mid;
  }
  if (l >= e) return -1;
  int32_t x, om;
  up_entry(rows, packed, l, x, om);
  ++rc.ent;
  return x == k ? om : -1;
}

__device__ __forceinline__ bool in_sorted(const int32_t* a, int n, int32_t y, ReadCount& rc) {
  int l = 0, h = n;
  while (l < h) {
    const int mid = (l + h) >> 1;
    const int32_t x = __ldg(a + mid);
    ++rc.vtx;
    if (x < y) l = mid + 1; else h = mid;
  }
  if (l >= n) return false;
  ++rc.vtx;
  return __ldg(a + l) == y;
}

// e_i cap e_j into the cache (ascending) when omega_ij fits (warp-uniform; all lanes).
__device__ __forceinline__ bool stage_common(WarpCache& c, const int32_t* ei, int szi,
                                             const int32_t* ej, int szj, int wij, int lane,
                                             ReadCount& rc) {
  if (wij > kCommonMax) return false;
  const bool a_is_i = szi <= szj;
  const int32_t* a = a_is_i ? ei : ej;
  const int32_t* b = a_is_i ? ej : ei;
  const int na = a_is_i ? szi : szj, nb = a_is_i ? szj : szi;
  int n = 0;
  for (int t0 = 0; t0 < na; t0 += 32) {
    const int t = t0 + lane;
    bool in = false;
    int32_t y = 0;
    if (t < na) {
      y = __ldg(a + t);
      ++rc.vtx;
      in = in_sorted(b, nb, y, rc);
    }
    const unsigned bal = __ballot_sync(kFull, in);
    if (in && n + __popc(bal & ((1u << lane) - 1u)) < kCommonMax)
      c.common[n + __popc(bal & ((1u << lane) - 1u))] = y;
    n += __popc(bal);
  }
  __syncwarp();
  return n == wij;
}

// g = |e_i cap e_j cap e_k|
__device__ __forceinline__ int common3(const WarpCache& c, bool staged, int wij,
                                       const int32_t* ei, int szi, const int32_t* ej, int szj,
                                       const int32_t* ek, int szk, ReadCount& rc) {
  if (staged) {
    int gg = 0;
    for (int t = 0; t < wij; ++t) gg += in_sorted(ek, szk, c.common[t], rc);
    return gg;
  }
  rc.vtx += (unsigned long long)(szi + szj + szk);
  return triple_common(ei, szi, ej, szj, ek, szk);
}

__device__ __forceinline__ int region_bits7(int szi, int szj, int szk, int wij, int wik, int wjk,
                                            int gg) {
  const int ra = szi - wij - wik + gg, rb = szj - wij - wjk + gg, rc = szk - wik - wjk + gg;
  return (ra > 0) | ((rb > 0) << 1) | ((rc > 0) << 2) | ((wij > gg) << 3) | ((wjk > gg) << 4) |
         ((wik > gg) << 5) | ((gg > 0) << 6);
}

// Bucket index of a row-pointer array: bucket b covers entries [b << shift, (b+1) << shift)
// and first[b] is the row holding entry b << shift, so the row of entry m lies in
// [first[m >> shift], first[(m >> shift) + 1]] (first has one more, sentinel, entry).
struct RowIndex {
  const int32_t* first;
  int shift;
  int64_t buckets;
};

// Row of entry m: the last i with ptr[i] <= m (searched between the bucket bounds).
__device__ __forceinline__ int32_t row_of(const int64_t* __restrict__ ptr, int32_t ne,
                                          const RowIndex& ix, uint64_t m, int lane,
                                          ReadCount& rc) {
  int32_t lo = 0, hi = ne - 1;
  if (ix.first) {
    const int64_t b = (int64_t)(m >> ix.shift);
    lo = __ldg(ix.first + b);
    hi = __ldg(ix.first + b + 1);
    if (lane == 0) rc.ptr += 1;   // two 4-byte reads
  }
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(ptr + mid) <= (int64_t)m) lo = mid; else hi = mid - 1;
    if (lane == 0) ++rc.ptr;
  }
  return lo;
}

// first[b] for every bucket: row i writes the buckets whose first entry it holds.
__global__ void k_row_index(const int64_t* __restrict__ ptr, int32_t ne, int shift,
                            int64_t buckets, int32_t* __restrict__ first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b0 = (ptr[i] + ((int64_t(1) << shift) - 1)) >> shift;
    const int64_t b1 = (ptr[i + 1] + ((int64_t(1) << shift) - 1)) >> shift;
    for (int64_t b = b0; b < b1; ++b) first[b] = (int32_t)i;
    if (i == ne - 1) first[buckets] = (int32_t)(ne - 1);
  }
}

// One warp per sample (grid-stride).  raw[0..23] += per-pattern counts; work[0..2] +=
// the reads made (ReadCount).
__global__ void __launch_bounds__(kSampleWarps * 32)
    k_sample(DevGraph g, const int64_t* __restrict__ up_ptr, RowIndex ix, Oriented up, int packed,
             uint64_t W, uint64_t seed, uint64_t first, uint64_t num,
             unsigned long long* __restrict__ raw, unsigned long long* __restrict__ work) {
  __shared__ uint32_t hist[kSampleWarps][24];
  __shared__ uint8_t lut[128];
  __shared__ WarpCache cache[kSampleWarps];
  ReadCount rc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpCache& cw = cache[w];
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
    const int32_t i = row_of(up_ptr, g.ne, ix, m, lane, rc);
    const int64_t ib = (int64_t)m, ie = __ldg(up_ptr + i + 1);
    int32_t j, wij;
    up_entry(up, packed, ib, j, wij);
    const int64_t jb = __ldg(up_ptr + j), je = __ldg(up_ptr + j + 1);
    const int32_t* ei = g.e_idx + g.e_ptr[i];
    const int32_t* ej = g.e_idx + g.e_ptr[j];
    const int szi = g.esize[i], szj = g.esize[j];
    if (lane == 0) {
      rc.ptr += 3;
      rc.ent += 1;
    }
    __syncwarp();   // the previous draw's readers are done with the cache
    const bool walk = ie > ib + 1;   // warp-uniform
    const bool cached = walk && stage_row(cw, up, packed, jb, je, lane, rc);
    const bool staged = walk && stage_common(cw, ei, szi, ej, szj, wij, lane, rc);
    // k > j in upper(i) (the entries after m) that are in upper(j)
    for (int64_t a = ib + 1 + lane; a < ie; a += 32) {
      int32_t k, wik;
      up_entry(up, packed, a, k, wik);
      ++rc.ent;
      const int wjk = find_in_row(cw, cached, up, packed, jb, je, k, rc);
      if (wjk < 0) continue;
      const int32_t* ek = g.e_idx + g.e_ptr[k];
      const int szk = g.esize[k];
      const int gg = common3(cw, staged, wij, ei, szi, ej, szj, ek, szk, rc);
      atomicAdd(&hist[w][lut[region_bits7(szi, szj, szk, wij, wik, wjk, gg)]], 1u);
    }
  }
  rc.flush(work, lane);
  __syncthreads();
  for (int k = threadIdx.x; k < 24; k += blockDim.x) {
    unsigned long long x = 0;
    for (int ww = 0; ww < kSampleWarps; ++ww) x += hist[ww][k];
    if (x) atomicAdd(&raw[k], x);
  }
}

// ------------------------------------------------------------------ Appro-adv (Algorithm 7)

// cnt_t[i] = upper entries of intersection type = upc[i] - wcr[i]
__global__ void k_type_counts(const int32_t* __restrict__ upc, const int32_t* __restrict__ wcr,
                              int32_t ne, int32_t* __restrict__ cnt_t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x)
    cnt_t[i] = upc[i] - wcr[i];
}

__device__ __forceinline__ void put_up(const Oriented& o, int packed, int64_t at, int32_t j,
                                       int32_t om) {
  if (packed) {
    o.packed[at] = ((uint32_t)j << 8) | (uint32_t)om;
  } else {
    o.nbr[at] = j;
    o.omega[at] = om;
  }
}

// One warp per row: the sorted upper row split, order kept, into its intersection-type
// entries (t) and inclusion-type entries (c) (Def. 2.3: omega_ij = min(|e_i|, |e_j|)).
__global__ void k_split_types(const DevGraph g, const int64_t* __restrict__ up_ptr, Oriented up,
                              int packed, const int64_t* __restrict__ t_ptr, Oriented t,
                              const int64_t* __restrict__ c_ptr, Oriented c) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < g.ne; i += warps) {
    const int64_t b = up_ptr[i], e = up_ptr[i + 1];
    const int32_t szi = g.esize[i];
    int64_t nt = t_ptr[i], nc = c_ptr[i];
    for (int64_t p0 = b; p0 < e; p0 += 32) {
      const int64_t p = p0 + lane;
      int32_t j = 0, om = 0;
      bool incl = false;
      if (p < e) {
        up_entry(up, packed, p, j, om);
        incl = om == min(szi, g.esize[j]);
      }
      const unsigned bc = __ballot_sync(kFull, p < e && incl);
      const unsigned bt = __ballot_sync(kFull, p < e && !incl);
      const unsigned below = (1u << lane) - 1u;
      if (p < e) {
        if (incl) put_up(c, packed, nc + __popc(bc & below), j, om);
        else put_up(t, packed, nt + __popc(bt & below), j, om);
      }
      nt += __popc(bt);
      nc += __popc(bc);
    }
  }
}

// pattern -> class (0 CCC, 1 TCC, 2 TTC, 3 TTT; Sec. 2)
__constant__ int8_t c_class_of[24] = {-1, 0, 1, 1, 1, 1, 2, 2, 2, 3, 3, 3, 3,
                                      3,  3, 3, 3, 3, 3, 3, 3, -1, -1, -1};

struct AdvSet {
  const int64_t* ptr;   // rows of the drawn type
  RowIndex ix;          // bucket index of ptr
  Oriented ent;
  uint64_t Wx;          // hyperwedges of that type
  int type;             // 0 intersection, 1 inclusion
  int cls;              // class counted
  uint32_t stream;      // Philox counter word 2
};

__device__ __forceinline__ int wedge_type(int om, int sa, int sb) { return om == min(sa, sb); }

// One warp per draw of set `st`: the drawn (i, j), every k in N(i) cap N(j) (the shorter
// row walked, the longer searched); the triangle counts when its class is st.cls and
// (i, j) is its first hyperwedge of type st.type in O.  raw[0..23] += per-pattern counts.
__global__ void __launch_bounds__(kSampleWarps * 32)
    k_sample_adv(DevGraph g, AdvSet st, const int64_t* __restrict__ full_ptr, Oriented full,
                 int packed, uint64_t seed, uint64_t first, uint64_t num,
                 unsigned long long* __restrict__ raw) {
  __shared__ uint32_t hist[kSampleWarps][24];
  __shared__ uint8_t lut[128];
  __shared__ WarpCache cache[kSampleWarps];
  ReadCount rc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpCache& cw = cache[w];
  for (int k = threadIdx.x; k < 128; k += blockDim.x) lut[k] = c_sample_lut[k];
  for (int k = lane; k < 24; k += 32) hist[w][k] = 0;
  __syncthreads();
  const uint64_t warps = (uint64_t)gridDim.x * kSampleWarps;
  for (uint64_t s = (uint64_t)blockIdx.x * kSampleWarps + w; s < num; s += warps) {
    const uint64_t n = first + s;
    uint32_t c[4] = {(uint32_t)n, (uint32_t)(n >> 32), st.stream, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t r = ((uint64_t)c[1] << 32) | c[0];
    const uint64_t m = __umul64hi(r, st.Wx);
    const int32_t i = row_of(st.ptr, g.ne, st.ix, m, lane, rc);
    int32_t j, wij;
    up_entry(st.ent, packed, (int64_t)m, j, wij);
    const int32_t* ei = g.e_idx + g.e_ptr[i];
    const int32_t* ej = g.e_idx + g.e_ptr[j];
    const int szi = g.esize[i], szj = g.esize[j];
    // walk the shorter neighbour row, search the longer one
    int64_t ab = __ldg(full_ptr + i), ae = __ldg(full_ptr + i + 1);
    int64_t bb = __ldg(full_ptr + j), be = __ldg(full_ptr + j + 1);
    const bool swap = (ae - ab) > (be - bb);
    if (swap) {
      int64_t t0 = ab, t1 = ae;
      ab = bb;
      ae = be;
      bb = t0;
      be = t1;
    }
    __syncwarp();
    const bool cached = stage_row(cw, full, packed, bb, be, lane, rc);
    const bool staged = stage_common(cw, ei, szi, ej, szj, wij, lane, rc);
    for (int64_t a = ab + lane; a < ae; a += 32) {
      int32_t k, wa;
      up_entry(full, packed, a, k, wa);
      ++rc.ent;
      if (k == i || k == j) continue;
      const int wb = find_in_row(cw, cached, full, packed, bb, be, k, rc);
      if (wb < 0) continue;
      const int wik = swap ? wb : wa, wjk = swap ? wa : wb;
      const int32_t* ek = g.e_idx + g.e_ptr[k];
      const int szk = g.esize[k];
      const int gg = common3(cw, staged, wij, ei, szi, ej, szj, ek, szk, rc);
      const int pat = lut[region_bits7(szi, szj, szk, wij, wik, wjk, gg)];
      if (c_class_of[pat] != st.cls) continue;
      // the triangle's hyperwedges in O, (a,b) < (a,c) < (b,c) for a < b < c; the
      // first of the drawn type must be (i, j)
      const int tij = wedge_type(wij, szi, szj), tik = wedge_type(wik, szi, szk),
                tjk = wedge_type(wjk, szj, szk);
      int32_t v0 = i, v1 = j, v2 = k;
      int t01 = tij, t02 = tik, t12 = tjk;   // types of the pairs (v0,v1), (v0,v2), (v1,v2)
      // sort the three ids, carrying the pair types along
      if (v0 > v1) { int32_t q = v0; v0 = v1; v1 = q; int tq = t02; t02 = t12; t12 = tq; }
      if (v1 > v2) { int32_t q = v1; v1 = v2; v2 = q; int tq = t01; t01 = t02; t02 = tq; }
      if (v0 > v1) { int32_t q = v0; v0 = v1; v1 = q; int tq = t02; t02 = t12; t12 = tq; }
      int32_t oa, ob;
      if (t01 == st.type) { oa = v0; ob = v1; }
      else if (t02 == st.type) { oa = v0; ob = v2; }
      else { oa = v1; ob = v2; }
      if (oa == min(i, j) && ob == max(i, j)) atomicAdd(&hist[w][pat], 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 24; k += blockDim.x) {
    unsigned long long x = 0;
    for (int ww = 0; ww < kSampleWarps; ++ww) x += hist[ww][k];
    if (x) atomicAdd(&raw[k], x);
  }
}

// ------------------------------------------------------------------ single-pattern enumeration

// One warp per hyperwedge (i, j) of the upper rows (m over 0 .. W-1): every k > j in both
// upper(i) and upper(j) closes the triangle i < j < k (each found once); those of pattern
// `target` (0 = all) are appended to out as (i, j, k), while fewer than cap were written.
__global__ void __launch_bounds__(kSampleWarps * 32)
    k_enumerate(DevGraph g, const int64_t* __restrict__ up_ptr, RowIndex ix, Oriented up,
                int packed, uint64_t W, int target, int32_t* __restrict__ out,
                unsigned long long cap, unsigned long long* __restrict__ count) {
  __shared__ uint8_t lut[128];
  __shared__ WarpCache cache[kSampleWarps];
  ReadCount rc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpCache& cw = cache[w];
  for (int k = threadIdx.x; k < 128; k += blockDim.x) lut[k] = c_sample_lut[k];
  __syncthreads();
  const uint64_t warps = (uint64_t)gridDim.x * kSampleWarps;
  for (uint64_t m = (uint64_t)blockIdx.x * kSampleWarps + w; m < W; m += warps) {
    const int32_t i = row_of(up_ptr, g.ne, ix, m, lane, rc);
    const int64_t ie = __ldg(up_ptr + i + 1);
    if ((int64_t)m + 1 >= ie) continue;   // nothing after (i, j) in upper(i)
    int32_t j, wij;
    up_entry(up, packed, (int64_t)m, j, wij);
    const int64_t jb = __ldg(up_ptr + j), je = __ldg(up_ptr + j + 1);
    const int32_t* ei = g.e_idx + g.e_ptr[i];
    const int32_t* ej = g.e_idx + g.e_ptr[j];
    const int szi = g.esize[i], szj = g.esize[j];
    __syncwarp();
    const bool cached = stage_row(cw, up, packed, jb, je, lane, rc);
    const bool staged = stage_common(cw, ei, szi, ej, szj, wij, lane, rc);
    for (int64_t a0 = (int64_t)m + 1; a0 < ie; a0 += 32) {   // warp-uniform trip count
      const int64_t a = a0 + lane;
      bool hit = false;
      int32_t k = 0;
      if (a < ie) {
        int32_t wik;
        up_entry(up, packed, a, k, wik);
        const int wjk = find_in_row(cw, cached, up, packed, jb, je, k, rc);
        if (wjk >= 0) {
          const int32_t* ek = g.e_idx + g.e_ptr[k];
          const int szk = g.esize[k];
          const int gg = common3(cw, staged, wij, ei, szi, ej, szj, ek, szk, rc);
          hit = target == 0 || lut[region_bits7(szi, szj, szk, wij, wik, wjk, gg)] == target;
        }
      }
      const unsigned bal = __ballot_sync(kFull, hit);
      if (!bal) continue;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(bal));
      base = __shfl_sync(kFull, base, 0);
      if (hit) {
        const unsigned long long at = base + __popc(bal & ((1u << lane) - 1u));
        if (at < cap) {
          out[3 * at] = i;
          out[3 * at + 1] = j;
          out[3 * at + 2] = k;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ the sub-hypergraph G'

// Priority of hyperedge i: Philox4x32-10(counter (i, 0, 1, 0), key seed), x1 << 32 | x0.
__global__ void k_priority(int32_t ne, uint64_t seed, unsigned long long* __restrict__ pr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)i, 0u, 1u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    pr[i] = ((unsigned long long)c[1] << 32) | c[0];
  }
}

// Radix-select pass: histogram of the 16-bit digit at `shift` over the priorities whose
// higher bits equal `prefix` (mask `pmask`).
__global__ void k_digit_hist(const unsigned long long* __restrict__ pr, int32_t ne, int shift,
                             unsigned long long pmask, unsigned long long prefix,
                             unsigned int* __restrict__ hist) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = pr[i];
    if ((x & pmask) == prefix) atomicAdd(&hist[(x >> shift) & 0xffffu], 1u);
  }
}

// keep[i] = 1 for priorities below the threshold T, and for those equal to T while
// their rank among the equal ones (in id order, eq_rank = exclusive scan) is < need
__global__ void k_equal_flags(const unsigned long long* __restrict__ pr, int32_t ne,
                              unsigned long long T, int32_t* __restrict__ eq) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x)
    eq[i] = pr[i] == T;
}

__global__ void k_keep_flags(const unsigned long long* __restrict__ pr, int32_t ne,
                             unsigned long long T, const int64_t* __restrict__ eq_rank,
                             int64_t need, int32_t* __restrict__ keep) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = pr[i];
    keep[i] = x < T || (x == T && eq_rank[i] < need);
  }
}

// kept hyperedges in id order: position = exclusive scan of keep; their sizes
__global__ void k_compact_kept(const int32_t* __restrict__ keep, const int64_t* __restrict__ pos,
                               const int32_t* __restrict__ esize, int32_t ne,
                               int32_t* __restrict__ ids, int32_t* __restrict__ sizes) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x)
    if (keep[i]) {
      ids[pos[i]] = (int32_t)i;
      sizes[pos[i]] = esize[i];
    }
}

// one warp per kept hyperedge: copy its vertex row into the sub-hypergraph's CSR
__global__ void k_gather_rows(const int64_t* __restrict__ e_ptr, const int32_t* __restrict__ e_idx,
                              const int32_t* __restrict__ ids, int32_t nk,
                              const int64_t* __restrict__ sub_ptr, int32_t* __restrict__ sub_idx) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nk; q += warps) {
    const int32_t i = ids[q];
    const int64_t b = e_ptr[i], len = e_ptr[i + 1] - b, o = sub_ptr[q];
    for (int64_t t = lane; t < len; t += 32) sub_idx[o + t] = e_idx[b + t];
  }
}

int grid_n(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b > 65535) b = 65535;
  if (b < 1) b = 1;
  return (int)b;
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

int row_index_shift(uint64_t entries, int32_t rows) {
  int sh = 0;   // bucket of about entries / rows entries, at least 1
  while (rows > 0 && (entries >> (sh + 1)) >= (uint64_t)rows) ++sh;
  return sh;
}

int64_t row_index_buckets(uint64_t entries, int shift) {
  return (int64_t)((entries + (uint64_t(1) << shift) - 1) >> shift);
}

void launch_row_index(const int64_t* ptr, int32_t ne, uint64_t entries, int32_t* first,
                      cudaStream_t s) {
  if (ne == 0) return;
  const int sh = row_index_shift(entries, ne);
  note_launch();
  k_row_index<<<grid_n(ne, 256), 256, 0, s>>>(ptr, ne, sh, row_index_buckets(entries, sh), first);
}

static RowIndex make_index(const int32_t* first, uint64_t entries, int32_t ne) {
  RowIndex ix{first, 0, 0};
  if (first) {
    ix.shift = row_index_shift(entries, ne);
    ix.buckets = row_index_buckets(entries, ix.shift);
  }
  return ix;
}

void launch_sample(const DevGraph& g, const int64_t* up_ptr, const int32_t* up_index,
                   const Oriented& up, int packed, uint64_t W, uint64_t seed, uint64_t first,
                   uint64_t num, unsigned long long* raw, unsigned long long* work, cudaStream_t s,
                   int nsm) {
  if (num == 0 || W == 0) return;
  uint64_t blocks = (num + kSampleWarps - 1) / kSampleWarps;
  if (blocks > (uint64_t)nsm * 16) blocks = (uint64_t)nsm * 16;
  note_launch();
  k_sample<<<(unsigned)blocks, kSampleWarps * 32, 0, s>>>(
      g, up_ptr, make_index(up_index, W, g.ne), up, packed, W, seed, first, num, raw, work);
}

void launch_type_counts(const int32_t* upc, const int32_t* wcr, int32_t ne, int32_t* cnt_t,
                        cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_type_counts<<<grid_n(ne, 256), 256, 0, s>>>(upc, wcr, ne, cnt_t);
}

void launch_split_types(const DevGraph& g, const int64_t* up_ptr, const Oriented& up, int packed,
                        const int64_t* t_ptr, const Oriented& t, const int64_t* c_ptr,
                        const Oriented& c, cudaStream_t s) {
  if (g.ne == 0) return;
  note_launch();
  k_split_types<<<grid_n(g.ne, 8), 256, 0, s>>>(g, up_ptr, up, packed, t_ptr, t, c_ptr, c);
}

void launch_sample_adv(const DevGraph& g, const int64_t* set_ptr, const int32_t* set_index,
                       const Oriented& set_ent, uint64_t Wx, int type, int cls, uint32_t stream,
                       const int64_t* full_ptr, const Oriented& full, int packed, uint64_t seed,
                       uint64_t first, uint64_t num, unsigned long long* raw, cudaStream_t s,
                       int nsm) {
  if (num == 0 || Wx == 0) return;
  AdvSet st{set_ptr, make_index(set_index, Wx, g.ne), set_ent, Wx, type, cls, stream};
  uint64_t blocks = (num + kSampleWarps - 1) / kSampleWarps;
  if (blocks > (uint64_t)nsm * 16) blocks = (uint64_t)nsm * 16;
  note_launch();
  k_sample_adv<<<(unsigned)blocks, kSampleWarps * 32, 0, s>>>(g, st, full_ptr, full, packed, seed,
                                                               first, num, raw);
}

void launch_priority(int32_t ne, uint64_t seed, unsigned long long* pr, cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_priority<<<grid_n(ne, 256), 256, 0, s>>>(ne, seed, pr);
}

void launch_digit_hist(const unsigned long long* pr, int32_t ne, int shift,
                       unsigned long long pmask, unsigned long long prefix, unsigned int* hist,
                       cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_digit_hist<<<grid_n(ne, 256), 256, 0, s>>>(pr, ne, shift, pmask, prefix, hist);
}

void launch_equal_flags(const unsigned long long* pr, int32_t ne, unsigned long long T,
                        int32_t* eq, cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_equal_flags<<<grid_n(ne, 256), 256, 0, s>>>(pr, ne, T, eq);
}

void launch_keep_flags(const unsigned long long* pr, int32_t ne, unsigned long long T,
                       const int64_t* eq_rank, int64_t need, int32_t* keep, cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_keep_flags<<<grid_n(ne, 256), 256, 0, s>>>(pr, ne, T, eq_rank, need, keep);
}

void launch_compact_kept(const int32_t* keep, const int64_t* pos, const int32_t* esize, int32_t ne,
                         int32_t* ids, int32_t* sizes, cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_compact_kept<<<grid_n(ne, 256), 256, 0, s>>>(keep, pos, esize, ne, ids, sizes);
}

void launch_gather_rows(const int64_t* e_ptr, const int32_t* e_idx, const int32_t* ids, int32_t nk,
                        const int64_t* sub_ptr, int32_t* sub_idx, cudaStream_t s) {
  if (nk == 0) return;
  note_launch();
  k_gather_rows<<<grid_n(nk, 8), 256, 0, s>>>(e_ptr, e_idx, ids, nk, sub_ptr, sub_idx);
}

void launch_enumerate(const DevGraph& g, const int64_t* up_ptr, const int32_t* up_index,
                      const Oriented& up, int packed, uint64_t W, int target, int32_t* out,
                      unsigned long long cap, unsigned long long* count, cudaStream_t s, int nsm) {
  if (W == 0) return;
  uint64_t blocks = (W + kSampleWarps - 1) / kSampleWarps;
  if (blocks > (uint64_t)nsm * 16) blocks = (uint64_t)nsm * 16;
  note_launch();
  k_enumerate<<<(unsigned)blocks, kSampleWarps * 32, 0, s>>>(
      g, up_ptr, make_index(up_index, W, g.ne), up, packed, W, target, out, cap, count);
}

}  // namespace hg
