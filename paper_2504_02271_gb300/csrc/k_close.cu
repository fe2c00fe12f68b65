// K3/K4/K5: hyper-triangle closure, classification and per-pattern reduction
// (step two of the two-step framework, Sec. 3.2-3.3).
//
// Every hyper-triangle {e_u, e_v, e_w} (Def. 2.4) is found exactly once, from
// its lowest-ranked hyperedge u in the degree order: v and w are both
// out-neighbours of u, and w is an out-neighbour of v.  The team that owns u
//   1. inserts out(u) into a two-table cuckoo set (key x -> its index k in out(u)),
//   2. records for every out-neighbour x the set Omega_ux = e_u cap e_x as a bit
//      mask over the positions of e_u (scanning E_y for each vertex y of e_u),
//   3. streams out(v) for every v in out(u) and looks each w up in the set.
// A hit is a hyper-triangle.  With m_uv, m_uw the masks, F the mask of all of e_u,
// omega_vw from the entry of out(v), r_x = |e_x| - omega_ux (the part of e_x outside
// e_u) and t = omega_vw - popc(m_uv & m_uw) (the part of e_v cap e_w outside e_u), the
// seven Venn regions of Sec. 2 are non-empty exactly when
//   (a) F & ~(m_uv | m_uw) != 0   (b) r_v > t   (c) r_w > t   (d) m_uv & ~m_uw != 0
//   (e) t > 0   (f) m_uw & ~m_uv != 0   (g) m_uv & m_uw != 0
// (inclusion-exclusion: b = |e_v| - omega_uv - omega_vw + g = r_v - t, and so on).
// The seven bits, labelled (u, v, w), index a block-local 128-bin histogram that is
// flushed to 64-bit global counters; the host folds the labelled masks into canonical
// masks and patterns.
#include <climits>
#include <mutex>

#include <cooperative_groups.h>
#include <type_traits>

#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBins = 128;     // labelled region masks (bit r = region r non-empty)
constexpr int kHistCopies = 4; // spread same-pattern increments of the block kernel
// Global-table teams: one block of kWideThreads per hyperedge, kWideBlocksPerSm blocks
// per SM; fewer, wider blocks keep fewer teams' tables in flight (they live in global
// memory, so the resident set decides the L2 hit rate).
#ifndef HG_WIDE_THREADS
#define HG_WIDE_THREADS 256
#endif
constexpr int kWideThreads = HG_WIDE_THREADS;
constexpr int kWideFilterLog2 = 18;   // 32 KiB shared filter per wide-team block
constexpr int kWideUnroll = 4;        // 32-entry loads in flight per warp
constexpr int kWideBlocksPerSm = 1024 / kWideThreads;

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

// Labelled region mask of the hyper-triangle (u, v, w) from one-word vertex masks (see
// the header): fu = all of e_u, muv/muw = Omega_uv/Omega_uw, rv/rw = |e_x| - omega_ux,
// om = omega_vw.
__device__ __forceinline__ uint32_t region_bits(uint32_t fu, uint32_t muv, uint32_t muw, int rv,
                                                int rw, int om) {
  const uint32_t i = muv & muw;
  const int t = om - __popc(i);
  return (uint32_t)((fu & ~(muv | muw)) != 0u) | ((uint32_t)(rv > t) << 1) |
         ((uint32_t)(rw > t) << 2) | ((uint32_t)((muv & ~muw) != 0u) << 3) |
         ((uint32_t)(t > 0) << 4) | ((uint32_t)((muw & ~muv) != 0u) << 5) |
         ((uint32_t)(i != 0u) << 6);
}

__device__ __forceinline__ uint32_t full_mask(int sz) { return sz >= 32 ? ~0u : (1u << sz) - 1u; }

// ------------------------------------------------------------------ warp per u
//
// One warp owns one hyperedge u with |e_u| <= 32 and out-degree <= D.  Shared
// memory per warp holds out(u) as a two-table cuckoo set: key x sits at slot
// h1(x) of table 1 or at slot h2(x) of table 2 (2D slots each, so at most a
// quarter of the slots are used), each slot packing x with its index k in out(u).
// A lookup is two shared loads, two xors and a min, the same on every lane: no
// probing loop, no divergence.  Keys that insertion could not place within
// kCuckooTries evictions go to a small stash that every lookup of the team also
// scans; a team whose stash overflows is handed to the global-table teams.
// Per-neighbour arrays hold the list base (row start minus the prefix of the list
// lengths), the prefix sums themselves, the Omega_ux mask and |e_x|.  The closure
// walks the concatenation of the out(v) lists as one flat range: lane l takes flat
// entries base + l + 32 q, so each load instruction reads 32 consecutive entries and
// every slot is full.  Hits are queued and classified 32 at a time, so the
// classification runs with every lane active.

// Entries of out(v) loaded per lane before their probes (loads in flight per warp):
// warp_unroll(D_LOG2) in the warp teams, kBlockUnroll in the block teams.  On the
// co-authorship workload the out-degree-128 teams were fastest with 6 (6.01 ms; 8: 6.13,
// 10: 6.09), the out-degree-64 and -256 ones with 10 (0.875 and 1.184 ms; 8: 0.885 and
// 1.198).  HG_CLOSE_WARP_UNROLL sets one value for all three.
#ifdef HG_CLOSE_WARP_UNROLL
__host__ __device__ constexpr int warp_unroll(int) { return HG_CLOSE_WARP_UNROLL; }
#else
__host__ __device__ constexpr int warp_unroll(int d_log2) { return d_log2 == 7 ? 6 : 10; }
#endif
// warps of a block team (one block per SM: shared memory holds one team's tables).  On
// the tag-shaped prefix of 500,000 hyperedges 16, 24 and 32 warps took 7.22, 5.73 and
// 5.16 s per step (the teams were latency-bound at 16 warps per SM).  The unpacked
// layout's hit queue is 4x wider, so it keeps to 24 warps (its out-degree-4096 tables
// with 32 warps would leave under 2 KB of the 227 KB a block may use).
#ifndef HG_BLOCK_WARPS
#define HG_BLOCK_WARPS 32
#endif
constexpr int kBlockWarps = HG_BLOCK_WARPS;
constexpr int kBlockWarpsUnpacked = HG_BLOCK_WARPS < 24 ? HG_BLOCK_WARPS : 24;
constexpr int kBlockUnroll = 8;
constexpr int kQueue = 32 * kBlockUnroll + 32;
constexpr int kCuckooTries = 16;
constexpr int kStash = 8;

// OFF32: the oriented rows hold fewer than 2^32 entries, so row starts fit 32 bits.  In
// the packed layout every |e| < 256, so sizes fit 8 bits.  The smaller per-warp state
// lets more warps share an SM.
template <int D_LOG2, bool PACKED, bool OFF32>
struct alignas(16) WarpTables {
  static constexpr int D = 1 << D_LOG2;      // max out-degree of u
  static constexpr int T_LOG2 = D_LOG2 + 1;  // slots per cuckoo table
  static constexpr int T = 1 << T_LOG2;
  static constexpr bool kPacked = PACKED;
  static_assert(D <= 256, "neighbour indices are packed in 8 bits");
  static constexpr int kUnroll = warp_unroll(D_LOG2);   // loads in flight per lane
  static constexpr int kQueue = 32 * kUnroll + 32;       // a round of hits plus a partial one
  // (x << 8) | k; all ones = empty.  Packed rows have x < 2^24.
  using Item = typename std::conditional<PACKED, uint32_t, unsigned long long>::type;
  using Off = typename std::conditional<OFF32, uint32_t, int64_t>::type;
  using Sz = typename std::conditional<PACKED, uint8_t, uint16_t>::type;
  Item c1[T];
  Item c2[T];
  Item stash[kStash];
  // entry f of the flat range of all out(x), x in out(u), lies at packed/nbr index
  // adj[k] + f for the out-neighbour k whose list holds f (the list's start in the rows
  // minus kpre[k]; modulo 2^32 when Off is 32-bit, which every true index fits)
  Off adj[D];
  int32_t kpre[D + 1];                       // exclusive prefix of the out-degrees of out(u)
  uint32_t kmask[D];                         // Omega_ux of the k-th out-neighbour x
  Sz ksz[D];                                 // |e_x|, then |e_x| - omega_ux once masks are built
  uint32_t queue[kQueue];                    // hits: (k_v << 24) | (k_w << 8) | omega_vw
  int32_t qom[PACKED ? 1 : kQueue];          // omega_vw when it may not fit 8 bits
  int32_t nstash;
};

__device__ __forceinline__ uint32_t cuckoo_h1(uint32_t key, int t_log2) {
  return (key * 0x9E3779B1u) >> (32 - t_log2);
}
__device__ __forceinline__ uint32_t cuckoo_h2(uint32_t key, int t_log2) {
  return (key * 0x85EBCA6Bu) >> (32 - t_log2);
}

// Index k in out(u) of hyperedge x, or -1.  Branch-free but for the stash scan,
// whose length nst is the same on every lane of the warp.  An item (x << 8) | k
// xor-ed with x << 8 leaves exactly k (< 256) when the keys agree, and a value of
// at least 256 otherwise.  The empty item (all ones) would answer 255 to a key whose
// low 24 bits are all ones; no hyperedge id of a packed layout (< 2^24 - 1) has
// them, and lanes without an entry look up u itself, which is never in out(u).
// A key sits in at most one place, so the smaller of the xor-ed items is k on a hit and
// at least 256 otherwise: one min and one compare decide it.
template <class TT, bool STASH = true>
__device__ __forceinline__ int warp_find(const TT& t, int32_t x, int nst) {
  using Item = typename TT::Item;
  const uint32_t key = (uint32_t)x;
  const Item k8 = (Item)key << 8;
  const Item a = t.c1[cuckoo_h1(key, TT::T_LOG2)] ^ k8;
  const Item b = t.c2[cuckoo_h2(key, TT::T_LOG2)] ^ k8;
  Item m = a < b ? a : b;
  if (STASH) {
    for (int i = 0; i < nst; ++i) {
      const Item c = t.stash[i] ^ k8;
      m = c < m ? c : m;
    }
  }
  return m < 256 ? (int)m : -1;
}

// Start of out(x)'s entries in the oriented rows: a pointer per layout, so that a probe
// addresses entry j of the current row with one 32-bit index.
template <bool PACKED>
struct RowPtr {
  const uint32_t* p;   // packed entries
  const int32_t* n;    // unpacked: neighbour ids
  const int32_t* w;    // unpacked: omega
  __device__ __forceinline__ void at(const Oriented& o, int64_t off) {
    if (PACKED) {
      p = o.packed + off;
    } else {
      n = o.nbr + off;
      w = o.omega + off;
    }
  }
  __device__ __forceinline__ void load(int32_t j, int32_t& nbr, int32_t& om) const {
    if (PACKED) {
      const uint32_t x = __ldg(p + j);
      nbr = (int32_t)(x >> 8);
      om = (int32_t)(x & 0xffu);
    } else {
      nbr = __ldg(n + j);
      om = __ldg(w + j);
    }
  }
  // packed layout only: the entry as stored, (nbr << 8) | omega
  __device__ __forceinline__ uint32_t raw(int32_t j) const { return __ldg(p + j); }
};

__device__ __forceinline__ uint32_t filt_bit(uint32_t key, int bits_log2) {
  return (key * 0x85EBCA6Bu) >> (32 - bits_log2);
}

// Per-lane run-length accumulation of pattern increments (most lanes repeat the
// same pattern many times): one shared atomic per run instead of per triangle.
struct RunHist {
  uint32_t pat = 0, run = 0;
  __device__ __forceinline__ void add(uint32_t p, uint32_t* hist) {
    if (p == pat && run < 0x7fffffffu) {
      ++run;
    } else {
      if (run) atomicAdd(&hist[pat], run);
      pat = p;
      run = 1;
    }
  }
  __device__ __forceinline__ void flush(uint32_t* hist) {
    if (run) atomicAdd(&hist[pat], run);
    run = 0;
  }
};

// Move a warp's shared bins (after its lanes' runs) into the global bins `out`.
__device__ __forceinline__ void warp_flush(RunHist& rh, uint32_t* hist,
                                           unsigned long long* __restrict__ out, int lane) {
  rh.flush(hist);
  __syncwarp();
  for (int k = lane; k < kBins; k += 32) {
    const uint32_t x = hist[k];
    if (x) {
      atomicAdd(&out[k], (unsigned long long)x);
      hist[k] = 0;
    }
  }
  __syncwarp();
}

// Classify queued hit number `at`: v and w are out-neighbours number kv and kw of u.
template <class TT>
__device__ __forceinline__ void classify_queued(const TT& t, int at, uint32_t fu, uint32_t* hist,
                                                RunHist& rh) {
  const uint32_t e = t.queue[at];
  const uint32_t kv = e >> 24, kw = (e >> 8) & 0xffu;
  const int om = TT::kPacked ? (int)(e & 0xffu) : t.qom[at];
  rh.add(region_bits(fu, t.kmask[kv], t.kmask[kw], t.ksz[kv], t.ksz[kw], om), hist);
}

// Step 3 of a warp team: the flat range of all out(v), v in out(u) (F entries), 32
// consecutive entries per window, lane l taking entry f0 + l.  The window's lists are
// found by a warp-uniform cursor over the prefix sums kpre: the lanes start in the list
// that holds f0, and every list that starts inside the window moves the lanes at or past
// its start over to it (predicated, no divergent branch).  TT::kUnroll windows are
// loaded before their probes; hits are queued and classified 32 at a time.  STASH =
// false when the team's stash is empty (the usual case): the probes then skip the stash
// scan altogether.
template <class TT, bool STASH>
__device__ __forceinline__ void warp_walk(TT& t, const Oriented& o, int32_t u, int32_t du,
                                          int32_t F, int nst, uint32_t fu, uint32_t* hist,
                                          RunHist& rh, int lane) {
  constexpr bool PACKED = TT::kPacked;
  constexpr int kWarpUnroll = TT::kUnroll;
  using Off = typename TT::Off;
  int qn = 0;   // queued hits (the same on every lane)
  // uniform cursor: list wk starts at or before the next window; wnext = kpre[wk + 1]
  int wk = 0;
  int32_t wnext = t.kpre[1];
  Off wadj = t.adj[0];
  for (int32_t base = 0; base < F; base += 32 * kWarpUnroll) {
    // packed: the raw entry (w << 8) | omega_vw in one register; no entry: u << 8
    // (u is never in out(u)).  Unpacked: w and omega_vw apart.
    int32_t ent_w[kWarpUnroll], ent_om[PACKED ? 1 : kWarpUnroll], ent_k[kWarpUnroll];
#pragma unroll
    for (int q = 0; q < kWarpUnroll; ++q) {
      const int32_t f0 = base + 32 * q, f = f0 + lane;
      const int32_t wend = f0 + 32 < F ? f0 + 32 : F;
      Off my_adj = wadj;
      int my_k = wk;
      while (wnext < wend) {   // uniform: list wk + 1 starts inside this window
        ++wk;                  // (wk + 1 < du: wnext < F = kpre[du])
        wadj = t.adj[wk];
        if (f >= wnext) {
          my_adj = wadj;
          my_k = wk;
        }
        wnext = t.kpre[wk + 1];
      }
      ent_k[q] = my_k;
      const Off at = my_adj + (Off)f;
      if (PACKED) {
        ent_w[q] = (int32_t)((uint32_t)u << 8);
        if (f < F) ent_w[q] = (int32_t)__ldg(o.packed + at);
      } else {
        ent_w[q] = u;
        ent_om[q] = 0;
        if (f < F) {
          ent_w[q] = __ldg(o.nbr + at);
          ent_om[q] = __ldg(o.omega + at);
        }
      }
    }
    // probe; hits go to the warp's queue as (index of v, index of w, omega_vw)
#pragma unroll
    for (int q = 0; q < kWarpUnroll; ++q) {
      const int32_t x = PACKED ? (int32_t)((uint32_t)ent_w[q] >> 8) : ent_w[q];
      const int kw = warp_find<TT, STASH>(t, x, nst);
      const bool hit = kw >= 0;
      const unsigned bal = __ballot_sync(kFull, hit);
      if (hit) {
        const int at = qn + __popc(bal & ((1u << lane) - 1u));
        t.queue[at] = ((uint32_t)ent_k[q] << 24) | ((uint32_t)kw << 8) |
                      (PACKED ? ((uint32_t)ent_w[q] & 0xffu) : 0u);
        if (!PACKED) t.qom[at] = ent_om[PACKED ? 0 : q];
      }
      qn += __popc(bal);
    }
    __syncwarp();
    // classify full rounds of 32 hits with every lane busy
    while (qn >= 32) {
      qn -= 32;
      classify_queued(t, qn + lane, fu, hist, rh);
      __syncwarp();
    }
  }
  if (lane < qn) classify_queued(t, lane, fu, hist, rh);
  __syncwarp();
}

// Threads of warp teams resident per SM that the register allocation aims at: 1,280 for
// the out-degree-128 teams (six 6-warp blocks at 56 registers: 7.58 -> 7.33 ms on the
// co-authorship workload), 1,024 for the others (at 1,280 the out-degree-256 teams
// spill and slow down, 1.46 -> 1.55 ms).
#ifndef HG_WARP128_THREADS_PER_SM
#define HG_WARP128_THREADS_PER_SM 1280
#endif
__host__ __device__ constexpr int warp_threads_per_sm(int d_log2) {
  return d_log2 == 7 ? HG_WARP128_THREADS_PER_SM : 1024;
}

template <int D_LOG2, int WARPS, bool PACKED, bool OFF32>
__global__ void __launch_bounds__(WARPS * 32, warp_threads_per_sm(D_LOG2) / (WARPS * 32))
    k_close_warp(DevGraph g, Oriented o, const int32_t* __restrict__ list,
                 const int32_t* __restrict__ n_p, unsigned long long* __restrict__ hist_out,
                 unsigned long long* __restrict__ work, int32_t* __restrict__ counter,
                 int32_t* __restrict__ overflow, int32_t* __restrict__ n_overflow, int handover) {
  using TT = WarpTables<D_LOG2, PACKED, OFF32>;
  using Item = typename TT::Item;
  constexpr int T = TT::T, T_LOG2 = TT::T_LOG2;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  TT* tabs = reinterpret_cast<TT*>(dyn_smem);   // WARPS tables
  __shared__ uint32_t hist[WARPS][kBins];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  TT& t = tabs[w];
  for (int k = lane; k < kBins; k += 32) hist[w][k] = 0;
  __syncthreads();
  const int32_t n = *n_p;
  RunHist rh;
  unsigned long long probes = 0, gathers = 0, outs = 0, since_flush = 0;
  int32_t cur = 0;   // member whose bins the shared histogram holds

  while (true) {
    int r = 0;
    if (lane == 0) r = atomicAdd(counter, 1);
    r = __shfl_sync(kFull, r, 0);
    if (r >= n) break;
    const int32_t u = list[r];
    const int32_t m = member_of(g, u);
    if (m != cur || since_flush > (1ull << 30)) {   // 32-bit bins stay far from overflow
      warp_flush(rh, hist[w], hist_out + (size_t)cur * kBins, lane);
      cur = m;
      since_flush = 0;
    }
    const int32_t du = o.dplus[u];
    const int64_t bu = o.row_ptr[u];
    const int64_t eb = g.e_ptr[u];
    const int32_t szu = (int32_t)(g.e_ptr[u + 1] - eb);

    {   // both cuckoo tables to empty, 16 bytes per store
      uint4* c = reinterpret_cast<uint4*>(t.c1);
      constexpr int kVec = (int)(2 * T * sizeof(Item) / 16);
      for (int s = lane; s < kVec; s += 32) c[s] = make_uint4(~0u, ~0u, ~0u, ~0u);
    }
    if (lane == 0) t.nstash = 0;
    // vertex y of e_u at lane p: its E_y range (one round trip for all p)
    int64_t yb = 0, ye = 0;
    if (lane < szu) {
      const int32_t y = __ldg(g.e_idx + eb + lane);
      yb = __ldg(g.v_ptr + y);
      ye = __ldg(g.v_ptr + y + 1);
    }
    __syncwarp();
    // 1. out(u) into the cuckoo set
    for (int k = lane; k < du; k += 32) {
      int32_t x, om;
      get_entry<PACKED>(o, bu + k, x, om);
      const int64_t xb = __ldg(o.row_ptr + x);
      const int32_t xc = __ldg(o.dplus + x);
      const int32_t xs = __ldg(g.esize + x);
      Item it = ((Item)(uint32_t)x << 8) | (Item)k;
      bool second = false;   // the table the item in hand goes to next
      for (int tries = 0; tries < kCuckooTries; ++tries) {
        const uint32_t key = (uint32_t)(it >> 8);
        Item* slot = second ? &t.c2[cuckoo_h2(key, T_LOG2)] : &t.c1[cuckoo_h1(key, T_LOG2)];
        it = atomicExch(slot, it);
        if (it == ~(Item)0) break;
        second = !second;   // the evicted item sat at its own slot of this table
      }
      if (it != ~(Item)0) {
        const int at = atomicAdd(&t.nstash, 1);
        if (at < kStash) t.stash[at] = it;
      }
      t.kmask[k] = 0;
      t.ksz[k] = (typename TT::Sz)xs;
      t.adj[k] = (typename TT::Off)xb;   // the list start until the prefix sums exist
      t.kpre[k + 1] = xc;                 // the out-degree until the prefix sums exist
    }
    __syncwarp();
    const int nst = *((volatile int32_t*)&t.nstash);
    if (nst > kStash || handover) {   // warp-uniform: the global-table teams take u
      if (lane == 0) overflow[atomicAdd(n_overflow, 1)] = u;
      __syncwarp();
      continue;
    }
    // 2. Omega_ux masks: flat walk over the E_y lists of the vertices of e_u (fewer
    // than 2^30 entries in all: the build refuses larger rows, so the prefix sums are
    // 32-bit; each lane keeps the 64-bit start of its list minus its exclusive prefix)
    {
      const int32_t len = (int32_t)(ye - yb);   // lanes >= szu hold 0
      int32_t incl = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t o2 = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += o2;
      }
      const int64_t ybase = yb - (incl - len);   // flat position f of this list: v_idx[ybase + f]
      const int32_t total = __shfl_sync(kFull, incl, 31);
      gathers += (unsigned long long)total;
      for (int32_t f0 = 0; f0 < total; f0 += 32) {   // warp-uniform: all lanes shuffle
        const int32_t f = f0 + lane;
        int lo = 0, hi = 31;   // owner p: first lane whose inclusive prefix exceeds f
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const int mid = (lo + hi) >> 1;
          if (__shfl_sync(kFull, incl, mid) > f) hi = mid; else lo = mid + 1;
        }
        const int p = lo;
        const int64_t start = __shfl_sync(kFull, ybase, p);
        if (f >= total) continue;
        const int32_t x = __ldg(g.v_idx + start + f);
        const int kx = warp_find(t, x, nst);
        if (kx >= 0) atomicOr(&t.kmask[kx], 1u << p);   // lanes may be at different p
      }
    }
    // out-degrees -> their exclusive prefix kpre, list starts -> adj = start - kpre (each
    // lane reads and rewrites only its own k)
    int32_t F = 0;
    for (int k0 = 0; k0 < du; k0 += 32) {   // warp-uniform
      const int k = k0 + lane;
      const int32_t c = k < du ? t.kpre[k + 1] : 0;
      int32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t o2 = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += o2;
      }
      if (k < du) {
        t.kpre[k + 1] = F + incl;
        t.adj[k] -= (typename TT::Off)(F + incl - c);
      }
      F += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) t.kpre[0] = 0;
    probes += (unsigned long long)F;
    since_flush += (unsigned long long)F;
    outs += (unsigned long long)du;
    __syncwarp();
    // |e_x| -> |e_x| - omega_ux, the part of e_x outside e_u
    for (int k = lane; k < du; k += 32)
      t.ksz[k] = (typename TT::Sz)(t.ksz[k] - __popc(t.kmask[k]));
    const uint32_t fu = full_mask(szu);
    __syncwarp();

    // 3. closure over the flat range of all out(v), v in out(u)
    if (nst == 0) warp_walk<TT, false>(t, o, u, du, F, nst, fu, hist[w], rh, lane);
    else warp_walk<TT, true>(t, o, u, du, F, nst, fu, hist[w], rh, lane);
  }
  warp_flush(rh, hist[w], hist_out + (size_t)cur * kBins, lane);
  if (lane == 0) {
    atomicAdd(&work[0], probes);
    atomicAdd(&work[1], gathers);
    atomicAdd(&work[2], outs);
  }
}

// ------------------------------------------------------------------ block per u (shared tables)
//
// One block owns one hyperedge u with |e_u| <= 32 and out-degree <= D.  out(u)
// is a two-table cuckoo set with 2D slots per table.  A slot stores a key by
// quotient: with the odd multiplier A of its table, p = x A mod 2^32 is a
// bijection of x, the top T_LOG2 bits of p are the slot and the remaining
// 31 - D_LOG2 bits are stored beside the index k of x in out(u), so 31 bits
// identify (x, k) exactly and the top bit marks an empty slot.  An evicted key
// is recovered from its slot and remainder with the inverse of A.  Keys not
// placed within kCuckooTries evictions go to a stash; a team whose stash
// overflows is handed to the global-table teams.  Per-k arrays hold the Omega_ux
// mask, |e_x|, and the place and prefix-summed length of out(x).  The flat range
// of all out(v) entries is cut into WARPS slices of equal length; each warp walks
// its slice like the warp kernel (32 consecutive entries per load, lookup, queue,
// 32-wide classification).

constexpr uint32_t kCuckooA1 = 0x9E3779B1u, kCuckooA1Inv = 0x0E8B2F51u;
constexpr uint32_t kCuckooA2 = 0x85EBCA6Bu, kCuckooA2Inv = 0xA5CB9243u;
static_assert(kCuckooA1 * kCuckooA1Inv == 1u && kCuckooA2 * kCuckooA2Inv == 1u,
              "multiplicative inverses mod 2^32");

// DMAX below 2^D_LOG2 (the 6,144 shape): indices keep D_LOG2 bits, each table has
// 2^D_LOG2 slots (at most 3/8 of both tables in use), and a slot's remainder and index
// fill all 32 bits; the empty word (all ones) still matches no key, because its index
// field (all ones) is at least DMAX.
template <int D_LOG2, int WARPS, bool PACKED, int DMAX = (1 << D_LOG2)>
struct alignas(16) BlockTables {
  static constexpr int D = DMAX;
  static constexpr int T_LOG2 = DMAX == (1 << D_LOG2) ? D_LOG2 + 1 : D_LOG2;
  static constexpr int T = 1 << T_LOG2;
  static_assert(DMAX == (1 << D_LOG2) || (DMAX < (1 << D_LOG2) && 4 * DMAX <= 3 * (1 << D_LOG2)),
                "a smaller DMAX keeps the tables at most 3/8 full");
  uint32_t c1[T];
  uint32_t c2[T];
  int32_t skey[kStash];
  int32_t sidx[kStash];
  int64_t kbeg[D];
  int32_t kpre[D + 1];       // exclusive prefix of the out-degrees of out(u)
  uint32_t kmask[D];
  uint16_t ksz[D];           // |e_x|, then |e_x| - omega_ux once masks are built
  uint32_t queue[WARPS][kQueue];   // hits: (k_v << 16) | k_w ; omega in qom
  uint8_t qom8[PACKED ? WARPS : 1][PACKED ? kQueue : 1];
  int32_t qom[PACKED ? 1 : WARPS][PACKED ? 1 : kQueue];
  int64_t ylen[32], yincl[32], ybeg[32];
  int32_t nstash;
};

// Index k in out(u) of hyperedge x, or -1 (x = -1 matches nothing: keys are < 2^31).
template <int D_LOG2, int WARPS, bool PACKED, int DMAX, bool STASH = true>
__device__ __forceinline__ int block_find(const BlockTables<D_LOG2, WARPS, PACKED, DMAX>& t,
                                          int32_t x, int nst) {
  constexpr int SH = 32 - BlockTables<D_LOG2, WARPS, PACKED, DMAX>::T_LOG2;   // remainder bits
  constexpr uint32_t RM = (1u << SH) - 1u;
  const uint32_t p1 = (uint32_t)x * kCuckooA1, p2 = (uint32_t)x * kCuckooA2;
  // an item (remainder << D_LOG2) | k xor-ed with the key's remainder so shifted is k
  // (< DMAX) when the remainders agree, and at least 2^D_LOG2 otherwise; an empty slot
  // gives at least DMAX (the top bit, or an index field of all ones); a key sits in at
  // most one table
  const uint32_t a = t.c1[p1 >> SH] ^ ((p1 & RM) << D_LOG2);
  const uint32_t b = t.c2[p2 >> SH] ^ ((p2 & RM) << D_LOG2);
  const uint32_t m = a < b ? a : b;
  int k = m < (uint32_t)DMAX ? (int)m : -1;
  if (STASH)
    for (int i = 0; i < nst; ++i) k = t.skey[i] == x ? t.sidx[i] : k;
  return k;
}

// Step 3 of a block team, for warp w: the slice [f_lo, f_hi) of the flat range of all
// out(v), v in out(u), walked like the warp teams' (kBlockUnroll loads in flight, a
// cursor per lane, queued 32-wide classification); the slice start is found by a
// binary search over the prefix sums kpre of the out-degrees.
template <int D_LOG2, int WARPS, bool PACKED, int DMAX, bool STASH>
__device__ __forceinline__ void block_walk(BlockTables<D_LOG2, WARPS, PACKED, DMAX>& t,
                                           const Oriented& o, int32_t u, int32_t du,
                                           int32_t f_lo, int32_t f_hi, int nst, uint32_t fu,
                                           uint32_t* hist, RunHist& rh, int lane, int w) {
  int qn = 0;
  uint32_t* queue = t.queue[w];
  // cursor of this lane: first entry f_lo + lane -> (ck, cj); past the slice: ck = du
  int ck = du, cj = 0, ccnt = INT32_MAX;
  RowPtr<PACKED> rp;
  rp.at(o, 0);
  {
    const int32_t f0 = f_lo + lane;
    int lo = 0, hi = du;   // last k with kpre[k] <= f0
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (t.kpre[mid] <= f0) lo = mid; else hi = mid - 1;
    }
    if (f0 < f_hi && lo < du) {
      ck = lo;
      cj = f0 - t.kpre[ck];
      ccnt = t.kpre[ck + 1] - t.kpre[ck];
      rp.at(o, t.kbeg[ck]);
    }
  }
  for (int32_t base = f_lo; base < f_hi; base += 32 * kBlockUnroll) {
    int32_t ent_w[kBlockUnroll], ent_om[PACKED ? 1 : kBlockUnroll], ent_k[kBlockUnroll];
#pragma unroll
    for (int q = 0; q < kBlockUnroll; ++q) {
      ent_k[q] = ck;
      const bool in = ck < du && base + q * 32 + lane < f_hi;
      if (PACKED) {
        ent_w[q] = (int32_t)((uint32_t)u << 8);   // no entry: u, never in out(u)
        if (in) ent_w[q] = (int32_t)rp.raw(cj);
      } else {
        ent_w[q] = u;
        ent_om[q] = 0;
        if (in) rp.load(cj, ent_w[q], ent_om[q]);
      }
      cj += 32;
      if (cj >= ccnt) {
        do {
          cj -= ccnt;
          ++ck;
          ccnt = ck < du ? t.kpre[ck + 1] - t.kpre[ck] : INT32_MAX;
        } while (cj >= ccnt);
        if (ck < du) rp.at(o, t.kbeg[ck]);
      }
    }
#pragma unroll
    for (int q = 0; q < kBlockUnroll; ++q) {
      const int32_t x = PACKED ? (int32_t)((uint32_t)ent_w[q] >> 8) : ent_w[q];
      const int kw = block_find<D_LOG2, WARPS, PACKED, DMAX, STASH>(t, x, nst);
      const bool hit = kw >= 0;
      const unsigned bal = __ballot_sync(kFull, hit);
      if (hit) {
        const int at = qn + __popc(bal & ((1u << lane) - 1u));
        queue[at] = ((uint32_t)ent_k[q] << 16) | (uint32_t)kw;
        if (PACKED) t.qom8[w][at] = (uint8_t)((uint32_t)ent_w[q] & 0xffu);
        else t.qom[w][at] = ent_om[PACKED ? 0 : q];
      }
      qn += __popc(bal);
    }
    __syncwarp();
    while (qn >= 32) {
      qn -= 32;
      const int at = qn + lane;
      const uint32_t e = queue[at];
      const uint32_t kv = e >> 16, kw = e & 0xffffu;
      const int om = PACKED ? (int)t.qom8[w][at] : t.qom[w][at];
      rh.add(region_bits(fu, t.kmask[kv], t.kmask[kw], t.ksz[kv], t.ksz[kw], om), hist);
      __syncwarp();
    }
  }
  if (lane < qn) {
    const uint32_t e = queue[lane];
    const uint32_t kv = e >> 16, kw = e & 0xffffu;
    const int om = PACKED ? (int)t.qom8[w][lane] : t.qom[w][lane];
    rh.add(region_bits(fu, t.kmask[kv], t.kmask[kw], t.ksz[kv], t.ksz[kw], om), hist);
  }
  __syncwarp();
}

template <int D_LOG2, int WARPS, bool PACKED, int DMAX>
__global__ void __launch_bounds__(WARPS * 32, 1)
    k_close_block(DevGraph g, Oriented o, const int32_t* __restrict__ list,
                  const int32_t* __restrict__ n_p, unsigned long long* __restrict__ hist_out,
                  unsigned long long* __restrict__ work, int32_t* __restrict__ counter,
                  int32_t* __restrict__ overflow, int32_t* __restrict__ n_overflow, int handover) {
  using TT = BlockTables<D_LOG2, WARPS, PACKED, DMAX>;
  // shared pattern bins: one set per warp, or 8 sets shared by the warps when the tables
  // leave no room for more (the 6,144 shape)
  constexpr int HC = DMAX == (1 << D_LOG2) ? WARPS : 8;
  constexpr int T = TT::T, SH = 32 - TT::T_LOG2;
  constexpr uint32_t RM = (1u << SH) - 1u, KM = (1u << D_LOG2) - 1u;
  constexpr int NT = WARPS * 32;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  TT& t = *reinterpret_cast<TT*>(dyn_smem);
  __shared__ uint32_t hist[HC][kBins];
  __shared__ int32_t s_r;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < HC * kBins; k += NT) (&hist[0][0])[k] = 0;
  const int32_t n = *n_p;
  RunHist rh;
  unsigned long long probes = 0, gathers = 0, outs = 0, since_flush = 0;
  int32_t cur = 0;   // member whose bins the shared histograms hold
  auto block_flush = [&]() {
    rh.flush(hist[w % HC]);
    __syncthreads();
    for (int k = threadIdx.x; k < kBins; k += NT) {
      unsigned long long x = 0;
      for (int ww = 0; ww < HC; ++ww) {
        x += hist[ww][k];
        hist[ww][k] = 0;
      }
      if (x) atomicAdd(&hist_out[(size_t)cur * kBins + k], x);
    }
    __syncthreads();
  };

  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_r = atomicAdd(counter, 1);
    __syncthreads();
    const int32_t r = s_r;
    if (r >= n) break;
    const int32_t u = list[r];
    const int32_t m = member_of(g, u);   // the same on every thread
    if (m != cur || since_flush > (1ull << 30)) {   // 32-bit bins stay far from overflow
      block_flush();
      cur = m;
      since_flush = 0;
    }
    const int32_t du = o.dplus[u];
    const int64_t bu = o.row_ptr[u];
    const int64_t eb = g.e_ptr[u];
    const int32_t szu = (int32_t)(g.e_ptr[u + 1] - eb);
    {   // both cuckoo tables to empty, 16 bytes per store
      uint4* c = reinterpret_cast<uint4*>(t.c1);
      for (int s = threadIdx.x; s < 2 * T / 4; s += NT) c[s] = make_uint4(~0u, ~0u, ~0u, ~0u);
    }
    if (threadIdx.x == 0) t.nstash = 0;
    if (w == 0) {   // E_y ranges of the vertices of e_u and their prefix sums
      int64_t yb = 0, len = 0;
      if (lane < szu) {
        const int32_t y = __ldg(g.e_idx + eb + lane);
        yb = __ldg(g.v_ptr + y);
        len = __ldg(g.v_ptr + y + 1) - yb;
      }
      int64_t incl = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int64_t o2 = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += o2;
      }
      t.ylen[lane] = len;
      t.yincl[lane] = incl;
      t.ybeg[lane] = yb;
    }
    __syncthreads();
    // 1. out(u) into the cuckoo set; out-degrees into kpre[k + 1] for the prefix sum
    for (int k = threadIdx.x; k < du; k += NT) {
      int32_t x, om;
      get_entry<PACKED>(o, bu + k, x, om);
      uint32_t key = (uint32_t)x, kk = (uint32_t)k;
      bool second = false, placed = false;
      for (int tries = 0; tries < kCuckooTries; ++tries) {
        const uint32_t pa = key * (second ? kCuckooA2 : kCuckooA1);
        const uint32_t slot = pa >> SH;
        uint32_t* c = second ? t.c2 : t.c1;
        const uint32_t e = atomicExch(&c[slot], ((pa & RM) << D_LOG2) | kk);
        if (e == ~0u) {
          placed = true;
          break;
        }
        // the evicted key sat at `slot` of this table: rebuild it from slot and remainder
        key = ((slot << SH) | (e >> D_LOG2)) * (second ? kCuckooA2Inv : kCuckooA1Inv);
        kk = e & KM;
        second = !second;
      }
      if (!placed) {
        const int at = atomicAdd(&t.nstash, 1);
        if (at < kStash) {
          t.skey[at] = (int32_t)key;
          t.sidx[at] = (int32_t)kk;
        }
      }
      t.kbeg[k] = __ldg(o.row_ptr + x);
      t.kpre[k + 1] = __ldg(o.dplus + x);
      t.ksz[k] = (uint16_t)__ldg(g.esize + x);
      t.kmask[k] = 0;
    }
    __syncthreads();
    const int nst = t.nstash;   // read after a barrier: uniform
    if (nst > kStash || handover) {   // the global-table teams take u
      if (threadIdx.x == 0) overflow[atomicAdd(n_overflow, 1)] = u;
      continue;
    }
    // 2. Omega_ux masks over the flat E_y range; prefix of the out-degrees (warp 0)
    {
      const int64_t total = t.yincl[31];
      if (threadIdx.x == 0) gathers += (unsigned long long)total;
      for (int64_t f = threadIdx.x; f < total; f += NT) {
        int lo = 0, hi = 31;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (t.yincl[mid] > f) hi = mid; else lo = mid + 1;
        }
        const int p = lo;
        const int32_t x = __ldg(g.v_idx + t.ybeg[p] + (f - (t.yincl[p] - t.ylen[p])));
        const int k = block_find(t, x, nst);
        if (k >= 0) atomicOr(&t.kmask[k], 1u << p);
      }
    }
    if (w == 0) {   // in place: kpre[k + 1] holds the out-degree of out-neighbour k
      int32_t run = 0;
      for (int k0 = 0; k0 < du; k0 += 32) {
        const int k = k0 + lane;
        const int32_t c = k < du ? t.kpre[k + 1] : 0;
        int32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int32_t o2 = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += o2;
        }
        if (k < du) t.kpre[k + 1] = run + incl;
        run += __shfl_sync(kFull, incl, 31);
      }
      if (lane == 0) t.kpre[0] = 0;
    }
    __syncthreads();
    // |e_x| -> |e_x| - omega_ux, the part of e_x outside e_u
    for (int k = threadIdx.x; k < du; k += NT) t.ksz[k] = (uint16_t)(t.ksz[k] - __popc(t.kmask[k]));
    __syncthreads();
    const uint32_t fu = full_mask(szu);
    const int32_t F = t.kpre[du];
    since_flush += (unsigned long long)F;   // the same on every thread
    if (threadIdx.x == 0) {
      probes += (unsigned long long)F;
      outs += (unsigned long long)du;
    }
    // 3. closure: warp w walks the flat slice [F*w/WARPS, F*(w+1)/WARPS)
    const int32_t f_lo = (int32_t)((int64_t)F * w / WARPS), f_hi = (int32_t)((int64_t)F * (w + 1) / WARPS);
    if (nst == 0)
      block_walk<D_LOG2, WARPS, PACKED, DMAX, false>(t, o, u, du, f_lo, f_hi, nst, fu, hist[w % HC],
                                                     rh, lane, w);
    else
      block_walk<D_LOG2, WARPS, PACKED, DMAX, true>(t, o, u, du, f_lo, f_hi, nst, fu, hist[w % HC],
                                                    rh, lane, w);
  }
  block_flush();
  if (threadIdx.x == 0) {
    atomicAdd(&work[0], probes);
    atomicAdd(&work[1], gathers);
    atomicAdd(&work[2], outs);
  }
}

// ------------------------------------------------------------------ block per u (wide)
// Any |e_u| (masks of `words` 32-bit words) and any out-degree; tables in global scratch.

// Per block: out(u) as a two-table cuckoo set coded by quotient like the block teams'
// (2^(dl+1) slots per table for du <= 2^dl), a stash with room for every key (these
// teams hand nothing over), and per out-neighbour arrays (Omega_ux of `words` words,
// |e_x|, list length and start).  Only the slots and the du rows of masks in use are
// cleared per u.
struct WideScratch {
  uint32_t* c1;     // [cap]
  uint32_t* c2;     // [cap]
  uint32_t* mask;   // [dmax * words]
  int32_t* ksz;     // [dmax] |e_x|, then |e_x| - omega_ux once masks are built
  int32_t* kcnt;    // [dmax]
  int64_t* kbeg;    // [dmax]
  int32_t* skey;    // [dmax]
  int32_t* sidx;    // [dmax]
  int32_t* nstash;  // [1] stash length (cluster teams: shared by the cluster's blocks)
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline size_t wide_block_bytes(int64_t cap, int64_t words, int64_t dmax) {
  return align256(cap * 4) * 2 + align256(dmax * words * 4) + align256(dmax * 4) * 4 +
         align256(dmax * 8) + 256;
}

__device__ WideScratch wide_carve(char* base, int64_t cap, int64_t words, int64_t dmax) {
  WideScratch w;
  w.c1 = (uint32_t*)base;
  base += align256(cap * 4);
  w.c2 = (uint32_t*)base;
  base += align256(cap * 4);
  w.mask = (uint32_t*)base;
  base += align256(dmax * words * 4);
  w.ksz = (int32_t*)base;
  base += align256(dmax * 4);
  w.kcnt = (int32_t*)base;
  base += align256(dmax * 4);
  w.kbeg = (int64_t*)base;
  base += align256(dmax * 8);
  w.skey = (int32_t*)base;
  base += align256(dmax * 4);
  w.sidx = (int32_t*)base;
  base += align256(dmax * 4);
  w.nstash = (int32_t*)base;
  return w;
}

// Index k in out(u) of hyperedge x in the tables of a team with du <= 2^dl, or -1.
__device__ __forceinline__ int wide_find(const WideScratch& t, int32_t x, int dl, int nst) {
  const int sh = 31 - dl;
  const uint32_t rm = (1u << sh) - 1u, km = (1u << dl) - 1u;
  const uint32_t p1 = (uint32_t)x * kCuckooA1, p2 = (uint32_t)x * kCuckooA2;
  const uint32_t a = t.c1[p1 >> sh], b = t.c2[p2 >> sh];
  int k = (a >> dl) == (p1 & rm) ? (int)(a & km) : -1;
  k = (b >> dl) == (p2 & rm) ? (int)(b & km) : k;
  for (int i = 0; i < nst; ++i) k = t.skey[i] == x ? t.sidx[i] : k;
  return k;
}

template <bool PACKED>
__global__ void __launch_bounds__(kWideThreads, kWideBlocksPerSm)
    k_close_wide(DevGraph g, Oriented o, const int32_t* __restrict__ list,
                 const int32_t* __restrict__ n_p, int64_t cap_max, int64_t words_max,
                 int64_t dmax, char* __restrict__ scratch, unsigned long long* __restrict__ hist_out,
                 unsigned long long* __restrict__ work, int32_t* __restrict__ counter) {
  __shared__ uint32_t hist[kHistCopies][kBins];
  __shared__ int32_t s_r;
  __shared__ unsigned long long s_since;   // probes since the last flush (block-wide)
  __shared__ int32_t s_nstash;
  // out(u) membership filter: 16 bits per key up to 16,384 keys (fewer beyond), so that
  // most absent keys are rejected without touching the table in global memory
  __shared__ uint32_t filt[(1 << kWideFilterLog2) / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kW = kWideThreads / 32;
  WideScratch t = wide_carve(scratch + wide_block_bytes(cap_max, words_max, dmax) * blockIdx.x,
                             cap_max, words_max, dmax);
  for (int k = threadIdx.x; k < kHistCopies * kBins; k += blockDim.x) (&hist[0][0])[k] = 0;
  const int32_t n = *n_p;
  uint32_t* my_hist = hist[lane & (kHistCopies - 1)];
  unsigned long long probes = 0, gathers = 0, outs = 0;
  int32_t cur = 0;   // member whose bins the shared histograms hold
  if (threadIdx.x == 0) s_since = 0;
  auto block_flush = [&]() {
    __syncthreads();
    for (int k = threadIdx.x; k < kBins; k += kWideThreads) {
      unsigned long long x = 0;
      for (int c = 0; c < kHistCopies; ++c) {
        x += hist[c][k];
        hist[c][k] = 0;
      }
      if (x) atomicAdd(&hist_out[(size_t)cur * kBins + k], x);
    }
    if (threadIdx.x == 0) s_since = 0;
    __syncthreads();
  };
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_r = atomicAdd(counter, 1);
    __syncthreads();
    const int32_t r = s_r;
    if (r >= n) break;
    const int32_t u = list[r];
    const int32_t m = member_of(g, u);   // the same on every thread
    if (m != cur || s_since > (1ull << 28)) {   // s_since is read after a barrier: uniform
      block_flush();
      cur = m;
    }
    const int32_t du = o.dplus[u];
    const int64_t bu = o.row_ptr[u];
    const int64_t eb = g.e_ptr[u];
    const int32_t szu = (int32_t)(g.e_ptr[u + 1] - eb);
    const int32_t words = (szu + 31) / 32;
    if (threadIdx.x == 0) outs += (unsigned long long)du;
    int dl = 4;   // du <= 2^dl; 2^(dl+1) slots per cuckoo table
    while ((int64_t(1) << dl) < (int64_t)du) ++dl;
    const uint32_t tslots = 2u << dl;
    const int sh = 31 - dl;
    const uint32_t rm = (1u << sh) - 1u, km = (1u << dl) - 1u;
    int fl = 5;   // filter bits: 2^fl >= 16 du, at most 2^kWideFilterLog2
    while (fl < kWideFilterLog2 && (int64_t(1) << fl) < 16 * (int64_t)du) ++fl;
    for (uint32_t s = threadIdx.x; s < tslots; s += kWideThreads) {
      t.c1[s] = ~0u;
      t.c2[s] = ~0u;
    }
    for (int64_t s = threadIdx.x; s < (int64_t)du * words; s += kWideThreads) t.mask[s] = 0;
    for (int s = threadIdx.x; s < (1 << fl) / 32; s += kWideThreads) filt[s] = 0;
    if (threadIdx.x == 0) s_nstash = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < du; k += kWideThreads) {
      int32_t x, om;
      get_entry<PACKED>(o, bu + k, x, om);
      const uint32_t fb = filt_bit((uint32_t)x, fl);
      atomicOr(&filt[fb >> 5], 1u << (fb & 31));
      uint32_t key = (uint32_t)x, kk = (uint32_t)k;
      bool second = false, placed = false;
      for (int tries = 0; tries < kCuckooTries; ++tries) {
        const uint32_t pa = key * (second ? kCuckooA2 : kCuckooA1);
        const uint32_t slot = pa >> sh;
        const uint32_t e = atomicExch(second ? &t.c2[slot] : &t.c1[slot], ((pa & rm) << dl) | kk);
        if (e == ~0u) {
          placed = true;
          break;
        }
        key = ((slot << sh) | (e >> dl)) * (second ? kCuckooA2Inv : kCuckooA1Inv);
        kk = e & km;
        second = !second;
      }
      if (!placed) {   // room for every key: du <= dmax
        const int at = atomicAdd(&s_nstash, 1);
        t.skey[at] = (int32_t)key;
        t.sidx[at] = (int32_t)kk;
      }
      t.ksz[k] = __ldg(g.esize + x);
      t.kbeg[k] = __ldg(o.row_ptr + x);
      t.kcnt[k] = __ldg(o.dplus + x);
    }
    __syncthreads();
    const int nst = s_nstash;   // read after a barrier: uniform
    for (int p = w; p < szu; p += kW) {
      const int32_t y = __ldg(g.e_idx + eb + p);
      const int64_t yb = __ldg(g.v_ptr + y), ye = __ldg(g.v_ptr + y + 1);
      if (lane == 0) gathers += (unsigned long long)(ye - yb);
      for (int64_t q = yb + lane; q < ye; q += 32) {
        const int32_t x = __ldg(g.v_idx + q);
        const uint32_t fb = filt_bit((uint32_t)x, fl);
        if (!((filt[fb >> 5] >> (fb & 31)) & 1u)) continue;
        const int kx = wide_find(t, x, dl, nst);
        if (kx >= 0) atomicOr(&t.mask[(size_t)kx * words + (p >> 5)], 1u << (p & 31));
      }
    }
    __syncthreads();
    // |e_x| -> |e_x| - omega_ux, the part of e_x outside e_u
    for (int k = threadIdx.x; k < du; k += kWideThreads) {
      int om = 0;
      for (int q = 0; q < words; ++q) om += __popc(t.mask[(size_t)k * words + q]);
      t.ksz[k] -= om;
    }
    __syncthreads();
    for (int k = w; k < du; k += kW) {
      const uint32_t* muv = t.mask + (size_t)k * words;
      const int rv = t.ksz[k];
      const int64_t vb = t.kbeg[k];
      const int32_t cnt = t.kcnt[k];
      if (lane == 0) {
        probes += (unsigned long long)cnt;
        atomicAdd(&s_since, (unsigned long long)cnt);
      }
      // kWideUnroll independent 32-entry loads in flight per warp, then their probes
      for (int32_t j0 = 0; j0 < cnt; j0 += 32 * kWideUnroll) {
        int32_t wv[kWideUnroll], om[kWideUnroll];
#pragma unroll
        for (int q = 0; q < kWideUnroll; ++q) {
          const int32_t j = j0 + q * 32 + lane;
          wv[q] = -1;
          om[q] = 0;
          if (j < cnt) get_entry<PACKED>(o, vb + j, wv[q], om[q]);
        }
#pragma unroll
        for (int q = 0; q < kWideUnroll; ++q) {
          const int32_t x = wv[q];
          if (x < 0) continue;
          const uint32_t fb = filt_bit((uint32_t)x, fl);
          if (!((filt[fb >> 5] >> (fb & 31)) & 1u)) continue;
          const int kw = wide_find(t, x, dl, nst);
          if (kw < 0) continue;
          // the one-word rule of region_bits, word by word over e_u
          const uint32_t* muw = t.mask + (size_t)kw * words;
          uint32_t any_a = 0, any_d = 0, any_f = 0, any_g = 0;
          int gg = 0;
          for (int qq = 0; qq < words; ++qq) {
            const uint32_t a = muv[qq], b = muw[qq];
            const uint32_t fq = full_mask(szu - 32 * qq);
            any_a |= fq & ~(a | b);
            any_d |= a & ~b;
            any_f |= b & ~a;
            any_g |= a & b;
            gg += __popc(a & b);
          }
          const int tt = om[q] - gg, rw = t.ksz[kw];
          const uint32_t bits = (uint32_t)(any_a != 0u) | ((uint32_t)(rv > tt) << 1) |
                                ((uint32_t)(rw > tt) << 2) | ((uint32_t)(any_d != 0u) << 3) |
                                ((uint32_t)(tt > 0) << 4) | ((uint32_t)(any_f != 0u) << 5) |
                                ((uint32_t)(any_g != 0u) << 6);
          atomicAdd(&my_hist[bits], 1u);
        }
      }
    }
  }
  block_flush();
  if (lane == 0) {
    atomicAdd(&work[0], probes);
    atomicAdd(&work[1], gathers);
    atomicAdd(&work[2], outs);
  }
}

// ------------------------------------------------------------------ cluster per u (large)
//
// Teams of out-degree above kWideLargeMin: a thread-block cluster of C blocks of
// kClusterThreads threads shares one hyperedge u and one set of global-memory tables.
// Every phase of the team (clearing, cuckoo insertion, Omega_ux masks, |e_x| -
// omega_ux, closure) is cut across all C * kClusterThreads threads, with a cluster
// barrier between phases, so only (blocks on the GPU) / C teams' tables are in use at
// any time.  Rank 0 takes the next hyperedge from the counter and the others read it
// from rank 0's shared memory.  Reads of the team's tables, masks and per-out-neighbour
// arrays go through L2 (ld.global.cg): other blocks of the cluster wrote them.  Each
// block keeps its own membership filter of out(u) (every key) in shared memory, and its
// own histogram.  The closure gives each warp one v at a time; hits (w's index and
// omega_vw) are queued per warp and classified 32 at a time.  C = 1 by default: on the
// tag-shaped workload at full size C = 2, 4 and 8 were 2%, 9% and 39% slower (the
// tables of fewer teams at a time did not pay for the cluster barriers).

constexpr int kClusterThreads = 1024;
#ifndef HG_WIDE_CLUSTER
#define HG_WIDE_CLUSTER 1
#endif
constexpr int kWideCluster = HG_WIDE_CLUSTER;   // blocks per cluster team

__device__ __forceinline__ int wide_find_l2(const WideScratch& t, int32_t x, int dl, int nst) {
  const int sh = 31 - dl;
  const uint32_t rm = (1u << sh) - 1u, km = (1u << dl) - 1u;
  const uint32_t p1 = (uint32_t)x * kCuckooA1, p2 = (uint32_t)x * kCuckooA2;
  const uint32_t a = __ldcg(t.c1 + (p1 >> sh)), b = __ldcg(t.c2 + (p2 >> sh));
  int k = (a >> dl) == (p1 & rm) ? (int)(a & km) : -1;
  k = (b >> dl) == (p2 & rm) ? (int)(b & km) : k;
  for (int i = 0; i < nst; ++i) k = __ldcg(t.skey + i) == x ? __ldcg(t.sidx + i) : k;
  return k;
}

template <bool PACKED>
__global__ void __launch_bounds__(kClusterThreads, 1)
    k_close_cluster(DevGraph g, Oriented o, const int32_t* __restrict__ list,
                    const int32_t* __restrict__ n_p, int64_t cap_max, int64_t words_max,
                    int64_t dmax, char* __restrict__ scratch,
                    unsigned long long* __restrict__ hist_out, unsigned long long* __restrict__ work,
                    int32_t* __restrict__ counter) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), csize = (int)cluster.num_blocks();
  constexpr int kCU = 8;                       // entries of out(v) in flight per lane
  constexpr int kCC = 32 * kCU + 32;           // candidate queue per warp
  constexpr int kCH = 64;                      // hit queue per warp
  __shared__ uint32_t hist[kHistCopies][kBins];
  __shared__ int32_t s_r;
  __shared__ unsigned long long s_since;
  __shared__ uint32_t filt[(1 << kWideFilterLog2) / 32];
  __shared__ int32_t cx[kClusterThreads / 32][kCC];   // candidates: w (passed the filter)
  __shared__ int32_t co[kClusterThreads / 32][kCC];   //             omega_vw
  __shared__ int32_t qk[kClusterThreads / 32][kCH];   // hits: index of w in out(u)
  __shared__ int32_t qo[kClusterThreads / 32][kCH];   //       omega_vw
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int gt = rank * kClusterThreads + (int)threadIdx.x, GT = csize * kClusterThreads;
  const int gw = gt >> 5, GW = GT >> 5;
  WideScratch t = wide_carve(scratch + wide_block_bytes(cap_max, words_max, dmax) *
                                           (size_t)(blockIdx.x / csize),
                             cap_max, words_max, dmax);
  for (int k = threadIdx.x; k < kHistCopies * kBins; k += kClusterThreads) (&hist[0][0])[k] = 0;
  const int32_t n = *n_p;
  uint32_t* my_hist = hist[lane & (kHistCopies - 1)];
  RunHist rh;
  unsigned long long probes = 0, gathers = 0, outs = 0;
  int32_t cur = 0;
  if (threadIdx.x == 0) s_since = 0;
  __syncthreads();
  auto block_flush = [&]() {
    rh.flush(my_hist);
    __syncthreads();
    for (int k = threadIdx.x; k < kBins; k += kClusterThreads) {
      unsigned long long x = 0;
      for (int c = 0; c < kHistCopies; ++c) {
        x += hist[c][k];
        hist[c][k] = 0;
      }
      if (x) atomicAdd(&hist_out[(size_t)cur * kBins + k], x);
    }
    if (threadIdx.x == 0) s_since = 0;
    __syncthreads();
  };
  while (true) {
    if (rank == 0 && threadIdx.x == 0) s_r = atomicAdd(counter, 1);
    cluster.sync();
    const int32_t r = *cluster.map_shared_rank(&s_r, 0);
    if (r >= n) {
      cluster.sync();   // rank 0's shared memory stays until every block has read it
      break;
    }
    const int32_t u = list[r];
    const int32_t m = member_of(g, u);
    if (m != cur || s_since > (1ull << 28)) {   // read after a barrier: uniform in the block
      block_flush();
      cur = m;
    }
    const int32_t du = o.dplus[u];
    const int64_t bu = o.row_ptr[u];
    const int64_t eb = g.e_ptr[u];
    const int32_t szu = (int32_t)(g.e_ptr[u + 1] - eb);
    const int32_t words = (szu + 31) / 32;
    if (gt == 0) outs += (unsigned long long)du;
    int dl = 4;
    while ((int64_t(1) << dl) < (int64_t)du) ++dl;
    const uint32_t tslots = 2u << dl;
    const int sh = 31 - dl;
    const uint32_t rm = (1u << sh) - 1u, km = (1u << dl) - 1u;
    int fl = 5;
    while (fl < kWideFilterLog2 && (int64_t(1) << fl) < 16 * (int64_t)du) ++fl;
    // 1. clear the team's tables and masks (cluster-wide), and this block's filter
    for (uint32_t s = (uint32_t)gt; s < tslots; s += (uint32_t)GT) {
      t.c1[s] = ~0u;
      t.c2[s] = ~0u;
    }
    for (int64_t s = gt; s < (int64_t)du * words; s += GT) t.mask[s] = 0;
    if (gt == 0) *t.nstash = 0;
    for (int s = threadIdx.x; s < (1 << fl) / 32; s += kClusterThreads) filt[s] = 0;
    cluster.sync();
    // 2. out(u) into the cuckoo set (cluster-wide share of the keys); every key into
    //    this block's filter
    for (int k = gt; k < du; k += GT) {
      int32_t x, om;
      get_entry<PACKED>(o, bu + k, x, om);
      uint32_t key = (uint32_t)x, kk = (uint32_t)k;
      bool second = false, placed = false;
      for (int tries = 0; tries < kCuckooTries; ++tries) {
        const uint32_t pa = key * (second ? kCuckooA2 : kCuckooA1);
        const uint32_t slot = pa >> sh;
        const uint32_t e = atomicExch(second ? &t.c2[slot] : &t.c1[slot], ((pa & rm) << dl) | kk);
        if (e == ~0u) {
          placed = true;
          break;
        }
        key = ((slot << sh) | (e >> dl)) * (second ? kCuckooA2Inv : kCuckooA1Inv);
        kk = e & km;
        second = !second;
      }
      if (!placed) {   // room for every key: du <= dmax
        const int at = atomicAdd(t.nstash, 1);
        t.skey[at] = (int32_t)key;
        t.sidx[at] = (int32_t)kk;
      }
      t.ksz[k] = __ldg(g.esize + x);
      t.kbeg[k] = __ldg(o.row_ptr + x);
      t.kcnt[k] = __ldg(o.dplus + x);
    }
    for (int k = threadIdx.x; k < du; k += kClusterThreads) {
      int32_t x, om;
      get_entry<PACKED>(o, bu + k, x, om);
      const uint32_t fb = filt_bit((uint32_t)x, fl);
      atomicOr(&filt[fb >> 5], 1u << (fb & 31));
    }
    cluster.sync();
    const int nst = __ldcg(t.nstash);
    // 3. Omega_ux masks: vertex p of e_u per warp of the cluster
    for (int p = gw; p < szu; p += GW) {
      const int32_t y = __ldg(g.e_idx + eb + p);
      const int64_t yb = __ldg(g.v_ptr + y), ye = __ldg(g.v_ptr + y + 1);
      if (lane == 0) gathers += (unsigned long long)(ye - yb);
      for (int64_t q = yb + lane; q < ye; q += 32) {
        const int32_t x = __ldg(g.v_idx + q);
        const uint32_t fb = filt_bit((uint32_t)x, fl);
        if (!((filt[fb >> 5] >> (fb & 31)) & 1u)) continue;
        const int kx = wide_find_l2(t, x, dl, nst);
        if (kx >= 0) atomicOr(&t.mask[(size_t)kx * words + (p >> 5)], 1u << (p & 31));
      }
    }
    cluster.sync();
    // |e_x| -> |e_x| - omega_ux, the part of e_x outside e_u
    for (int k = gt; k < du; k += GT) {
      int om = 0;
      for (int q = 0; q < words; ++q) om += __popc(__ldcg(t.mask + (size_t)k * words + q));
      t.ksz[k] = __ldcg(t.ksz + k) - om;
    }
    cluster.sync();
    // 4. closure: out-neighbour k (= v) per warp of the cluster.  Entries of out(v) that
    //    pass this block's filter are queued as candidates; 32 candidates at a time are
    //    looked up in the global tables with every lane busy; hits (w's index and
    //    omega_vw) are queued and classified 32 at a time.
    for (int k = gw; k < du; k += GW) {
      const uint32_t* muv = t.mask + (size_t)k * words;
      const int rv = __ldcg(t.ksz + k);
      const int64_t vb = __ldcg(t.kbeg + k);
      const int32_t cnt = __ldcg(t.kcnt + k);
      if (lane == 0) {
        probes += (unsigned long long)cnt;
        atomicAdd(&s_since, (unsigned long long)cnt);
      }
      auto classify = [&](int at) {
        const int kw = qk[wl][at];
        const uint32_t* muw = t.mask + (size_t)kw * words;
        uint32_t any_a = 0, any_d = 0, any_f = 0, any_g = 0;
        int gg = 0;
        for (int qq = 0; qq < words; ++qq) {
          const uint32_t a = __ldcg(muv + qq), b = __ldcg(muw + qq);
          const uint32_t fq = full_mask(szu - 32 * qq);
          any_a |= fq & ~(a | b);
          any_d |= a & ~b;
          any_f |= b & ~a;
          any_g |= a & b;
          gg += __popc(a & b);
        }
        const int tt = qo[wl][at] - gg, rw = __ldcg(t.ksz + kw);
        rh.add((uint32_t)(any_a != 0u) | ((uint32_t)(rv > tt) << 1) | ((uint32_t)(rw > tt) << 2) |
                   ((uint32_t)(any_d != 0u) << 3) | ((uint32_t)(tt > 0) << 4) |
                   ((uint32_t)(any_f != 0u) << 5) | ((uint32_t)(any_g != 0u) << 6),
               my_hist);
      };
      int cq = 0, qn = 0;   // queued candidates and hits (the same on every lane)
      // look up candidates [cq - m, cq) (m <= 32, lane < m active); queue the hits and
      // classify full rounds of 32
      auto resolve = [&](int m) {
        cq -= m;
        int kw = -1, ow = 0;
        if (lane < m) {
          kw = wide_find_l2(t, cx[wl][cq + lane], dl, nst);
          ow = co[wl][cq + lane];
        }
        const bool hit = kw >= 0;
        const unsigned bal = __ballot_sync(kFull, hit);
        if (hit) {
          const int at = qn + __popc(bal & ((1u << lane) - 1u));
          qk[wl][at] = kw;
          qo[wl][at] = ow;
        }
        qn += __popc(bal);
        __syncwarp();
        if (qn >= 32) {
          qn -= 32;
          classify(qn + lane);
          __syncwarp();
        }
      };
      for (int32_t j0 = 0; j0 < cnt; j0 += 32 * kCU) {
        int32_t wv[kCU], om[PACKED ? 1 : kCU];
#pragma unroll
        for (int q = 0; q < kCU; ++q) {
          const int32_t j = j0 + q * 32 + lane;
          if (PACKED) {
            wv[q] = -1;   // raw entry (w << 8) | omega_vw; -1 = none
            if (j < cnt) wv[q] = (int32_t)__ldg(o.packed + vb + j);
          } else {
            wv[q] = -1;
            om[q] = 0;
            if (j < cnt) get_entry<PACKED>(o, vb + j, wv[q], om[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < kCU; ++q) {
          const int32_t x = PACKED ? (wv[q] == -1 ? -1 : (int32_t)((uint32_t)wv[q] >> 8)) : wv[q];
          bool pass = false;
          if (x >= 0) {
            const uint32_t fb = filt_bit((uint32_t)x, fl);
            pass = (filt[fb >> 5] >> (fb & 31)) & 1u;
          }
          const unsigned bal = __ballot_sync(kFull, pass);
          if (pass) {
            const int at = cq + __popc(bal & ((1u << lane) - 1u));
            cx[wl][at] = x;
            co[wl][at] = PACKED ? (int32_t)((uint32_t)wv[q] & 0xffu) : om[PACKED ? 0 : q];
          }
          cq += __popc(bal);
        }
        __syncwarp();
        while (cq >= 32) resolve(32);
      }
      if (cq > 0) resolve(cq);
      while (qn >= 32) {
        qn -= 32;
        classify(qn + lane);
        __syncwarp();
      }
      if (lane < qn) classify(lane);
      __syncwarp();
    }
    cluster.sync();   // the next team clears these tables
  }
  block_flush();
  if (lane == 0) {
    atomicAdd(&work[0], probes);
    atomicAdd(&work[1], gathers);
    atomicAdd(&work[2], outs);
  }
}

// ------------------------------------------------------------------ bucketing

constexpr int kWarpMaskBits = 32;   // warp tables keep Omega_ux in one 32-bit word

// Team shape of u (bucket index, -1 when u closes nothing).
__device__ __forceinline__ int close_bucket_of(int32_t d, int32_t sz, bool all_block,
                                               int warp_max, int block_max) {
  if (d < 2) return -1;
  if (all_block) return kWideBucket;
  if (sz <= kWarpMaskBits && d <= warp_max) return d <= 64 ? 0 : (d <= 128 ? 1 : 2);
  if (sz <= kWarpMaskBits && d <= 1024) return 3;
  if (sz <= kWarpMaskBits && d <= 2048) return 4;
  if (sz <= kWarpMaskBits && d <= block_max) return 5;
  return d > kWideLargeMin ? kClusterBucket : kWideBucket;
}

// Each block takes a contiguous range of kBucketRowsPerBlock hyperedges: it counts
// them per bucket in shared memory, reserves its slice of every list with one global
// atomic per bucket, then writes the hyperedges into the slices.  The largest
// out-degree and size of the wide bucket are reduced per warp before their atomics.
constexpr int kBucketThreads = 256;
constexpr int kBucketRowsPerThread = 8;
constexpr int kBucketRowsPerBlock = kBucketThreads * kBucketRowsPerThread;

__global__ void __launch_bounds__(kBucketThreads)
    k_bucket_close(DevGraph g, Oriented o, CloseBuckets b,
                   unsigned long long* __restrict__ wide_max, bool all_block, int warp_max,
                   int block_max, const uint8_t* __restrict__ sel) {
  __shared__ int32_t s_cnt[kCloseBuckets], s_base[kCloseBuckets];
  const int lane = threadIdx.x & 31;
  unsigned long long my_d = 0, my_s = 0;
  for (int64_t r0 = (int64_t)blockIdx.x * kBucketRowsPerBlock; r0 < g.ne;
       r0 += (int64_t)gridDim.x * kBucketRowsPerBlock) {
    if (threadIdx.x < kCloseBuckets) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    int bk[kBucketRowsPerThread];
#pragma unroll
    for (int q = 0; q < kBucketRowsPerThread; ++q) {   // rows r0 + q * 256 + thread
      const int64_t u = r0 + (int64_t)q * kBucketThreads + threadIdx.x;
      bk[q] = -1;
      if (u < g.ne && (!sel || sel[u])) {
        const int32_t d = o.dplus[u], sz = g.esize[u];
        bk[q] = close_bucket_of(d, sz, all_block, warp_max, block_max);
        if (bk[q] >= kWideBucket) {
          my_d = (unsigned long long)d > my_d ? (unsigned long long)d : my_d;
          my_s = (unsigned long long)sz > my_s ? (unsigned long long)sz : my_s;
        }
      }
#pragma unroll
      for (int k = 0; k < kCloseBuckets; ++k) {
        const unsigned bal = __ballot_sync(kFull, bk[q] == k);
        if (bal && lane == 0) atomicAdd(&s_cnt[k], __popc(bal));
      }
    }
    __syncthreads();
    if (threadIdx.x < kCloseBuckets) {
      const int32_t n = s_cnt[threadIdx.x];
      s_base[threadIdx.x] = n ? atomicAdd(&b.count[threadIdx.x], n) : 0;
      s_cnt[threadIdx.x] = 0;   // reused as the running offset
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kBucketRowsPerThread; ++q) {
      const int64_t u = r0 + (int64_t)q * kBucketThreads + threadIdx.x;
#pragma unroll
      for (int k = 0; k < kCloseBuckets; ++k) {
        const unsigned bal = __ballot_sync(kFull, bk[q] == k);
        if (!bal) continue;
        int at = 0;
        if (lane == 0) at = atomicAdd(&s_cnt[k], __popc(bal));
        at = __shfl_sync(kFull, at, 0);
        if (bk[q] == k) b.lists[k][s_base[k] + at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)u;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int dd = 16; dd > 0; dd >>= 1) {
    const unsigned long long od = __shfl_down_sync(kFull, my_d, dd);
    const unsigned long long os = __shfl_down_sync(kFull, my_s, dd);
    my_d = od > my_d ? od : my_d;
    my_s = os > my_s ? os : my_s;
  }
  if (lane == 0 && (my_d | my_s)) {
    atomicMax(&wide_max[0], my_d);
    atomicMax(&wide_max[1], my_s);
  }
}

template <int D_LOG2, int WARPS, bool PACKED, bool OFF32>
void launch_warp_t(const DevGraph& g, const Oriented& o, const int32_t* list, int32_t n,
                   const int32_t* n_p, unsigned long long* hist, unsigned long long* work,
                   int32_t* counter, int32_t* overflow, int32_t* n_overflow, int handover,
                   cudaStream_t s, int nsm) {
  auto kern = k_close_warp<D_LOG2, WARPS, PACKED, OFF32>;
  const int smem = (int)(WARPS * sizeof(WarpTables<D_LOG2, PACKED, OFF32>));
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  int blocks = (n + WARPS - 1) / WARPS;
  if (blocks > per_sm * nsm) blocks = per_sm * nsm;
  note_launch();
  kern<<<blocks, WARPS * 32, smem, s>>>(g, o, list, n_p, hist, work, counter, overflow,
                                         n_overflow, handover);
}

template <int D_LOG2, int WARPS>
void launch_warp(const DevGraph& g, const Oriented& o, int packed, const int32_t* list, int32_t n,
                 const int32_t* n_p, unsigned long long* hist, unsigned long long* work,
                 int32_t* counter, int32_t* overflow, int32_t* n_overflow, int handover,
                 cudaStream_t s, int nsm) {
  const bool off32 = o.slots > 0 && o.slots < (int64_t(1) << 32);
  if (packed && off32)
    launch_warp_t<D_LOG2, WARPS, true, true>(g, o, list, n, n_p, hist, work, counter, overflow,
                                             n_overflow, handover, s, nsm);
  else if (packed)
    launch_warp_t<D_LOG2, WARPS, true, false>(g, o, list, n, n_p, hist, work, counter, overflow,
                                              n_overflow, handover, s, nsm);
  else if (off32)
    launch_warp_t<D_LOG2, WARPS, false, true>(g, o, list, n, n_p, hist, work, counter, overflow,
                                              n_overflow, handover, s, nsm);
  else
    launch_warp_t<D_LOG2, WARPS, false, false>(g, o, list, n, n_p, hist, work, counter,
                                               overflow, n_overflow, handover, s, nsm);
}

template <int D_LOG2, int WARPS, bool PACKED, int DMAX = (1 << D_LOG2)>
void launch_block_t(const DevGraph& g, const Oriented& o, const int32_t* list, int32_t n,
                    const int32_t* n_p, unsigned long long* hist, unsigned long long* work,
                    int32_t* counter, int32_t* overflow, int32_t* n_overflow, int handover,
                    cudaStream_t s, int nsm) {
  auto kern = k_close_block<D_LOG2, WARPS, PACKED, DMAX>;
  const int smem = (int)sizeof(BlockTables<D_LOG2, WARPS, PACKED, DMAX>);
  // the tables plus the kernel's static bins (one set per warp, or 8) and fetch slot fit
  // the 232,448 bytes of shared memory a block may use
  static_assert(sizeof(BlockTables<D_LOG2, WARPS, PACKED, DMAX>) +
                        sizeof(uint32_t) * kBins * (DMAX == (1 << D_LOG2) ? WARPS : 8) + 16 <=
                    232448,
                "block-team shared memory");
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  int blocks = n < per_sm * nsm ? n : per_sm * nsm;
  note_launch();
  kern<<<blocks, WARPS * 32, smem, s>>>(g, o, list, n_p, hist, work, counter, overflow,
                                         n_overflow, handover);
}

template <int D_LOG2>
void launch_block(const DevGraph& g, const Oriented& o, int packed, const int32_t* list, int32_t n,
                  const int32_t* n_p, unsigned long long* hist, unsigned long long* work,
                  int32_t* counter, int32_t* overflow, int32_t* n_overflow, int handover,
                  cudaStream_t s, int nsm) {
  if (packed)
    launch_block_t<D_LOG2, kBlockWarps, true>(g, o, list, n, n_p, hist, work, counter, overflow,
                                              n_overflow, handover, s, nsm);
  else
    launch_block_t<D_LOG2, kBlockWarpsUnpacked, false>(g, o, list, n, n_p, hist, work, counter,
                                                       overflow, n_overflow, handover, s, nsm);
}

}  // namespace

void launch_bucket_close(const DevGraph& g, const Oriented& o, CloseBuckets b,
                         unsigned long long* wide_max, bool all_block, int warp_max,
                         int block_max, const uint8_t* sel, cudaStream_t s) {
  if (g.ne == 0) return;
  int64_t blocks = (g.ne + kBucketRowsPerBlock - 1) / kBucketRowsPerBlock;
  if (blocks > 4096) blocks = 4096;
  note_launch();
  k_bucket_close<<<(unsigned)blocks, kBucketThreads, 0, s>>>(g, o, b, wide_max, all_block,
                                                             warp_max, block_max, sel);
}

size_t close_wide_scratch_bytes(int64_t cap, int64_t words, int64_t dmax, int nsm) {
  if (cap <= 0) return 0;
  return wide_block_bytes(cap, words, dmax) * (size_t)(nsm * kWideBlocksPerSm);
}

void launch_close(int bucket, const DevGraph& g, const Oriented& o, int packed,
                  const int32_t* list, int32_t n, const int32_t* n_p, int64_t wide_cap,
                  int64_t wide_words, int64_t wide_dmax, void* scratch, unsigned long long* hist,
                  unsigned long long* work, int32_t* counter, int32_t* overflow,
                  int32_t* n_overflow, int handover, cudaStream_t s, int nsm) {
  if (n <= 0) return;
  switch (bucket) {
    case 0:
      launch_warp<6, 8>(g, o, packed, list, n, n_p, hist, work, counter, overflow, n_overflow,
                        handover, s, nsm);
      break;
    case 1:
      launch_warp<7, 6>(g, o, packed, list, n, n_p, hist, work, counter, overflow, n_overflow,
                        handover, s, nsm);
      break;
    case 2:
      launch_warp<8, 4>(g, o, packed, list, n, n_p, hist, work, counter, overflow, n_overflow,
                        handover, s, nsm);
      break;
    case 3:
      launch_block<10>(g, o, packed, list, n, n_p, hist, work, counter, overflow, n_overflow,
                            handover, s, nsm);
      break;
    case 4:
      launch_block<11>(g, o, packed, list, n, n_p, hist, work, counter, overflow, n_overflow,
                            handover, s, nsm);
      break;
    case 5:   // the packed layout's shape reaches out-degree 6,144 (13-bit indices)
      if (packed)
        launch_block_t<13, kBlockWarps, true, kBlockMaxPacked>(g, o, list, n, n_p, hist, work,
                                                               counter, overflow, n_overflow,
                                                               handover, s, nsm);
      else
        launch_block_t<12, kBlockWarpsUnpacked, false>(g, o, list, n, n_p, hist, work, counter,
                                                       overflow, n_overflow, handover, s, nsm);
      break;
    case kClusterBucket: {
      // clusters of kWideCluster blocks, as many as can be resident at once
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kWideCluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.blockDim = dim3(kClusterThreads);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      auto kern = packed ? k_close_cluster<true> : k_close_cluster<false>;
      int clusters = 0;
      cfg.gridDim = dim3((unsigned)(nsm / kWideCluster * kWideCluster));
      if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        clusters = nsm / kWideCluster;
      }
      if (clusters > n) clusters = n;
      if (clusters < 1) clusters = 1;
      cfg.gridDim = dim3((unsigned)(clusters * kWideCluster));
      note_launch();
      cudaLaunchKernelEx(&cfg, kern, g, o, list, n_p, wide_cap, wide_words, wide_dmax,
                         (char*)scratch, hist, work, counter);
      break;
    }
    default: {
      int blocks = n < nsm * kWideBlocksPerSm ? n : nsm * kWideBlocksPerSm;
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
