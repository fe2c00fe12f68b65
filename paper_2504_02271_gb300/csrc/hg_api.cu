// C ABI of libhg: argument checks, device memory, and the order of the kernels
// of the two-step framework (Sec. 3.1 step one, Sec. 3.2-3.3 step two, Def. 5.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "hg_internal.cuh"

using namespace hg;

namespace {

// ---------------------------------------------------------------- allocator

struct AllocatorHooks {
  hg_alloc_fn alloc = nullptr;
  hg_free_fn free_fn = nullptr;
  void* ctx = nullptr;
};
std::mutex g_alloc_mu;
AllocatorHooks g_hooks;

struct Block {
  void* p;
  size_t bytes;
  hg_free_fn free_fn;  // the hook that owns it (nullptr = cudaFreeAsync)
  void* ctx;
};

// Device block of counters and flags shared by the kernels of one handle.
struct Small {
  int err;
  int32_t pad0;
  int32_t counters[16];       // work-fetch counters
  int32_t bucket_count[16];   // [0..2] wedge buckets, [3] handed-over teams, [4..9] close buckets
  unsigned long long wc;      // inclusion-type wedges
  unsigned long long max_cand;
  int32_t max_size;
  int32_t pad1;
  unsigned long long deg_stats[3];   // sum C(deg,2), max deg, sum deg
  unsigned long long out_stats[3];   // sum C(d+,2), max d+, sum d+
  unsigned long long wide_max[2];    // close bucket 3: max d+, max |e_u|
  unsigned long long hist[128];      // closure: labelled region masks; samplers: bins 0..20
  unsigned long long work[kCloseBuckets][3];   // closure per team shape: probes, E_y entries, out-entries
  unsigned long long found;                    // triples of hg_enumerate_pattern
  unsigned long long sample_work[3];           // last sampler launch: pointer, entry, id reads
};

struct KTime {
  const char* name;
  cudaEvent_t a, b;
};

}  // namespace

struct hg_graph {
  int device = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  int32_t nv = 0, ne = 0;
  int64_t nnz = 0;
  // load stage
  int64_t* e_ptr = nullptr;
  int32_t* e_idx = nullptr;
  int32_t* esize = nullptr;
  int64_t* v_ptr = nullptr;
  int32_t* v_idx = nullptr;
  int64_t* cand = nullptr;
  int32_t max_size = 0;
  int64_t max_cand = 0;
  Small* small = nullptr;
  void* scan_tmp = nullptr;
  std::vector<Block> load_blocks;
  // build stage
  std::vector<Block> build_blocks;
  int32_t* deg = nullptr;
  Oriented ori{};
  int packed = 0;
  int close_mode = 0;
  int warp_team_max = 256;   // of the last build (step two routes teams by it)
  hg_tuning tuned{};         // hg_autotune's choice, used by builds given no tuning
  bool has_tuned = false;
  uint64_t two_w = 0;
  bool built = false;
  hg_wedge_stats stats{};
  // every row's (j, omega_ij) in the capacity layout, kept for the samplers' rows
  int64_t* cap_ptr = nullptr;
  Oriented cap_rows{};
  int64_t* deg_ptr = nullptr;   // exclusive scan of deg (offsets of exact neighbour rows)
  DenseInfo dn{};
  int32_t* upc = nullptr;          // |{j > i : omega_ij > 0}| per row
  // sampling stage: rows of neighbours j > i sorted by j (order O of Sec. 2)
  std::vector<Block> sample_blocks;
  int64_t* up_ptr = nullptr;
  int32_t* up_index = nullptr;   // bucket index of up_ptr
  Oriented up{};
  bool upper_built = false;
  // Algorithm 7: the upper rows split by type, and every neighbour row sorted
  bool adv_built = false;
  int64_t* t_ptr = nullptr;
  int64_t* c_ptr = nullptr;
  int32_t* t_index = nullptr;
  int32_t* c_index = nullptr;
  Oriented t_ent{}, c_ent{}, full{};
  uint64_t Wt = 0, Wc = 0;
  // the sub-hypergraph G' for sigma < 1 (Algorithms 6-7, the sigma|E| draw), kept for its seed
  hg_graph* sub = nullptr;
  uint64_t sub_seed = 0;
  double sub_sigma = 1.0;
  uint64_t sample_work[3] = {0, 0, 0};   // of the last hg_sample_estimate
  // count stage
  std::vector<Block> count_blocks;
  bool counted = false;
  uint64_t counts[21] = {0};
  uint64_t masks[128] = {0};   // canonical region-mask histogram of the last count
  hg_close_stats cstats{};
  bool have_cstats = false;    // cstats describe the last hg_count_patterns or hg_count_owned
  // a wave of a batch: nm members, member m owning hyperedges [m_eoff[m], m_eoff[m+1])
  // and union vertices [m_voff[m], m_voff[m+1])
  int32_t nm = 0;
  int32_t* m_eoff = nullptr;
  int32_t* m_voff = nullptr;
  int32_t* wcr = nullptr;                 // per-row inclusion wedges (build)
  unsigned long long* mstats = nullptr;   // [nm][4]: sum deg, sum C(deg,2), W_c, max deg
  unsigned long long* mhist = nullptr;    // [nm][128] labelled region-mask bins (count)
  std::vector<unsigned long long> h_mstats;
  std::vector<uint64_t> h_mmasks;         // [nm][128] canonical region-mask histograms
  // timing
  bool timing = false;
  std::vector<KTime> pending;
  std::vector<std::pair<const char*, std::pair<float, int>>> times;  // static names
};

namespace hg {
void alloc_bypass_hooks(bool on);
static std::atomic<unsigned long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
}  // namespace hg

namespace {

// Threads of the library's own runtime (the server's workers) allocate with
// cudaMallocAsync even when the caller installed hooks: the hooks may call back into
// an interpreter that those threads must not wait on.
thread_local bool t_bypass_hooks = false;

void* dev_alloc(hg_graph* g, std::vector<Block>& owner, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  AllocatorHooks h;
  if (!t_bypass_hooks) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h = g_hooks;
  }
  void* p = nullptr;
  if (h.alloc) {
    p = h.alloc(bytes, (void*)g->stream, h.ctx);
  } else if (cudaMallocAsync(&p, bytes, g->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) owner.push_back(Block{p, bytes, h.alloc ? h.free_fn : nullptr, h.ctx});
  return p;
}

void release(hg_graph* g, std::vector<Block>& owner) {
  for (auto& b : owner) {
    if (b.free_fn) b.free_fn(b.p, b.bytes, (void*)g->stream, b.ctx);
    else cudaFreeAsync(b.p, g->stream);
  }
  owner.clear();
}

hg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HG_OK : HG_ERR_CUDA; }

#define HG_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return HG_ERR_CUDA;               \
  } while (0)

#define HG_TRY(st)                     \
  do {                                 \
    hg_status s_ = (st);               \
    if (s_ != HG_OK) return s_;        \
  } while (0)

hg_status dev_err_status(int e) {
  switch (e) {
    case DE_OK: return HG_OK;
    case DE_EMPTY: return HG_ERR_EMPTY_HYPEREDGE;
    case DE_RANGE: return HG_ERR_VERTEX_RANGE;
    case DE_DUPV: return HG_ERR_DUP_VERTEX;
    case DE_UNSORTED: return HG_ERR_UNSORTED;
    case DE_DUPEDGE: return HG_ERR_DUPLICATE_HYPEREDGE;
    case DE_PTR: return HG_ERR_INVALID_ARG;
    case DE_LIMIT: return HG_ERR_UNSUPPORTED;
    case DE_TIMEOUT: return HG_ERR_TIMEOUT;
    default: return HG_ERR_INTERNAL;
  }
}

// Read back the small block and check the error word.
hg_status sync_small(hg_graph* g, Small* host) {
  HG_CUDA(cudaMemcpyAsync(host, g->small, sizeof(Small), cudaMemcpyDeviceToHost, g->stream));
  HG_CUDA(cudaStreamSynchronize(g->stream));
  HG_CUDA(cudaGetLastError());
  return dev_err_status(host->err);
}

void t_begin(hg_graph* g, const char* name) {
  if (!g->timing) return;
  KTime k{name, nullptr, nullptr};
  cudaEventCreate(&k.a);
  cudaEventCreate(&k.b);
  cudaEventRecord(k.a, g->stream);
  g->pending.push_back(k);
}

void t_end(hg_graph* g) {
  if (!g->timing || g->pending.empty()) return;
  cudaEventRecord(g->pending.back().b, g->stream);
}

// Called after a synchronising point: fold the pending event pairs into g->times.
void t_collect(hg_graph* g) {
  for (auto& k : g->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, k.a, k.b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    bool found = false;
    for (auto& t : g->times)
      if (std::strcmp(t.first, k.name) == 0) {
        t.second.first += ms;
        t.second.second += 1;
        found = true;
      }
    if (!found) g->times.push_back({k.name, {ms, 1}});
    cudaEventDestroy(k.a);
    cudaEventDestroy(k.b);
  }
  g->pending.clear();
}

DevGraph dev_graph(const hg_graph* g) {
  DevGraph d;
  d.nv = g->nv;
  d.ne = g->ne;
  d.nnz = g->nnz;
  d.e_ptr = g->e_ptr;
  d.e_idx = g->e_idx;
  d.esize = g->esize;
  d.v_ptr = g->v_ptr;
  d.v_idx = g->v_idx;
  d.m_eoff = g->m_eoff;
  d.nm = g->nm;
  return d;
}

// ---------------------------------------------------------------- pattern table
//
// Pattern of a labelled region mask (bit r = region r of (a)..(g), Sec. 2) from
// set relations.  Each hyperedge is the union of its non-empty regions, so
// equality, containment and intersection of hyperedges are the same relations
// on their sets of non-empty regions.
//   class by the number of inclusion-type pairs (Def. 2.3): 3 CCC, 2 TCC, 1 TTC,
//   0 TTT (Sec. 2);
//   TCC: the third hyperedge lies inside both others (2 if it equals their
//        intersection, else 3) or contains both (4 if it equals their union,
//        else 5) - the tests of Algorithm 5;
//   TTC: with big containing small and z the third, 6 if big and small meet z
//        in the same vertices, 7 if big = small + (big cap z), else 8 -
//        Algorithm 5's omega tests;
//   TTT: region g non-empty gives 9-16, empty gives 17-20 (Sec. 3.2); inside a
//        subclass, ascending number of non-empty pairwise regions (d, e, f),
//        then of single regions (a, b, c).
int pattern_of(int m) {
  const int U = (1 << 0) | (1 << 3) | (1 << 5) | (1 << 6);
  const int V = (1 << 1) | (1 << 3) | (1 << 4) | (1 << 6);
  const int W = (1 << 2) | (1 << 4) | (1 << 5) | (1 << 6);
  const int S[3] = {m & U, m & V, m & W};
  auto sub = [](int x, int y) { return (x & ~y) == 0; };
  auto incl = [&](int x, int y) { return sub(S[x], S[y]) || sub(S[y], S[x]); };
  for (int x = 0; x < 3; ++x)
    for (int y = x + 1; y < 3; ++y) {
      if (!(S[x] & S[y])) return 0;   // not a hyper-triangle
      if (S[x] == S[y]) return 0;     // equal hyperedges
    }
  const int pairs[3][3] = {{0, 1, 2}, {1, 2, 0}, {0, 2, 1}};  // (x, y, third)
  int nc = 0;
  for (auto& p : pairs) nc += incl(p[0], p[1]);
  if (nc == 3) return 1;
  if (nc == 2) {
    for (auto& p : pairs) {
      if (incl(p[0], p[1])) continue;
      const int x = S[p[0]], y = S[p[1]], z = S[p[2]];
      if (sub(z, x) && sub(z, y)) return z == (x & y) ? 2 : 3;
      return z == (x | y) ? 4 : 5;
    }
  }
  if (nc == 1) {
    for (auto& p : pairs) {
      if (!incl(p[0], p[1])) continue;
      const int big = sub(S[p[1]], S[p[0]]) ? S[p[0]] : S[p[1]];
      const int small = big == S[p[0]] ? S[p[1]] : S[p[0]];
      const int z = S[p[2]];
      if ((big & z) == (small & z)) return 6;
      if (big == (small | (big & z))) return 7;
      return 8;
    }
  }
  const int pw = ((m >> 3) & 1) + ((m >> 4) & 1) + ((m >> 5) & 1);
  const int sg = (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1);
  if ((m >> 6) & 1) {
    static const int dense[4][4] = {{0, 0, 0, 9}, {0, 0, 0, 10}, {0, 0, 11, 12}, {13, 14, 15, 16}};
    return dense[pw][sg];
  }
  return pw == 3 ? 17 + sg : 0;
}

void build_lut(uint8_t lut[128]) {
  for (int m = 0; m < 128; ++m) lut[m] = (uint8_t)pattern_of(m);
}

// Canonical form of a labelled region mask: the smallest mask among the six orders of
// the three hyperedges.  Region r is coded by the hyperedges holding it (bit 0 = first,
// bit 1 = second, bit 2 = third: a 1, b 2, c 4, d 3, e 6, f 5, g 7); reordering the
// hyperedges permutes those three bits.
int canonical_of(int m) {
  static const int kCode[7] = {1, 2, 4, 3, 6, 5, 7};
  static const int kOrders[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                    {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int best = 127;
  for (const auto& o : kOrders) {
    int out = 0;
    for (int r = 0; r < 7; ++r) {
      if (!(m >> r & 1)) continue;
      int code = 0;   // new position q holds old hyperedge o[q]
      for (int q = 0; q < 3; ++q) code |= (kCode[r] >> o[q] & 1) << q;
      for (int r2 = 0; r2 < 7; ++r2)
        if (kCode[r2] == code) out |= 1 << r2;
    }
    best = std::min(best, out);
  }
  return best;
}

// Fold 128 labelled-mask bins into canonical-mask bins and the 21 counts.  False when a
// bin that is not a hyper-triangle of three distinct hyperedges holds anything.
bool fold_masks(const unsigned long long labelled[128], uint64_t canon[128],
                uint64_t counts[21]) {
  uint8_t lut[128];
  build_lut(lut);
  std::memset(canon, 0, sizeof(uint64_t) * 128);
  std::memset(counts, 0, sizeof(uint64_t) * 21);
  for (int m = 0; m < 128; ++m) {
    if (!labelled[m]) continue;
    if (lut[m] == 0) return false;
    canon[canonical_of(m)] += labelled[m];
    counts[lut[m]] += labelled[m];
    counts[0] += labelled[m];
  }
  return true;
}

hg_status check_device(int* dev, int* nsm) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return HG_ERR_NO_DEVICE;
  }
  HG_CUDA(cudaGetDevice(dev));
  cudaDeviceProp p;
  HG_CUDA(cudaGetDeviceProperties(&p, *dev));
  if (p.major != 10 || p.minor != 3) return HG_ERR_NO_DEVICE;  // built for sm_103a only
  *nsm = p.multiProcessorCount;
  return HG_OK;
}

template <typename T>
T* alloc_t(hg_graph* g, std::vector<Block>& owner, int64_t n) {
  return static_cast<T*>(dev_alloc(g, owner, (size_t)std::max<int64_t>(n, 1) * sizeof(T)));
}

// Wave members for load_impl: host arrays of nm + 1 union offsets, and the
// offset of the wave's first incidence in the caller's edge_ptr.
struct WaveInput {
  const int32_t* eoff;
  const int32_t* voff;
  int64_t base;
  // members stored apart (hg_load_batch_members): member q of the wave has its own
  // offsets m_eptr[q][0 .. ne_q] (from 0) and ids m_evtx[q]; noff = its first incidence
  const int64_t* const* m_eptr = nullptr;
  const int32_t* const* m_evtx = nullptr;
  const int64_t* noff = nullptr;
};

hg_status load_impl(hg_graph* g, const int64_t* edge_ptr, const int32_t* edge_vtx, int on_dev,
                    const WaveInput* wave = nullptr) {
  cudaStream_t s = g->stream;
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  g->small = alloc_t<Small>(g, g->load_blocks, 1);
  g->e_ptr = alloc_t<int64_t>(g, g->load_blocks, (int64_t)g->ne + 1);
  g->e_idx = alloc_t<int32_t>(g, g->load_blocks, g->nnz);
  g->esize = alloc_t<int32_t>(g, g->load_blocks, g->ne);
  g->v_ptr = alloc_t<int64_t>(g, g->load_blocks, (int64_t)g->nv + 1);
  g->v_idx = alloc_t<int32_t>(g, g->load_blocks, g->nnz);
  g->cand = alloc_t<int64_t>(g, g->load_blocks, g->ne);
  int32_t* vdeg = alloc_t<int32_t>(g, g->load_blocks, g->nv);
  const int64_t scan_n = std::max<int64_t>(std::max<int64_t>(g->nv, g->ne), 1);
  g->scan_tmp = dev_alloc(g, g->load_blocks, scan_tmp_bytes(scan_n));
  if (!g->small || !g->e_ptr || !g->e_idx || !g->esize || !g->v_ptr || !g->v_idx || !g->cand ||
      !vdeg || !g->scan_tmp)
    return HG_ERR_OOM;
  HG_CUDA(cudaMemsetAsync(g->small, 0, sizeof(Small), s));
  if (wave && wave->m_eptr) {
    // gather the members (in order: a member's last offset is overwritten by the next
    // member's first), then shift offsets by each member's first incidence
    for (int32_t q = 0; q < g->nm; ++q) {
      const int64_t ne_q = wave->eoff[q + 1] - wave->eoff[q];
      const int64_t nnz_q = wave->noff[q + 1] - wave->noff[q];
      HG_CUDA(cudaMemcpyAsync(g->e_ptr + wave->eoff[q], wave->m_eptr[q],
                              sizeof(int64_t) * (size_t)(ne_q + 1), kind, s));
      if (nnz_q > 0)
        HG_CUDA(cudaMemcpyAsync(g->e_idx + wave->noff[q], wave->m_evtx[q],
                                sizeof(int32_t) * (size_t)nnz_q, kind, s));
    }
  } else {
    HG_CUDA(cudaMemcpyAsync(g->e_ptr, edge_ptr, sizeof(int64_t) * ((size_t)g->ne + 1), kind, s));
    if (g->nnz > 0)
      HG_CUDA(cudaMemcpyAsync(g->e_idx, edge_vtx, sizeof(int32_t) * (size_t)g->nnz, kind, s));
  }
  if (wave) {
    g->m_eoff = alloc_t<int32_t>(g, g->load_blocks, (int64_t)g->nm + 1);
    g->m_voff = alloc_t<int32_t>(g, g->load_blocks, (int64_t)g->nm + 1);
    if (!g->m_eoff || !g->m_voff) return HG_ERR_OOM;
    HG_CUDA(cudaMemcpyAsync(g->m_eoff, wave->eoff, sizeof(int32_t) * ((size_t)g->nm + 1),
                            cudaMemcpyHostToDevice, s));
    HG_CUDA(cudaMemcpyAsync(g->m_voff, wave->voff, sizeof(int32_t) * ((size_t)g->nm + 1),
                            cudaMemcpyHostToDevice, s));
    if (wave->m_eptr) {
      int64_t* noff = alloc_t<int64_t>(g, g->load_blocks, (int64_t)g->nm + 1);
      if (!noff) return HG_ERR_OOM;
      HG_CUDA(cudaMemcpyAsync(noff, wave->noff, sizeof(int64_t) * ((size_t)g->nm + 1),
                              cudaMemcpyHostToDevice, s));
      launch_add_member_base(g->e_ptr, g->ne, g->m_eoff, g->nm, noff, s);
    } else {
      launch_sub_base(g->e_ptr, g->ne, wave->base, s);
    }
  }
  Small h;
  launch_check_ptr(g->e_ptr, g->ne, g->nnz, &g->small->err, s);
  HG_TRY(sync_small(g, &h));
  if (wave) {
    launch_localize(dev_graph(g), g->m_voff, g->e_idx, &g->small->err, s);
    HG_TRY(sync_small(g, &h));
  }
  HG_CUDA(cudaMemsetAsync(vdeg, 0, sizeof(int32_t) * (size_t)g->nv, s));
  DevGraph d = dev_graph(g);
  launch_validate_rows(d, g->esize, vdeg, &g->small->err, s);
  HG_TRY(sync_small(g, &h));
  scan_i32_to_i64(vdeg, g->v_ptr, g->nv, g->scan_tmp, s);
  HG_CUDA(cudaMemsetAsync(vdeg, 0, sizeof(int32_t) * (size_t)g->nv, s));  // reused as cursors
  launch_scatter(d, vdeg, g->v_idx, s);
  launch_candidates(d, g->cand, &g->small->max_cand, &g->small->max_size, s);
  HG_TRY(sync_small(g, &h));
  g->max_cand = (int64_t)h.max_cand;
  g->max_size = h.max_size;
  return HG_OK;
}

// Heavy x heavy hyperwedges on the tensor cores (dense tiles): choose the heavy set,
// fill its 0/1 e4m3 matrix, multiply.  Leaves dn->heavy_idx null when not used.
constexpr int64_t kDenseMinRows = 256;                  // below this a tile pass does not pay
constexpr int64_t kDenseMaxBytes = int64_t(8) << 30;    // matrix + omega budget

hg_status dense_impl(hg_graph* g, const hg_tuning* opt, DenseInfo* dn) {
  cudaStream_t s = g->stream;
  *dn = DenseInfo{};
  const int32_t want = opt ? opt->dense_min_size : 0;
  if (want < 0 || g->ne == 0) return HG_OK;
  const bool forced = want > 0;
  const int32_t min_size = forced ? want : 32;
  const int64_t cap = (opt && opt->dense_max_count > 0) ? opt->dense_max_count
                                                        : std::max<int64_t>(g->ne / 100, 1);
  if (g->max_size < min_size || min_size > kDenseMaxOmega) return HG_OK;
  // size histogram -> smallest threshold >= min_size keeping at most `cap` hyperedges of at
  // most kDenseMaxOmega vertices (the tile output holds omega in 16 bits); larger
  // hyperedges stay on the hash path
  const int32_t max_bin = std::min<int32_t>(g->max_size, kDenseMaxOmega + 1);
  unsigned long long* hist = alloc_t<unsigned long long>(g, g->build_blocks, (int64_t)max_bin + 1);
  if (!hist) return HG_ERR_OOM;
  HG_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * ((size_t)max_bin + 1), s));
  launch_size_hist(g->esize, g->ne, max_bin, hist, s);
  std::vector<unsigned long long> h((size_t)max_bin + 1);
  HG_CUDA(cudaMemcpyAsync(h.data(), hist, sizeof(unsigned long long) * h.size(),
                          cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaStreamSynchronize(s));
  int64_t above = 0;
  int32_t t = kDenseMaxOmega + 1;
  for (int32_t k = std::min<int32_t>(max_bin, kDenseMaxOmega); k >= min_size; --k) {
    if (above + (int64_t)h[k] > cap) break;
    above += (int64_t)h[k];
    t = k;
  }
  if (above == 0 || (!forced && above < kDenseMinRows)) return HG_OK;
  const int64_t rows_pad = dense_round_rows(above), k_pad = dense_round_k(g->nv);
  if (rows_pad * (k_pad + 2 * rows_pad) > kDenseMaxBytes) return HG_OK;   // stays on the hash path
  int32_t* heavy_idx = alloc_t<int32_t>(g, g->build_blocks, g->ne);
  int32_t* ids = alloc_t<int32_t>(g, g->build_blocks, above);
  uint8_t* a = alloc_t<uint8_t>(g, g->build_blocks, rows_pad * k_pad);
  uint16_t* omega = alloc_t<uint16_t>(g, g->build_blocks, rows_pad * rows_pad);
  if (!heavy_idx || !ids || !a || !omega) return HG_ERR_OOM;
  int32_t* count = g->small->counters + 8;
  HG_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t), s));
  HG_CUDA(cudaMemsetAsync(a, 0, (size_t)(rows_pad * k_pad), s));
  launch_pick_heavy(g->esize, g->ne, t, kDenseMaxOmega, (int32_t)above, heavy_idx, ids, count, s);
  launch_fill_dense(g->e_ptr, g->e_idx, ids, (int32_t)above, a, k_pad, s);
  t_begin(g, "dense_omega");
  HG_CUDA(launch_dense_omega(a, above, rows_pad, k_pad, omega, &g->small->err, s));
  t_end(g);
  Small hs;
  HG_TRY(sync_small(g, &hs));
  if (hs.counters[8] != (int32_t)above) return HG_ERR_INTERNAL;
  dn->heavy_idx = heavy_idx;
  dn->ids = ids;
  dn->omega = omega;
  dn->ld = rows_pad;
  dn->nh = (int32_t)above;
  return HG_OK;
}

hg_status free_graph(hg_graph* g);

// Drop what the samplers built on this handle (upper rows, Algorithm 7 rows, G').
void release_sampling(hg_graph* g) {
  release(g, g->sample_blocks);
  g->upper_built = false;
  g->adv_built = false;
  if (g->sub) {
    free_graph(g->sub);
    g->sub = nullptr;
  }
}

constexpr int64_t kOrientSlackBytes = int64_t(8) << 30;   // oriented rows with room for deg(i)

// The tuning fields that have a closed range (checked before a build changes anything).
bool tuning_ok(const hg_tuning* opt) {
  if (!opt) return true;
  const int32_t lm = opt->gather_light_max, wm = opt->warp_team_max;
  return opt->close_mode >= 0 && opt->close_mode <= 2 && opt->orient_exact >= 0 &&
         opt->orient_exact <= 1 && (lm == 0 || (lm >= 32 && lm <= wedge_light_max_cand(1))) &&
         (wm == 0 || wm == 64 || wm == 128 || wm == 256);
}

hg_status build_impl(hg_graph* g, const hg_tuning* opt, hg_wedge_stats* out) {
  // the gather and closure kernels keep a hyperedge's incidence prefix sums (the E_y
  // lists of its vertices, laid end to end) in 32 bits, and the heavy rows' tables use
  // 32-bit slot indices for twice a row's incidences
  if (g->max_cand >= (int64_t(1) << 30)) return HG_ERR_UNSUPPORTED;
  if (!opt && g->has_tuned) opt = &g->tuned;
  g->close_mode = opt ? opt->close_mode : 0;
  g->warp_team_max = (opt && opt->warp_team_max) ? opt->warp_team_max : 256;
  // (the packed flag is set below from the sizes; the same rule decides it here)
  const int packed_layout = (g->ne < (int64_t(1) << 24) && g->max_size < 256) ? 1 : 0;
  const int light_max = std::min((opt && opt->gather_light_max) ? opt->gather_light_max
                                                                 : wedge_light_max_cand(1),
                                 wedge_light_max_cand(packed_layout));
  cudaStream_t s = g->stream;
  release(g, g->count_blocks);
  release_sampling(g);
  release(g, g->build_blocks);
  g->built = false;
  g->counted = g->have_cstats = false;
  const int64_t ne = g->ne;
  const size_t ne1 = (size_t)std::max<int64_t>(ne, 1);
  g->packed = (ne < (int64_t(1) << 24) && g->max_size < 256) ? 1 : 0;
  Small h;
  HG_CUDA(cudaMemsetAsync(g->small, 0, sizeof(Small), s));
  g->deg = alloc_t<int32_t>(g, g->build_blocks, ne);
  int32_t* rows = alloc_t<int32_t>(g, g->build_blocks, 3 * ne);
  int32_t* cap = alloc_t<int32_t>(g, g->build_blocks, ne);
  g->cap_ptr = alloc_t<int64_t>(g, g->build_blocks, ne + 1);
  g->deg_ptr = alloc_t<int64_t>(g, g->build_blocks, ne + 1);
  g->ori.row_ptr = alloc_t<int64_t>(g, g->build_blocks, ne + 1);
  g->ori.dplus = alloc_t<int32_t>(g, g->build_blocks, ne);
  g->upc = alloc_t<int32_t>(g, g->build_blocks, ne);
  g->wcr = alloc_t<int32_t>(g, g->build_blocks, ne);
  if (!g->deg || !rows || !cap || !g->cap_ptr || !g->deg_ptr || !g->ori.row_ptr ||
      !g->ori.dplus || !g->upc || !g->wcr)
    return HG_ERR_OOM;
  g->mstats = nullptr;
  if (g->nm > 0) {
    g->mstats = alloc_t<unsigned long long>(g, g->build_blocks, 4 * (int64_t)g->nm);
    if (!g->mstats) return HG_ERR_OOM;
  }
  WedgeBuckets wb;
  for (int k = 0; k < 3; ++k) wb.rows[k] = rows + k * ne;
  wb.count = g->small->bucket_count;
  launch_bucket_rows(g->cand, g->ne, wb, light_max, s);
  // capacity layout of the gather pass: min(gathered incidences, |E| - 1) per row
  launch_cap_rows(g->cand, g->ne, cap, s);
  scan_i32_to_i64(cap, g->cap_ptr, ne, g->scan_tmp, s);
  int64_t total_cap = 0;
  HG_CUDA(cudaMemcpyAsync(&total_cap, g->cap_ptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HG_TRY(sync_small(g, &h));
  int32_t nb[3] = {h.bucket_count[0], h.bucket_count[1], h.bucket_count[2]};
  unsigned long long* scratch = nullptr;
  if (nb[2] > 0) {
    scratch = static_cast<unsigned long long*>(
        dev_alloc(g, g->build_blocks, wedge_heavy_scratch_bytes(g->max_cand, g->nsm)));
    if (!scratch) return HG_ERR_OOM;
  }
  g->cap_rows = Oriented{};
  g->cap_rows.row_ptr = g->cap_ptr;
  if (g->packed) {
    g->cap_rows.packed = alloc_t<uint32_t>(g, g->build_blocks, total_cap);
    if (!g->cap_rows.packed) return HG_ERR_OOM;
  } else {
    g->cap_rows.nbr = alloc_t<int32_t>(g, g->build_blocks, total_cap);
    g->cap_rows.omega = alloc_t<int32_t>(g, g->build_blocks, total_cap);
    if (!g->cap_rows.nbr || !g->cap_rows.omega) return HG_ERR_OOM;
  }
  DevGraph d = dev_graph(g);
  DenseInfo dn{};
  HG_TRY(dense_impl(g, opt, &dn));
  HG_CUDA(cudaMemsetAsync(g->deg, 0, sizeof(int32_t) * ne1, s));
  HG_CUDA(cudaMemsetAsync(g->upc, 0, sizeof(int32_t) * ne1, s));
  HG_CUDA(cudaMemsetAsync(g->wcr, 0, sizeof(int32_t) * ne1, s));
  HG_CUDA(cudaMemsetAsync(g->small->counters, 0, sizeof(int32_t) * 16, s));
  t_begin(g, "wedge_gather");
  launch_wedge_rows(d, wb, nb, g->max_cand, g->cand, g->deg, &g->small->wc, g->cap_rows, g->packed,
                    scratch,
                    &g->small->err, g->small->counters, dn, RowCounts{g->upc, g->wcr}, s, g->nsm);
  t_end(g);
  // orientation by (deg, id).  Out-lists go to rows with room for deg(i) entries (offsets
  // = the scan of deg, one filter pass) while 2W slots fit kOrientSlackBytes; beyond that
  // to an exact layout (a counting pass, its scan, then the filter pass).
  t_begin(g, "wedge_orient");
  scan_i32_to_i64(g->deg, g->deg_ptr, ne, g->scan_tmp, s);
  reduce_deg_stats(g->deg, ne, g->small->deg_stats, s);
  t_end(g);
  int64_t two_w = 0;
  HG_CUDA(cudaMemcpyAsync(&two_w, g->deg_ptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HG_TRY(sync_small(g, &h));
  g->two_w = (uint64_t)two_w;
  const int64_t entry_bytes = g->packed ? 4 : 8;
  const bool exact = (opt && opt->orient_exact) || two_w * entry_bytes > kOrientSlackBytes;
  int64_t slots = two_w;
  if (exact) {
    t_begin(g, "wedge_orient");
    launch_filter_rows(0, true, g->cap_ptr, g->deg, g->cap_rows, g->deg, g->ne, g->packed,
                       nullptr, Oriented{}, g->ori.dplus, s);
    scan_i32_to_i64(g->ori.dplus, g->ori.row_ptr, ne, g->scan_tmp, s);
    t_end(g);
    HG_CUDA(cudaMemcpyAsync(&slots, g->ori.row_ptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HG_CUDA(cudaStreamSynchronize(s));
  } else {
    HG_CUDA(cudaMemcpyAsync(g->ori.row_ptr, g->deg_ptr, sizeof(int64_t) * ((size_t)ne + 1),
                            cudaMemcpyDeviceToDevice, s));
  }
  g->ori.slots = slots;
  if (g->packed) {
    g->ori.packed = alloc_t<uint32_t>(g, g->build_blocks, slots);
    if (!g->ori.packed) return HG_ERR_OOM;
  } else {
    g->ori.nbr = alloc_t<int32_t>(g, g->build_blocks, slots);
    g->ori.omega = alloc_t<int32_t>(g, g->build_blocks, slots);
    if (!g->ori.nbr || !g->ori.omega) return HG_ERR_OOM;
  }
  t_begin(g, "wedge_emit");
  launch_filter_rows(0, false, g->cap_ptr, g->deg, g->cap_rows, g->deg, g->ne, g->packed,
                     g->ori.row_ptr, g->ori, exact ? nullptr : g->ori.dplus, s);
  reduce_deg_stats(g->ori.dplus, ne, g->small->out_stats, s);
  t_end(g);
  if (g->nm > 0) {
    g->h_mstats.assign(4 * (size_t)g->nm, 0);
    launch_member_stats(d, g->deg, g->wcr, g->mstats, s);
    HG_CUDA(cudaMemcpyAsync(g->h_mstats.data(), g->mstats, sizeof(unsigned long long) * g->h_mstats.size(),
                            cudaMemcpyDeviceToHost, s));
  }
  HG_TRY(sync_small(g, &h));
  t_collect(g);
  hg_wedge_stats& st = g->stats;
  std::memset(&st, 0, sizeof(st));
  st.W = (uint64_t)two_w / 2;
  st.W_c = h.wc;
  st.W_t = st.W - st.W_c;
  st.connected = h.deg_stats[0];
  st.max_deg = h.deg_stats[1];
  st.max_out_deg = h.out_stats[1];
  st.dense_edges = (uint64_t)dn.nh;
  if (h.deg_stats[2] != (unsigned long long)two_w || h.out_stats[2] != st.W ||
      (exact && (uint64_t)slots != st.W) || (two_w & 1) || two_w > total_cap)
    return HG_ERR_INTERNAL;
  g->dn = dn;
  g->built = true;
  if (out) *out = st;
  return HG_OK;
}

// Rows of neighbours j > i with omega_ij, sorted by j: the hyperwedges in the
// order O of Sec. 2, row i starting at up_ptr[i].  Built on the first sampling call.
hg_status upper_impl(hg_graph* g) {
  cudaStream_t s = g->stream;
  const int64_t ne = g->ne;
  release(g, g->sample_blocks);
  g->up_ptr = alloc_t<int64_t>(g, g->sample_blocks, ne + 1);
  if (!g->up_ptr) return HG_ERR_OOM;
  scan_i32_to_i64(g->upc, g->up_ptr, ne, g->scan_tmp, s);
  int64_t w = 0;
  HG_CUDA(cudaMemcpyAsync(&w, g->up_ptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaStreamSynchronize(s));
  if ((uint64_t)w != g->stats.W) return HG_ERR_INTERNAL;
  g->up = Oriented{};
  g->up.row_ptr = g->up_ptr;
  if (g->packed) {
    g->up.packed = alloc_t<uint32_t>(g, g->sample_blocks, w);
    if (!g->up.packed) return HG_ERR_OOM;
  } else {
    g->up.nbr = alloc_t<int32_t>(g, g->sample_blocks, w);
    g->up.omega = alloc_t<int32_t>(g, g->sample_blocks, w);
    if (!g->up.nbr || !g->up.omega) return HG_ERR_OOM;
  }
  t_begin(g, "upper_emit");
  launch_filter_rows(1, false, g->cap_ptr, g->deg, g->cap_rows, g->deg, g->ne, g->packed,
                     g->up_ptr, g->up, nullptr, s);
  t_end(g);
  t_begin(g, "upper_sort");
  HG_CUDA(launch_sort_upper(g->up_ptr, g->ne, g->up, g->packed, &g->small->err, s, g->nsm));
  t_end(g);
  g->up_index = alloc_t<int32_t>(g, g->sample_blocks,
                                 row_index_buckets(g->stats.W, row_index_shift(g->stats.W, g->ne)) + 1);
  if (!g->up_index) return HG_ERR_OOM;
  launch_row_index(g->up_ptr, g->ne, g->stats.W, g->up_index, s);
  Small h;
  HG_TRY(sync_small(g, &h));
  t_collect(g);
  g->upper_built = true;
  return HG_OK;
}

// Algorithm 7's rows: the upper rows split by hyperwedge type (order kept), and
// every neighbour row N(i) sorted by id (offsets: the scan of the full degrees).
hg_status adv_impl(hg_graph* g) {
  if (!g->upper_built) HG_TRY(upper_impl(g));
  cudaStream_t s = g->stream;
  const int64_t ne = g->ne;
  int32_t* cnt_t = alloc_t<int32_t>(g, g->sample_blocks, ne);
  g->t_ptr = alloc_t<int64_t>(g, g->sample_blocks, ne + 1);
  g->c_ptr = alloc_t<int64_t>(g, g->sample_blocks, ne + 1);
  if (!cnt_t || !g->t_ptr || !g->c_ptr) return HG_ERR_OOM;
  launch_type_counts(g->upc, g->wcr, g->ne, cnt_t, s);
  scan_i32_to_i64(cnt_t, g->t_ptr, ne, g->scan_tmp, s);
  scan_i32_to_i64(g->wcr, g->c_ptr, ne, g->scan_tmp, s);
  int64_t wt = 0, wc = 0;
  HG_CUDA(cudaMemcpyAsync(&wt, g->t_ptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaMemcpyAsync(&wc, g->c_ptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaStreamSynchronize(s));
  if ((uint64_t)wt + (uint64_t)wc != g->stats.W || (uint64_t)wc != g->stats.W_c) return HG_ERR_INTERNAL;
  g->Wt = (uint64_t)wt;
  g->Wc = (uint64_t)wc;
  g->t_ent = Oriented{};
  g->c_ent = Oriented{};
  g->full = Oriented{};
  g->full.row_ptr = g->deg_ptr;
  if (g->packed) {
    g->t_ent.packed = alloc_t<uint32_t>(g, g->sample_blocks, wt);
    g->c_ent.packed = alloc_t<uint32_t>(g, g->sample_blocks, wc);
    g->full.packed = alloc_t<uint32_t>(g, g->sample_blocks, (int64_t)g->two_w);
    if (!g->t_ent.packed || !g->c_ent.packed || !g->full.packed) return HG_ERR_OOM;
  } else {
    g->t_ent.nbr = alloc_t<int32_t>(g, g->sample_blocks, wt);
    g->t_ent.omega = alloc_t<int32_t>(g, g->sample_blocks, wt);
    g->c_ent.nbr = alloc_t<int32_t>(g, g->sample_blocks, wc);
    g->c_ent.omega = alloc_t<int32_t>(g, g->sample_blocks, wc);
    g->full.nbr = alloc_t<int32_t>(g, g->sample_blocks, (int64_t)g->two_w);
    g->full.omega = alloc_t<int32_t>(g, g->sample_blocks, (int64_t)g->two_w);
    if (!g->t_ent.nbr || !g->t_ent.omega || !g->c_ent.nbr || !g->c_ent.omega || !g->full.nbr ||
        !g->full.omega)
      return HG_ERR_OOM;
  }
  DevGraph d = dev_graph(g);
  t_begin(g, "adv_split");
  launch_split_types(d, g->up_ptr, g->up, g->packed, g->t_ptr, g->t_ent, g->c_ptr, g->c_ent, s);
  t_end(g);
  g->t_index = alloc_t<int32_t>(g, g->sample_blocks,
                                row_index_buckets(g->Wt, row_index_shift(g->Wt, g->ne)) + 1);
  g->c_index = alloc_t<int32_t>(g, g->sample_blocks,
                                row_index_buckets(g->Wc, row_index_shift(g->Wc, g->ne)) + 1);
  if (!g->t_index || !g->c_index) return HG_ERR_OOM;
  launch_row_index(g->t_ptr, g->ne, g->Wt, g->t_index, s);
  launch_row_index(g->c_ptr, g->ne, g->Wc, g->c_index, s);
  t_begin(g, "full_emit");
  launch_filter_rows(2, false, g->cap_ptr, g->deg, g->cap_rows, g->deg, g->ne, g->packed,
                     g->deg_ptr, g->full, nullptr, s);
  t_end(g);
  t_begin(g, "full_sort");
  HG_CUDA(launch_sort_upper(g->deg_ptr, g->ne, g->full, g->packed, &g->small->err, s, g->nsm));
  t_end(g);
  Small h;
  HG_TRY(sync_small(g, &h));
  t_collect(g);
  g->adv_built = true;
  return HG_OK;
}

// G' (Algorithms 6-7, the sigma|E| draw): the ceil(sigma |E|) hyperedges with the smallest Philox
// priorities (ties by id), renumbered in id order, as a handle of its own with step one
// built.  The k-th smallest priority is found by a 4-pass radix select (16-bit digits).
hg_status subgraph_impl(hg_graph* g, uint64_t seed, double sigma) {
  if (g->sub && g->sub_seed == seed && g->sub_sigma == sigma) return HG_OK;
  if (g->sub) {
    free_graph(g->sub);
    g->sub = nullptr;
  }
  cudaStream_t s = g->stream;
  const int32_t ne = g->ne;
  const int64_t keep = (int64_t)std::ceil(sigma * (double)ne);
  std::vector<Block> tmp;
  struct Releaser {
    hg_graph* g;
    std::vector<Block>& b;
    ~Releaser() { release(g, b); }
  } rel{g, tmp};
  unsigned long long* pr = alloc_t<unsigned long long>(g, tmp, ne);
  unsigned int* hist = alloc_t<unsigned int>(g, tmp, 65536);
  int32_t* flags = alloc_t<int32_t>(g, tmp, ne);
  int64_t* rank = alloc_t<int64_t>(g, tmp, (int64_t)ne + 1);
  int32_t* ids = alloc_t<int32_t>(g, tmp, keep);
  int32_t* sizes = alloc_t<int32_t>(g, tmp, keep);
  int64_t* sub_ptr = alloc_t<int64_t>(g, tmp, keep + 1);
  if (!pr || !hist || !flags || !rank || !ids || !sizes || !sub_ptr) return HG_ERR_OOM;
  launch_priority(ne, seed, pr, s);
  unsigned long long prefix = 0, pmask = 0;
  int64_t less = 0;   // priorities below the current prefix range
  std::vector<unsigned int> h(65536);
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 48 - 16 * pass;
    HG_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned int) * 65536, s));
    launch_digit_hist(pr, ne, shift, pmask, prefix, hist, s);
    HG_CUDA(cudaMemcpyAsync(h.data(), hist, sizeof(unsigned int) * 65536, cudaMemcpyDeviceToHost, s));
    HG_CUDA(cudaStreamSynchronize(s));
    int64_t cum = 0;
    int d = 0;
    for (; d < 65536; ++d) {
      if (less + cum + (int64_t)h[(size_t)d] >= keep) break;
      cum += h[(size_t)d];
    }
    if (d == 65536) return HG_ERR_INTERNAL;
    less += cum;
    prefix |= (unsigned long long)d << shift;
    pmask |= 0xffffull << shift;
  }
  const unsigned long long T = prefix;   // the keep-th smallest priority
  const int64_t need = keep - less;      // how many priorities equal to T are kept
  launch_equal_flags(pr, ne, T, flags, s);
  scan_i32_to_i64(flags, rank, ne, g->scan_tmp, s);
  launch_keep_flags(pr, ne, T, rank, need, flags, s);
  scan_i32_to_i64(flags, rank, ne, g->scan_tmp, s);
  launch_compact_kept(flags, rank, g->esize, ne, ids, sizes, s);
  int64_t kept = 0;
  HG_CUDA(cudaMemcpyAsync(&kept, rank + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaStreamSynchronize(s));
  if (kept != keep) return HG_ERR_INTERNAL;
  scan_i32_to_i64(sizes, sub_ptr, keep, g->scan_tmp, s);
  int64_t nnz = 0;
  HG_CUDA(cudaMemcpyAsync(&nnz, sub_ptr + keep, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaStreamSynchronize(s));
  int32_t* sub_idx = alloc_t<int32_t>(g, tmp, nnz);
  if (!sub_idx) return HG_ERR_OOM;
  launch_gather_rows(g->e_ptr, g->e_idx, ids, (int32_t)keep, sub_ptr, sub_idx, s);
  hg_graph* sub = new hg_graph();
  sub->device = g->device;
  sub->nsm = g->nsm;
  sub->stream = s;
  sub->nv = g->nv;
  sub->ne = (int32_t)keep;
  sub->nnz = nnz;
  hg_status st = load_impl(sub, sub_ptr, sub_idx, 1);
  if (st == HG_OK) st = build_impl(sub, nullptr, nullptr);
  if (st != HG_OK) {
    cudaStreamSynchronize(s);
    free_graph(sub);
    return st;
  }
  g->sub = sub;
  g->sub_seed = seed;
  g->sub_sigma = sigma;
  return HG_OK;
}

hg_status sample_adv_impl(hg_graph* g, uint64_t seed, uint64_t first, uint64_t num, double sigma,
                          uint32_t class_mask, uint64_t raw[21], double est[21], uint64_t info[8]) {
  if (!g->adv_built) HG_TRY(adv_impl(g));
  cudaStream_t s = g->stream;
  uint8_t lut[128];
  build_lut(lut);
  sample_set_lut(lut, s);
  const uint64_t Wt = g->Wt, Wc = g->Wc, W = Wt + Wc;
  uint64_t alpha[4] = {0, 0, 0, 0};
  if (W > 0) {   // Algorithm 7's sample split: exact floors
    const unsigned __int128 den = (unsigned __int128)W * W;
    alpha[0] = (uint64_t)((unsigned __int128)Wt * Wt * num / den);
    alpha[1] = (uint64_t)((unsigned __int128)Wc * Wc * num / den);
    alpha[2] = alpha[3] = (uint64_t)((unsigned __int128)Wt * Wc * num / den);
  }
  static const int kType[4] = {0, 1, 0, 1};    // intersection, inclusion, intersection, inclusion
  static const int kClass[4] = {3, 0, 2, 1};   // TTT, CCC, TTC, TCC
  static const int kClassOf[21] = {-1, 0, 1, 1, 1, 1, 2, 2, 2, 3, 3, 3,
                                   3,  3, 3, 3, 3, 3, 3, 3, 3};
  if (info) {
    info[0] = W;
    info[1] = Wt;
    info[2] = Wc;
    for (int x = 0; x < 4; ++x) info[3 + x] = alpha[x];
    info[7] = (uint64_t)g->ne;
  }
  for (int p = 0; p <= 20; ++p) {
    raw[p] = 0;
    est[p] = 0.0;
  }
  DevGraph d = dev_graph(g);
  const double s3 = sigma * sigma * sigma;
  for (int x = 0; x < 4; ++x) {
    if (!(class_mask >> kClass[x] & 1u) || alpha[x] == 0) continue;
    const bool incl = kType[x] == 1;
    const uint64_t Wx = incl ? Wc : Wt;
    HG_CUDA(cudaMemsetAsync(g->small->hist, 0, sizeof(g->small->hist), s));
    t_begin(g, "sample_adv");
    launch_sample_adv(d, incl ? g->c_ptr : g->t_ptr, incl ? g->c_index : g->t_index,
                      incl ? g->c_ent : g->t_ent, Wx, kType[x], kClass[x], (uint32_t)(1 + x),
                      g->deg_ptr, g->full, g->packed, seed, first, alpha[x], g->small->hist,
                      s, g->nsm);
    t_end(g);
    Small h;
    HG_TRY(sync_small(g, &h));
    if (h.hist[0] != 0) return HG_ERR_INTERNAL;
    const double scale = (double)Wx / (double)alpha[x];
    for (int p = 1; p <= 20; ++p) {
      if (kClassOf[p] != kClass[x]) {
        if (h.hist[p] != 0) return HG_ERR_INTERNAL;
        continue;
      }
      raw[p] = h.hist[p];
      est[p] = ((double)h.hist[p] * scale) / s3;
    }
  }
  t_collect(g);
  for (int p = 1; p <= 20; ++p) {
    raw[0] += raw[p];
    est[0] += est[p];
  }
  return HG_OK;
}

hg_status sample_impl(hg_graph* g, uint64_t seed, uint64_t first, uint64_t num, double sigma,
                      uint64_t raw[21], double est[21]) {
  if (!g->upper_built) HG_TRY(upper_impl(g));
  cudaStream_t s = g->stream;
  uint8_t lut[128];
  build_lut(lut);
  sample_set_lut(lut, s);
  HG_CUDA(cudaMemsetAsync(g->small->hist, 0, sizeof(g->small->hist), s));
  HG_CUDA(cudaMemsetAsync(g->small->sample_work, 0, sizeof(g->small->sample_work), s));
  DevGraph d = dev_graph(g);
  t_begin(g, "sample");
  launch_sample(d, g->up_ptr, g->up_index, g->up, g->packed, g->stats.W, seed, first, num,
                g->small->hist, g->small->sample_work, s, g->nsm);
  t_end(g);
  Small h;
  HG_TRY(sync_small(g, &h));
  t_collect(g);
  if (h.hist[0] != 0) return HG_ERR_INTERNAL;
  for (int k = 0; k < 3; ++k) g->sample_work[k] = h.sample_work[k];
  uint64_t total = 0;
  for (int p = 1; p <= 20; ++p) total += h.hist[p];
  raw[0] = total;
  for (int p = 1; p <= 20; ++p) raw[p] = h.hist[p];
  // Algorithm 6: each drawn hyperwedge stands for W / num of them; each hyper-triangle
  // survives the vertex sampling of rate sigma with probability sigma^3
  const double scale = num ? (double)g->stats.W / (double)num : 0.0;
  const double s3 = sigma * sigma * sigma;
  for (int p = 0; p <= 20; ++p) est[p] = num ? ((double)raw[p] * scale) / s3 : 0.0;
  return HG_OK;
}

// h_sel: NULL (every hyper-triangle), or one host byte per hyperedge: then only the
// hyper-triangles owned by the hyperedges u with h_sel[u] != 0 (their teams alone run).
hg_status count_impl(hg_graph* g, uint64_t counts[21], const uint8_t* h_sel = nullptr) {
  cudaStream_t s = g->stream;
  release(g, g->count_blocks);
  g->counted = g->have_cstats = false;
  const int64_t ne = g->ne;
  Small h;
  int32_t* lists = alloc_t<int32_t>(g, g->count_blocks, (kCloseBuckets + 1) * ne);  // + overflow
  if (!lists) return HG_ERR_OOM;
  uint8_t* sel = nullptr;
  if (h_sel) {
    sel = alloc_t<uint8_t>(g, g->count_blocks, std::max<int64_t>(ne, 1));
    if (!sel) return HG_ERR_OOM;
    HG_CUDA(cudaMemcpyAsync(sel, h_sel, (size_t)ne, cudaMemcpyHostToDevice, s));
  }
  HG_CUDA(cudaMemsetAsync(g->small->bucket_count + 3, 0, sizeof(int32_t) * (1 + kCloseBuckets), s));
  HG_CUDA(cudaMemsetAsync(g->small->wide_max, 0, sizeof(g->small->wide_max), s));
  HG_CUDA(cudaMemsetAsync(g->small->hist, 0, sizeof(g->small->hist), s));
  HG_CUDA(cudaMemsetAsync(g->small->work, 0, sizeof(g->small->work), s));
  HG_CUDA(cudaMemsetAsync(g->small->counters, 0, sizeof(int32_t) * 16, s));
  // pattern bins: one set per member of a batch wave, else the handle's own
  unsigned long long* hist = g->small->hist;
  if (g->nm > 0) {
    g->mhist = alloc_t<unsigned long long>(g, g->count_blocks, (int64_t)g->nm * 128);
    if (!g->mhist) return HG_ERR_OOM;
    HG_CUDA(cudaMemsetAsync(g->mhist, 0, sizeof(unsigned long long) * 128 * (size_t)g->nm, s));
    hist = g->mhist;
  }
  CloseBuckets cb;
  for (int k = 0; k < kCloseBuckets; ++k) cb.lists[k] = lists + k * ne;
  cb.count = g->small->bucket_count + 4;
  int32_t* overflow = lists + kCloseBuckets * ne;
  int32_t* n_overflow = g->small->bucket_count + 3;
  DevGraph d = dev_graph(g);
  t_begin(g, "close_bucket");
  // warp tables keep |e_x| in 16 bits: larger hyperedges send everything to block teams
  launch_bucket_close(d, g->ori, cb, g->small->wide_max,
                      g->close_mode == 1 || g->max_size >= 65536, g->warp_team_max,
                      g->packed ? kBlockMaxPacked : kBlockMaxUnpacked, sel, s);
  t_end(g);
  HG_TRY(sync_small(g, &h));
  int32_t n[kCloseBuckets];
  for (int k = 0; k < kCloseBuckets; ++k) n[k] = h.bucket_count[4 + k];
  // block-kernel scratch: any out-degree and |e_u| of bucket 3, and the warp
  // and block buckets' limits (the largest out-degree of a non-empty one, |e_u| 32) for
  // hyperedges they hand over
  int64_t team_dmax = 256;
  for (int k = 3; k < kWideBucket; ++k)
    if (n[k] > 0)
      team_dmax = k < 5 ? int64_t(1024) << (k - 3) : (g->packed ? kBlockMaxPacked : kBlockMaxUnpacked);
  const int64_t dmax = std::max<int64_t>((int64_t)h.wide_max[0], team_dmax);
  const int64_t words = std::max<int64_t>(((int64_t)h.wide_max[1] + 31) / 32, 1);
  int64_t cap = 16;
  while (cap < 2 * dmax) cap *= 2;
  void* scratch = dev_alloc(g, g->count_blocks, close_wide_scratch_bytes(cap, words, dmax, g->nsm));
  if (!scratch) return HG_ERR_OOM;
  static const char* names[kCloseBuckets] = {"close_warp256",   "close_warp512",
                                             "close_warp1024",  "close_block2048",
                                             "close_block4096", "close_block8192",
                                             "close_wide",      "close_cluster"};
  for (int k = kCloseBuckets - 1; k >= 0; --k) {
    if (n[k] <= 0) continue;
    t_begin(g, names[k]);
    launch_close(k, d, g->ori, g->packed, cb.lists[k], n[k], cb.count + k, cap, words, dmax,
                 scratch, hist, g->small->work[k], g->small->counters + k, overflow,
                 n_overflow, g->close_mode == 2 ? 1 : 0, s, g->nsm);
    t_end(g);
  }
  HG_TRY(sync_small(g, &h));
  const int32_t n_over = h.bucket_count[3];
  if (n_over > 0) {
    t_begin(g, "close_wide");
    launch_close(kWideBucket, d, g->ori, g->packed, overflow, n_over, n_overflow, cap, words, dmax,
                 scratch, hist, g->small->work[kWideBucket], g->small->counters + 8,
                 overflow, n_overflow, 0, s, g->nsm);
    t_end(g);
    HG_TRY(sync_small(g, &h));
  }
  t_collect(g);
  if (g->nm > 0) {   // per member, and the wave's bins as the sums of its members'
    std::vector<unsigned long long> lab(128 * (size_t)g->nm);
    HG_CUDA(cudaMemcpyAsync(lab.data(), g->mhist, sizeof(unsigned long long) * lab.size(),
                            cudaMemcpyDeviceToHost, s));
    HG_CUDA(cudaStreamSynchronize(s));
    g->h_mmasks.assign(128 * (size_t)g->nm, 0);
    for (int k = 0; k < 128; ++k) h.hist[k] = 0;
    uint64_t unused[21];
    for (int32_t m = 0; m < g->nm; ++m) {
      if (!fold_masks(lab.data() + 128 * (size_t)m, g->h_mmasks.data() + 128 * (size_t)m, unused))
        return HG_ERR_INTERNAL;
      for (int k = 0; k < 128; ++k) h.hist[k] += lab[128 * (size_t)m + k];
    }
  }
  if (!fold_masks(h.hist, g->masks, g->counts)) return HG_ERR_INTERNAL;
  std::memset(&g->cstats, 0, sizeof(g->cstats));
  for (int k = 0; k < kCloseBuckets; ++k) {
    g->cstats.bucket_probes[k] = h.work[k][0];
    g->cstats.bucket_gathers[k] = h.work[k][1];
    g->cstats.bucket_out_entries[k] = h.work[k][2];
    g->cstats.probes += h.work[k][0];
    g->cstats.gathers += h.work[k][1];
    g->cstats.out_entries += h.work[k][2];
  }
  for (int k = 0; k < kCloseBuckets; ++k) {
    g->cstats.bucket_teams[k] = (uint64_t)n[k];
    g->cstats.teams += (uint64_t)n[k];
  }
  g->cstats.bucket_teams[kWideBucket] += (uint64_t)n_over;   // handed from the warp kernels
  g->counted = true;
  g->have_cstats = true;
  if (counts) std::memcpy(counts, g->counts, sizeof(g->counts));
  return HG_OK;
}

// ---------------------------------------------------------------- autotuner
//
// Coordinate descent over the tuning fields whose best value depends on the input:
// starting from the defaults, each field in turn takes each of its other values with
// the others at the best so far, and keeps a value that lowers the measured time of
// step one plus step two (CUDA events on the handle's stream around hg_build_wedges and
// hg_count_patterns).  Every candidate must give the same counts, canonical mask
// histogram and wedge statistics; the handle ends built and counted with the choice.

struct TuneRun {
  hg_tuning t;
  float ms;
  uint64_t counts[21];
  uint64_t masks[128];
  hg_wedge_stats st;
};

hg_status time_candidate(hg_graph* g, const hg_tuning& t, TuneRun* r) {
  r->t = t;
  cudaEvent_t a = nullptr, b = nullptr;
  HG_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return HG_ERR_CUDA;
  }
  hg_status st = cuda_status(cudaEventRecord(a, g->stream));
  if (st == HG_OK) st = build_impl(g, &t, &r->st);
  if (st == HG_OK) st = count_impl(g, r->counts);
  if (st == HG_OK) st = cuda_status(cudaEventRecord(b, g->stream));
  if (st == HG_OK) st = cuda_status(cudaEventSynchronize(b));
  if (st == HG_OK) st = cuda_status(cudaEventElapsedTime(&r->ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::memcpy(r->masks, g->masks, sizeof(g->masks));
  return st;
}

bool same_result(const TuneRun& x, const TuneRun& y) {
  return std::memcmp(x.counts, y.counts, sizeof(x.counts)) == 0 &&
         std::memcmp(x.masks, y.masks, sizeof(x.masks)) == 0 && x.st.W == y.st.W &&
         x.st.W_c == y.st.W_c && x.st.connected == y.st.connected && x.st.max_deg == y.st.max_deg;
}

hg_status autotune_impl(hg_graph* g, hg_autotune_result* out) {
  std::vector<TuneRun> runs;
  auto run = [&](const hg_tuning& t) -> hg_status {
    if ((int)runs.size() >= HG_AUTOTUNE_MAX) return HG_OK;
    runs.emplace_back();
    HG_TRY(time_candidate(g, t, &runs.back()));
    if (!same_result(runs.front(), runs.back())) return HG_ERR_INTERNAL;
    return HG_OK;
  };
  hg_tuning best{};
  HG_TRY(run(best));
  size_t best_i = 0;
  // the fields, each with the values it may take besides the default (0)
  struct Knob {
    int32_t hg_tuning::*field;
    std::vector<int32_t> alts;
  };
  std::vector<Knob> knobs = {
      {&hg_tuning::warp_team_max, {128, 64}},
      {&hg_tuning::gather_light_max, {256, 128}},
      {&hg_tuning::orient_exact, {1}},
  };
  if (g->max_size >= 32) knobs.push_back({&hg_tuning::dense_min_size, {-1, 64}});
  for (const Knob& k : knobs) {
    const hg_tuning base = best;
    for (int32_t v : k.alts) {
      hg_tuning t = base;
      t.*(k.field) = v;
      const size_t before = runs.size();
      HG_TRY(run(t));
      if (runs.size() > before && runs.back().ms < runs[best_i].ms) {
        best = t;
        best_i = runs.size() - 1;
      }
    }
  }
  // leave the handle built and counted with the choice
  TuneRun last;
  HG_TRY(time_candidate(g, best, &last));
  if (!same_result(runs.front(), last)) return HG_ERR_INTERNAL;
  g->tuned = best;
  g->has_tuned = true;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->best = best;
    out->best_ms = runs[best_i].ms;
    out->best_index = (int32_t)best_i;
    out->num_tried = (int32_t)runs.size();
    for (size_t k = 0; k < runs.size(); ++k) {
      out->tried[k] = runs[k].t;
      out->ms[k] = runs[k].ms;
      std::memcpy(out->counts[k], runs[k].counts, sizeof(runs[k].counts));
    }
  }
  return HG_OK;
}

}  // namespace

// A batch: member hypergraphs grouped into waves, each wave one union handle.
struct hg_batch {
  cudaStream_t stream = nullptr;
  int32_t G = 0;
  std::vector<hg_graph*> waves;
  std::vector<int32_t> first;   // first member of each wave (+ G at the end)
  bool built = false, counted = false;
};

namespace {

hg_status free_graph(hg_graph* g) {
  cudaStream_t s = g->stream;
  release(g, g->count_blocks);
  release_sampling(g);
  release(g, g->build_blocks);
  release(g, g->load_blocks);
  cudaError_t e = cudaStreamSynchronize(s);
  for (auto& k : g->pending) {
    cudaEventDestroy(k.a);
    cudaEventDestroy(k.b);
  }
  delete g;
  return cuda_status(e);
}

void free_batch(hg_batch* b) {
  for (hg_graph* w : b->waves) free_graph(w);
  delete b;
}

constexpr int64_t kDefaultWaveEdges = (int64_t(1) << 24) - 1;   // packed 24-bit neighbour ids

// member_ptr/member_vtx (both or neither): members stored apart, member m's offsets
// member_ptr[m][0 .. ne_m] from 0; otherwise the concatenated edge_ptr / edge_vtx.
hg_status load_batch_impl(hg_batch* b, const int32_t* num_vertices, const int64_t* edge_off,
                          const int64_t* edge_ptr, const int32_t* edge_vtx, int on_dev,
                          int64_t max_wave_edges, int dev, int nsm,
                          const int64_t* const* member_ptr = nullptr,
                          const int32_t* const* member_vtx = nullptr,
                          const int64_t* member_nnz = nullptr) {
  cudaStream_t s = b->stream;
  const int32_t G = b->G;
  // greedy waves of consecutive members: at most max_wave_edges hyperedges (a
  // larger member gets a wave of its own) and fewer than 2^31 union vertices
  int32_t m = 0;
  while (m < G) {
    const int32_t m0 = m;
    int64_t ne = 0, nv = 0;
    while (m < G) {
      const int64_t dne = edge_off[m + 1] - edge_off[m], dnv = num_vertices[m];
      if (m > m0 && (ne + dne > max_wave_edges || nv + dnv > INT32_MAX)) break;
      ne += dne;
      nv += dnv;
      ++m;
    }
    if (ne > INT32_MAX || nv > INT32_MAX) return HG_ERR_UNSUPPORTED;
    b->first.push_back(m0);
  }
  b->first.push_back(G);
  for (size_t k = 0; k + 1 < b->first.size(); ++k) {
    const int32_t m0 = b->first[k], m1 = b->first[k + 1];
    const int64_t e0 = edge_off[m0], e1 = edge_off[m1];
    int64_t p0 = 0, p1 = 0;
    if (member_ptr) {
      std::vector<int32_t> eoff((size_t)(m1 - m0) + 1), voff((size_t)(m1 - m0) + 1);
      std::vector<int64_t> noff((size_t)(m1 - m0) + 1);
      int64_t nv = 0, nnz = 0;
      for (int32_t q = m0; q <= m1; ++q) {
        eoff[(size_t)(q - m0)] = (int32_t)(edge_off[q] - e0);
        voff[(size_t)(q - m0)] = (int32_t)nv;
        noff[(size_t)(q - m0)] = nnz;
        if (q < m1) {
          nv += num_vertices[q];
          nnz += member_nnz[q];
        }
      }
      hg_graph* g = new hg_graph();
      g->device = dev;
      g->nsm = nsm;
      g->stream = s;
      g->nv = (int32_t)std::max<int64_t>(nv, 1);
      g->ne = (int32_t)(e1 - e0);
      g->nnz = nnz;
      g->nm = m1 - m0;
      b->waves.push_back(g);
      WaveInput wi{eoff.data(), voff.data(), 0, member_ptr + m0, member_vtx + m0, noff.data()};
      HG_TRY(load_impl(g, nullptr, nullptr, on_dev, &wi));
      continue;
    }
    if (on_dev) {
      HG_CUDA(cudaMemcpyAsync(&p0, edge_ptr + e0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      HG_CUDA(cudaMemcpyAsync(&p1, edge_ptr + e1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      HG_CUDA(cudaStreamSynchronize(s));
    } else {
      p0 = edge_ptr[e0];
      p1 = edge_ptr[e1];
    }
    if (p0 < 0 || p1 < p0 || (p1 > p0 && !edge_vtx)) return HG_ERR_INVALID_ARG;
    std::vector<int32_t> eoff((size_t)(m1 - m0) + 1), voff((size_t)(m1 - m0) + 1);
    int64_t nv = 0;
    for (int32_t q = m0; q <= m1; ++q) {
      eoff[(size_t)(q - m0)] = (int32_t)(edge_off[q] - e0);
      voff[(size_t)(q - m0)] = (int32_t)nv;
      if (q < m1) nv += num_vertices[q];
    }
    hg_graph* g = new hg_graph();
    g->device = dev;
    g->nsm = nsm;
    g->stream = s;
    g->nv = (int32_t)std::max<int64_t>(nv, 1);
    g->ne = (int32_t)(e1 - e0);
    g->nnz = p1 - p0;
    g->nm = m1 - m0;
    b->waves.push_back(g);
    WaveInput wi{eoff.data(), voff.data(), p0};
    HG_TRY(load_impl(g, edge_ptr + e0, edge_vtx ? edge_vtx + p0 : nullptr, on_dev, &wi));
  }
  return HG_OK;
}

}  // namespace

extern "C" {

hg_status hg_set_allocator(hg_alloc_fn alloc, hg_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_hooks.alloc = alloc;
  g_hooks.free_fn = free_fn;
  g_hooks.ctx = ctx;
  return HG_OK;
}

hg_status hg_wait_flag(const int32_t* flag, int32_t limit_us, void* cuda_stream) {
  if (!flag || limit_us < 0) return HG_ERR_INVALID_ARG;
  int dev = 0, nsm = 0;
  HG_TRY(check_device(&dev, &nsm));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* err = nullptr;
  HG_CUDA(cudaMallocAsync(&err, sizeof(int), s));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    launch_wait_flag(flag, (int64_t)limit_us * 1000, err, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(err, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return HG_ERR_CUDA;
  return dev_err_status(h);
}

hg_status hg_load_csr(int32_t num_vertices, int32_t num_edges, const int64_t* edge_ptr,
                      const int32_t* edge_vtx, int inputs_on_device, void* cuda_stream,
                      hg_graph** out) {
  if (!out) return HG_ERR_INVALID_ARG;
  *out = nullptr;
  if (num_vertices < 1 || num_edges < 0 || !edge_ptr) return HG_ERR_INVALID_ARG;
  int dev = 0, nsm = 0;
  HG_TRY(check_device(&dev, &nsm));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int64_t nnz = 0;
  if (inputs_on_device) {
    HG_CUDA(cudaMemcpyAsync(&nnz, edge_ptr + num_edges, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HG_CUDA(cudaStreamSynchronize(s));
  } else {
    nnz = edge_ptr[num_edges];
  }
  if (nnz < 0 || (nnz > 0 && !edge_vtx)) return HG_ERR_INVALID_ARG;
  hg_graph* g = new hg_graph();
  g->device = dev;
  g->nsm = nsm;
  g->stream = s;
  g->nv = num_vertices;
  g->ne = num_edges;
  g->nnz = nnz;
  hg_status st = load_impl(g, edge_ptr, edge_vtx, inputs_on_device);
  if (st != HG_OK) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    release(g, g->load_blocks);
    cudaStreamSynchronize(s);
    delete g;
    return st;
  }
  *out = g;
  return HG_OK;
}

hg_status hg_build_wedges(hg_graph* g, const hg_tuning* opt, hg_wedge_stats* out) {
  if (!g || !tuning_ok(opt)) return HG_ERR_INVALID_ARG;   // the handle stays as it was
  hg_status st = build_impl(g, opt, out);
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
    g->built = false;
  }
  return st;
}

hg_status hg_autotune(hg_graph* g, hg_autotune_result* out) {
  if (!g) return HG_ERR_INVALID_ARG;
  if (g->nm > 0) return HG_ERR_UNSUPPORTED;   // a wave: hg_batch_autotune
  hg_status st = autotune_impl(g, out);
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
    g->built = g->counted = g->have_cstats = false;
  }
  return st;
}

hg_status hg_count_patterns(hg_graph* g, uint64_t counts[21]) {
  if (!g) return HG_ERR_INVALID_ARG;
  if (!g->built) return HG_ERR_STATE;
  hg_status st = count_impl(g, counts);
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
  }
  return st;
}

hg_status hg_sample_estimate(hg_graph* g, uint64_t seed, uint64_t first_sample,
                             uint64_t num_samples, double sigma, uint64_t raw[21],
                             double est[21]) {
  if (!g || !raw || !est || !(sigma > 0.0) || sigma > 1.0) return HG_ERR_INVALID_ARG;
  if (!g->built) return HG_ERR_STATE;
  if (g->nm > 0) return HG_ERR_UNSUPPORTED;
  if (num_samples > UINT64_MAX - first_sample) return HG_ERR_INVALID_ARG;
  hg_status st = HG_OK;
  hg_graph* h = g;
  if (sigma != 1.0) {
    st = subgraph_impl(g, seed, sigma);
    h = g->sub;
  }
  if (st == HG_OK) st = sample_impl(h, seed, first_sample, num_samples, sigma, raw, est);
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
  }
  return st;
}

hg_status hg_sample_estimate_adv(hg_graph* g, uint64_t seed, uint64_t first_sample,
                                 uint64_t num_samples, double sigma, uint32_t class_mask,
                                 uint64_t raw[21], double est[21], uint64_t info[8]) {
  if (!g || !raw || !est || !(sigma > 0.0) || sigma > 1.0 || class_mask > 15u)
    return HG_ERR_INVALID_ARG;
  if (!g->built) return HG_ERR_STATE;
  if (g->nm > 0) return HG_ERR_UNSUPPORTED;
  if (num_samples > UINT64_MAX - first_sample) return HG_ERR_INVALID_ARG;
  hg_status st = HG_OK;
  hg_graph* h = g;
  if (sigma != 1.0) {
    st = subgraph_impl(g, seed, sigma);
    h = g->sub;
  }
  if (st == HG_OK)
    st = sample_adv_impl(h, seed, first_sample, num_samples, sigma, class_mask, raw, est, info);
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
  }
  return st;
}

hg_status hg_enumerate_pattern(hg_graph* g, int32_t pattern, int32_t* triples, uint64_t capacity,
                               int triples_on_device, uint64_t* total) {
  if (!g || !total || pattern < 0 || pattern > 20 || (capacity > 0 && !triples) ||
      capacity > (UINT64_MAX / 12))
    return HG_ERR_INVALID_ARG;
  if (!g->built) return HG_ERR_STATE;
  if (g->nm > 0) return HG_ERR_UNSUPPORTED;
  auto run = [&]() -> hg_status {
    if (!g->upper_built) HG_TRY(upper_impl(g));
    cudaStream_t s = g->stream;
    uint8_t lut[128];
    build_lut(lut);
    sample_set_lut(lut, s);
    std::vector<Block> tmp;
    int32_t* out = triples;
    if (!triples_on_device && capacity > 0) {
      out = alloc_t<int32_t>(g, tmp, (int64_t)(3 * capacity));
      if (!out) return HG_ERR_OOM;
    }
    unsigned long long* count = &g->small->found;
    HG_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
    t_begin(g, "enumerate");
    launch_enumerate(dev_graph(g), g->up_ptr, g->up_index, g->up, g->packed, g->stats.W, pattern,
                     out, capacity, count, s, g->nsm);
    t_end(g);
    unsigned long long n = 0;
    HG_CUDA(cudaMemcpyAsync(&n, count, sizeof(n), cudaMemcpyDeviceToHost, s));
    HG_CUDA(cudaStreamSynchronize(s));
    if (!triples_on_device && capacity > 0 && n > 0)
      HG_CUDA(cudaMemcpyAsync(triples, out, sizeof(int32_t) * 3 * std::min<uint64_t>(n, capacity),
                              cudaMemcpyDeviceToHost, s));
    Small h;
    HG_TRY(sync_small(g, &h));
    release(g, tmp);
    t_collect(g);
    *total = n;
    return HG_OK;
  };
  hg_status st = run();
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
  }
  return st;
}

hg_status hg_clustering_coeff(hg_graph* g, const double eps[20], double* cc,
                              uint64_t* open_triples, uint64_t* connected_triples) {
  if (!g || !eps) return HG_ERR_INVALID_ARG;
  if (!g->counted) return HG_ERR_STATE;
  const uint64_t connected = g->stats.connected;
  const uint64_t open = connected - 3 * g->counts[0];
  // Def. 5.1: 3 * sum_p eps_p |triangles of pattern p| / |open hyper-triangles|
  double num = 0.0;
  for (int p = 1; p <= 20; ++p) num += eps[p - 1] * (double)g->counts[p];
  if (cc) *cc = open == 0 ? NAN : 3.0 * num / (double)open;
  if (open_triples) *open_triples = open;
  if (connected_triples) *connected_triples = connected;
  return HG_OK;
}

hg_status hg_free(hg_graph* g) {
  if (!g) return HG_ERR_INVALID_ARG;
  if (g->nm > 0) return HG_ERR_STATE;   // a wave belongs to its batch
  return free_graph(g);
}

hg_status hg_load_batch(int32_t num_graphs, const int32_t* num_vertices, const int64_t* edge_off,
                        const int64_t* edge_ptr, const int32_t* edge_vtx, int inputs_on_device,
                        int64_t max_wave_edges, void* cuda_stream, hg_batch** out) {
  if (!out) return HG_ERR_INVALID_ARG;
  *out = nullptr;
  if (num_graphs < 1 || !num_vertices || !edge_off || !edge_ptr || max_wave_edges < 0)
    return HG_ERR_INVALID_ARG;
  if (edge_off[0] != 0) return HG_ERR_INVALID_ARG;
  for (int32_t m = 0; m < num_graphs; ++m)
    if (num_vertices[m] < 1 || edge_off[m + 1] < edge_off[m] ||
        edge_off[m + 1] - edge_off[m] > INT32_MAX)
      return HG_ERR_INVALID_ARG;
  int dev = 0, nsm = 0;
  HG_TRY(check_device(&dev, &nsm));
  hg_batch* b = new hg_batch();
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->G = num_graphs;
  hg_status st = load_batch_impl(b, num_vertices, edge_off, edge_ptr, edge_vtx, inputs_on_device,
                                 max_wave_edges > 0 ? max_wave_edges : kDefaultWaveEdges, dev, nsm);
  if (st != HG_OK) {
    cudaStreamSynchronize(b->stream);
    cudaGetLastError();
    free_batch(b);
    cudaGetLastError();
    return st;
  }
  *out = b;
  return HG_OK;
}

hg_status hg_load_batch_members(int32_t num_graphs, const int32_t* num_vertices,
                                const int32_t* num_edges, const int64_t* const* edge_ptrs,
                                const int32_t* const* edge_vtxs, int inputs_on_device,
                                int64_t max_wave_edges, void* cuda_stream, hg_batch** out) {
  if (!out) return HG_ERR_INVALID_ARG;
  *out = nullptr;
  if (num_graphs < 1 || !num_vertices || !num_edges || !edge_ptrs || !edge_vtxs ||
      max_wave_edges < 0)
    return HG_ERR_INVALID_ARG;
  int dev = 0, nsm = 0;
  HG_TRY(check_device(&dev, &nsm));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  std::vector<int64_t> edge_off((size_t)num_graphs + 1, 0), nnz((size_t)num_graphs, 0);
  for (int32_t m = 0; m < num_graphs; ++m) {
    if (num_vertices[m] < 1 || num_edges[m] < 0 || !edge_ptrs[m]) return HG_ERR_INVALID_ARG;
    edge_off[(size_t)m + 1] = edge_off[(size_t)m] + num_edges[m];
    int64_t first = 0, last = 0;
    if (inputs_on_device) {
      HG_CUDA(cudaMemcpyAsync(&first, edge_ptrs[m], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      HG_CUDA(cudaMemcpyAsync(&last, edge_ptrs[m] + num_edges[m], sizeof(int64_t),
                              cudaMemcpyDeviceToHost, s));
      HG_CUDA(cudaStreamSynchronize(s));
    } else {
      first = edge_ptrs[m][0];
      last = edge_ptrs[m][num_edges[m]];
    }
    if (first != 0 || last < 0 || (last > 0 && !edge_vtxs[m])) return HG_ERR_INVALID_ARG;
    nnz[(size_t)m] = last;
  }
  hg_batch* b = new hg_batch();
  b->stream = s;
  b->G = num_graphs;
  hg_status st = load_batch_impl(b, num_vertices, edge_off.data(), nullptr, nullptr,
                                 inputs_on_device,
                                 max_wave_edges > 0 ? max_wave_edges : kDefaultWaveEdges, dev, nsm,
                                 edge_ptrs, edge_vtxs, nnz.data());
  if (st != HG_OK) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    free_batch(b);
    cudaGetLastError();
    return st;
  }
  *out = b;
  return HG_OK;
}

hg_status hg_batch_autotune(hg_batch* b, int32_t wave, hg_autotune_result* out) {
  if (!b || wave < -1 || wave >= (int32_t)b->waves.size()) return HG_ERR_INVALID_ARG;
  if (wave < 0) {   // the wave with the most hyperedges
    wave = 0;
    for (size_t k = 1; k < b->waves.size(); ++k)
      if (b->waves[k]->ne > b->waves[(size_t)wave]->ne) wave = (int32_t)k;
  }
  b->built = b->counted = false;
  hg_graph* g = b->waves[(size_t)wave];
  hg_status st = autotune_impl(g, out);
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
    g->built = g->counted = g->have_cstats = false;
    return st;
  }
  for (hg_graph* w : b->waves) {
    w->tuned = g->tuned;
    w->has_tuned = true;
  }
  return HG_OK;
}

hg_status hg_batch_build_wedges(hg_batch* b, const hg_tuning* opt) {
  if (!b || !tuning_ok(opt)) return HG_ERR_INVALID_ARG;   // the batch stays as it was
  b->built = b->counted = false;
  for (hg_graph* g : b->waves) {
    hg_status st = hg_build_wedges(g, opt, nullptr);
    if (st != HG_OK) return st;
  }
  b->built = true;
  return HG_OK;
}

// The 21 counts of member q of a wave, from its canonical mask histogram.
static void member_counts(const hg_graph* g, int32_t q, uint64_t counts[21]) {
  uint8_t lut[128];
  build_lut(lut);
  std::memset(counts, 0, sizeof(uint64_t) * 21);
  const uint64_t* mk = g->h_mmasks.data() + 128 * (size_t)q;
  for (int m = 0; m < 128; ++m) {
    counts[lut[m]] += mk[m];
    counts[0] += mk[m];
  }
}

hg_status hg_batch_count_patterns(hg_batch* b, uint64_t* counts, hg_wedge_stats* stats) {
  if (!b) return HG_ERR_INVALID_ARG;
  if (!b->built) return HG_ERR_STATE;
  b->counted = false;
  for (hg_graph* g : b->waves) {
    hg_status st = hg_count_patterns(g, nullptr);
    if (st != HG_OK) return st;
  }
  for (size_t k = 0; k < b->waves.size(); ++k) {
    const hg_graph* g = b->waves[k];
    for (int32_t q = 0; q < g->nm; ++q) {
      const size_t m = (size_t)(b->first[k] + q);
      uint64_t h[21];
      member_counts(g, q, h);
      const unsigned long long* st = g->h_mstats.data() + 4 * (size_t)q;
      if (counts)
        for (int p = 0; p <= 20; ++p) counts[21 * m + (size_t)p] = h[p];
      if (st[0] & 1) return HG_ERR_INTERNAL;
      if (stats) {
        hg_wedge_stats& w = stats[m];
        std::memset(&w, 0, sizeof(w));
        w.W = st[0] / 2;
        w.W_c = st[2];
        w.W_t = w.W - w.W_c;
        w.connected = st[1];
        w.max_deg = st[3];
      }
    }
  }
  b->counted = true;
  return HG_OK;
}

hg_status hg_batch_clustering_coeff(hg_batch* b, const double eps[20], double* cc,
                                    uint64_t* open_triples, uint64_t* connected_triples) {
  if (!b || !eps) return HG_ERR_INVALID_ARG;
  if (!b->counted) return HG_ERR_STATE;
  for (size_t k = 0; k < b->waves.size(); ++k) {
    const hg_graph* g = b->waves[k];
    for (int32_t q = 0; q < g->nm; ++q) {
      const size_t m = (size_t)(b->first[k] + q);
      uint64_t h[21];
      member_counts(g, q, h);
      const uint64_t total = h[0];
      const uint64_t connected = g->h_mstats[4 * (size_t)q + 1];
      const uint64_t open = connected - 3 * total;
      // Def. 5.1, summed in order p = 1..20 in IEEE double, as hg_clustering_coeff
      double num = 0.0;
      for (int p = 1; p <= 20; ++p) num += eps[p - 1] * (double)h[p];
      if (cc) cc[m] = open == 0 ? NAN : 3.0 * num / (double)open;
      if (open_triples) open_triples[m] = open;
      if (connected_triples) connected_triples[m] = connected;
    }
  }
  return HG_OK;
}

hg_status hg_batch_waves(hg_batch* b, int32_t* num_waves) {
  if (!b || !num_waves) return HG_ERR_INVALID_ARG;
  *num_waves = (int32_t)b->waves.size();
  return HG_OK;
}

hg_status hg_batch_wave(hg_batch* b, int32_t k, hg_graph** wave, int32_t* first_member,
                        int32_t* num_members) {
  if (!b || k < 0 || k >= (int32_t)b->waves.size()) return HG_ERR_INVALID_ARG;
  if (wave) *wave = b->waves[(size_t)k];
  if (first_member) *first_member = b->first[(size_t)k];
  if (num_members) *num_members = b->first[(size_t)k + 1] - b->first[(size_t)k];
  return HG_OK;
}

hg_status hg_batch_free(hg_batch* b) {
  if (!b) return HG_ERR_INVALID_ARG;
  free_batch(b);
  return HG_OK;
}

hg_status hg_close_stats_get(hg_graph* g, hg_close_stats* out) {
  if (!g || !out) return HG_ERR_INVALID_ARG;
  if (!g->have_cstats) return HG_ERR_STATE;
  *out = g->cstats;
  return HG_OK;
}

hg_status hg_sample_work_get(hg_graph* g, uint64_t work[3]) {
  if (!g || !work) return HG_ERR_INVALID_ARG;
  hg_graph* h = g->sub && g->sub->sample_work[1] ? g->sub : g;
  for (int k = 0; k < 3; ++k) work[k] = h->sample_work[k];
  return HG_OK;
}

hg_status hg_kernel_launches(uint64_t* n) {
  if (!n) return HG_ERR_INVALID_ARG;
  *n = hg::g_launches.load(std::memory_order_relaxed);
  return HG_OK;
}

hg_status hg_pattern_table(uint8_t lut[128]) {
  if (!lut) return HG_ERR_INVALID_ARG;
  build_lut(lut);
  return HG_OK;
}

hg_status hg_canonical_masks(uint8_t canon[128]) {
  if (!canon) return HG_ERR_INVALID_ARG;
  for (int m = 0; m < 128; ++m) canon[m] = (uint8_t)canonical_of(m);
  return HG_OK;
}

hg_status hg_mask_histogram(hg_graph* g, uint64_t masks[128]) {
  if (!g || !masks) return HG_ERR_INVALID_ARG;
  if (!g->counted) return HG_ERR_STATE;
  std::memcpy(masks, g->masks, sizeof(g->masks));
  return HG_OK;
}

hg_status hg_count_owned(hg_graph* g, const int32_t* owners, int32_t num_owners,
                         uint64_t counts[21], uint64_t masks[128]) {
  if (!g || !counts || num_owners < 0 || (num_owners > 0 && !owners)) return HG_ERR_INVALID_ARG;
  if (!g->built) return HG_ERR_STATE;
  if (g->nm > 0) return HG_ERR_UNSUPPORTED;
  std::vector<uint8_t> sel((size_t)std::max<int64_t>(g->ne, 1), 0);
  for (int32_t k = 0; k < num_owners; ++k) {
    if (owners[k] < 0 || (int64_t)owners[k] >= g->ne) return HG_ERR_INVALID_ARG;
    sel[(size_t)owners[k]] = 1;
  }
  hg_status st = count_impl(g, counts, sel.data());
  if (st != HG_OK) {
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    g->pending.clear();
  } else if (masks) {
    std::memcpy(masks, g->masks, sizeof(g->masks));
  }
  g->counted = false;   // the handle's bins hold a part of the hyper-triangles only
  return st;
}

hg_status hg_out_degrees(hg_graph* g, int32_t* out_degree) {
  if (!g || !out_degree) return HG_ERR_INVALID_ARG;
  if (!g->built) return HG_ERR_STATE;
  if (g->ne == 0) return HG_OK;
  HG_CUDA(cudaMemcpyAsync(out_degree, g->ori.dplus, sizeof(int32_t) * (size_t)g->ne,
                          cudaMemcpyDeviceToHost, g->stream));
  HG_CUDA(cudaStreamSynchronize(g->stream));
  return HG_OK;
}

hg_status hg_batch_mask_histogram(hg_batch* b, uint64_t* masks) {
  if (!b || !masks) return HG_ERR_INVALID_ARG;
  if (!b->counted) return HG_ERR_STATE;
  for (size_t k = 0; k < b->waves.size(); ++k) {
    const hg_graph* g = b->waves[k];
    std::memcpy(masks + 128 * (size_t)b->first[k], g->h_mmasks.data(),
                sizeof(uint64_t) * 128 * (size_t)g->nm);
  }
  return HG_OK;
}

const char* hg_status_str(hg_status s) {
  switch (s) {
    case HG_OK: return "ok";
    case HG_ERR_INVALID_ARG: return "invalid argument";
    case HG_ERR_EMPTY_HYPEREDGE: return "empty hyperedge";
    case HG_ERR_DUP_VERTEX: return "vertex repeated inside a hyperedge";
    case HG_ERR_VERTEX_RANGE: return "vertex id out of range";
    case HG_ERR_UNSORTED: return "hyperedge vertex list not ascending";
    case HG_ERR_DUPLICATE_HYPEREDGE: return "two hyperedges are equal";
    case HG_ERR_OOM: return "out of device memory";
    case HG_ERR_CUDA: return "CUDA runtime error";
    case HG_ERR_TIMEOUT: return "device wait timed out";
    case HG_ERR_STATE: return "call out of order";
    case HG_ERR_UNSUPPORTED: return "input beyond supported limits";
    case HG_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    case HG_ERR_INTERNAL: return "internal consistency check failed";
    case HG_ERR_CANCELLED: return "query cancelled before it ran";
  }
  return "unknown status";
}

hg_status hg_set_timing(hg_graph* g, int enable) {
  if (!g) return HG_ERR_INVALID_ARG;
  g->timing = enable != 0;
  return HG_OK;
}

hg_status hg_kernel_times(hg_graph* g, const char** names, float* ms, int32_t* launches,
                          int32_t* n) {
  if (!g || !n) return HG_ERR_INVALID_ARG;
  int32_t cap = *n, k = 0;
  for (auto& t : g->times) {
    if (k >= cap) break;
    if (names) names[k] = t.first;
    if (ms) ms[k] = t.second.first;
    if (launches) launches[k] = t.second.second;
    ++k;
  }
  *n = k;
  g->times.clear();
  return HG_OK;
}

}  // extern "C"

namespace hg {
void alloc_bypass_hooks(bool on) { t_bypass_hooks = on; }
}  // namespace hg
