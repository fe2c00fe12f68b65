// Internal declarations shared by the CUDA translation units of libhg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hg.h"

namespace hg {

constexpr int kWarp = 32;

// Error words written by kernels (first writer wins via atomicCAS).
enum DevErr : int {
  DE_OK = 0,
  DE_EMPTY = 1,
  DE_RANGE = 2,
  DE_DUPV = 3,
  DE_UNSORTED = 4,
  DE_DUPEDGE = 5,
  DE_PTR = 6,       // edge_ptr not monotone / out of [0, nnz]
  DE_INTERNAL = 7,  // a kernel-side consistency check failed
  DE_LIMIT = 8,     // an input row beyond a kernel's fixed capacity
  DE_TIMEOUT = 9,   // a bounded device wait gave up
};

__device__ __forceinline__ void dev_fail(int* err, int code) { atomicCAS(err, 0, code); }

// Oriented wedge entries.  Packed: (nbr << 8) | omega, used when |E| < 2^24 and
// every omega < 256; otherwise nbr and omega live in two int32 arrays.
struct Oriented {
  int64_t* row_ptr;   // [ne+1] start of row i (capacity deg(i))
  int32_t* dplus;     // [ne] used length of row i
  uint32_t* packed;   // [2W] packed entries, or nullptr
  int32_t* nbr;       // [2W] wide entries, or nullptr
  int32_t* omega;     // [2W]
  int64_t slots;      // entries the arrays hold (0 = not recorded)
};

struct DevGraph {
  int32_t nv, ne;
  int64_t nnz;
  const int64_t* e_ptr;
  const int32_t* e_idx;
  const int32_t* esize;
  const int64_t* v_ptr;
  const int32_t* v_idx;
  // a batch of disjoint member hypergraphs: member m owns hyperedges
  // [m_eoff[m], m_eoff[m+1]); nm == 0 for a single hypergraph
  const int32_t* m_eoff;
  int32_t nm;
};

// member owning hyperedge u (0 for a single hypergraph)
__device__ __forceinline__ int32_t member_of(const DevGraph& g, int32_t u) {
  int32_t lo = 0, hi = g.nm > 0 ? g.nm - 1 : 0;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(g.m_eoff + mid) <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------- launch wrappers (implemented in the .cu files) ----------------

// process-wide count of kernel launches made by the library (defined in hg_api.cu)
void note_launch(int n = 1);

// k_scan.cu
// out[0..n] = exclusive prefix sums of in[0..n) (out[n] = total); tmp >= scan_tmp_bytes(n).
size_t scan_tmp_bytes(int64_t n);
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s);
void scan_i64_to_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s);
// acc[0] += sum C(x,2), acc[1] = max x, acc[2] += sum x  over x in a[0..n)
void reduce_deg_stats(const int32_t* a, int64_t n, unsigned long long* acc, cudaStream_t s);

// k_load.cu
// One thread waits until *flag != 0, at most limit_ns of the global timer (and a bounded
// number of polls), else records DE_TIMEOUT in *err.
void launch_wait_flag(const int32_t* flag, int64_t limit_ns, int* err, cudaStream_t s);
void launch_check_ptr(const int64_t* e_ptr, int32_t ne, int64_t nnz, int* err, cudaStream_t s);
void launch_validate_rows(const DevGraph& g, int32_t* esize, int32_t* vdeg, int* err,
                          cudaStream_t s);
void launch_scatter(const DevGraph& g, int32_t* cursor, int32_t* v_idx, cudaStream_t s);
// cand[i] = sum_{v in e_i} (|E_v| - 1); also bucket rows by cand into lists
void launch_candidates(const DevGraph& g, int64_t* cand, unsigned long long* max_cand,
                       int32_t* max_size, cudaStream_t s);

// k_dense.cu: heavy x heavy omega on the tensor cores
struct DenseInfo {
  const int32_t* heavy_idx;   // [ne] position in the heavy list or -1; nullptr = no dense path
  const int32_t* ids;         // [nh] hyperedge id of each heavy position
  const uint16_t* omega;      // [rows_pad x rows_pad] omega of heavy pairs
  int64_t ld;                 // row stride of omega
  int32_t nh;
};
size_t dense_smem_bytes();
int64_t dense_round_rows(int64_t n);
int64_t dense_round_k(int64_t k);
void launch_size_hist(const int32_t* esize, int32_t ne, int32_t max_bin, unsigned long long* hist,
                      cudaStream_t s);
// heavy: min_size <= |e_i| <= max_size, at most cap of them
void launch_pick_heavy(const int32_t* esize, int32_t ne, int32_t min_size, int32_t max_size,
                       int32_t cap, int32_t* heavy_idx, int32_t* ids, int32_t* count,
                       cudaStream_t s);
// omega values the tile kernel writes exactly (uint16 output)
constexpr int32_t kDenseMaxOmega = 65535;
void launch_fill_dense(const int64_t* e_ptr, const int32_t* e_idx, const int32_t* ids, int32_t nh,
                       uint8_t* a, int64_t lda, cudaStream_t s);
cudaError_t launch_dense_omega(const uint8_t* a, int64_t rows, int64_t rows_pad, int64_t k_pad,
                               uint16_t* omega, int* err, cudaStream_t s);

// k_wedge.cu
struct WedgeBuckets {
  int32_t* rows[3];  // light (warp), medium (block, smem), heavy (block, global scratch)
  int32_t* count;    // [3] device counters
};
// rows gathering at most light_max incidences take one warp (light_max <= wedge_light_max_cand)
void launch_bucket_rows(const int64_t* cand, int32_t ne, WedgeBuckets b, int light_max,
                        cudaStream_t s);
// the largest gather count of a one-warp row in the packed (1) or unpacked (0) layout
int wedge_light_max_cand(int packed);
int wedge_medium_max_cand();
// Per-row outputs of the count pass (each may be null): upc[i] = |{j > i}|,
// wcr[i] = |{j > i : omega_ij = min(|e_i|, |e_j|)}| (inclusion-type hyperwedges).
struct RowCounts {
  int32_t* upc;
  int32_t* wcr;
};

// The gather pass of step one: deg(i), RowCounts, W_c into *wc, the duplicate check,
// and every (j, omega_ij) of row i written from rows.row_ptr[i] (a capacity layout:
// room for cap[i] = min(gathered incidences, |E| - 1) entries, see launch_cap_rows).
void launch_wedge_rows(const DevGraph& g, const WedgeBuckets& b, const int32_t* nb,
                       int64_t heavy_max_cand, const int64_t* cand, int32_t* deg,
                       unsigned long long* wc, const Oriented& rows, int packed,
                       unsigned long long* scratch, int* err, int32_t* work_counter,
                       const DenseInfo& dense, RowCounts rc, cudaStream_t s, int nsm);
void launch_cap_rows(const int64_t* cand, int32_t ne, int32_t* cap, cudaStream_t s);
// Filter rows of the capacity layout (len[i] entries from src_ptr[i]) into an exact layout
// (row i from dst_ptr[i]), order kept: keep 0 = j ranked above i in (deg, id), 1 = j > i,
// 2 = all.  count_only: write the number kept to cnt[i] instead.
void launch_filter_rows(int keep, bool count_only, const int64_t* src_ptr, const int32_t* len,
                        const Oriented& src, const int32_t* deg, int32_t ne, int packed,
                        const int64_t* dst_ptr, const Oriented& dst, int32_t* cnt,
                        cudaStream_t s);

// hg_api.cu: allocations of the calling thread skip the caller-installed hooks
void alloc_bypass_hooks(bool on);

// k_batch.cu
void launch_sub_base(int64_t* e_ptr, int32_t ne, int64_t base, cudaStream_t s);
void launch_add_member_base(int64_t* e_ptr, int32_t ne, const int32_t* m_eoff, int32_t nm,
                            const int64_t* noff, cudaStream_t s);
void launch_localize(const DevGraph& g, const int32_t* m_voff, int32_t* e_idx, int* err,
                     cudaStream_t s);
void launch_member_stats(const DevGraph& g, const int32_t* deg, const int32_t* wcr,
                         unsigned long long* out, cudaStream_t s);

// k_sample.cu
int sample_sort_max_log2();
void sample_set_lut(const uint8_t lut[128], cudaStream_t s);
cudaError_t launch_sort_upper(const int64_t* up_ptr, int32_t ne, const Oriented& up, int packed,
                              int* err, cudaStream_t s, int nsm);
// Bucket index of a row-pointer array of `entries` entries over ne rows (sampler row
// searches): row_index_buckets(entries, row_index_shift(entries, ne)) + 1 int32.
int row_index_shift(uint64_t entries, int32_t rows);
int64_t row_index_buckets(uint64_t entries, int shift);
void launch_row_index(const int64_t* ptr, int32_t ne, uint64_t entries, int32_t* first,
                      cudaStream_t s);
// work (may be null): [0] row-pointer reads, [1] upper-row entries read, [2] vertex ids merged;
// up_index (may be null): the bucket index of up_ptr
void launch_sample(const DevGraph& g, const int64_t* up_ptr, const int32_t* up_index,
                   const Oriented& up, int packed, uint64_t W, uint64_t seed, uint64_t first,
                   uint64_t num, unsigned long long* raw, unsigned long long* work, cudaStream_t s,
                   int nsm);
// Appro-adv (Algorithm 7)
void launch_type_counts(const int32_t* upc, const int32_t* wcr, int32_t ne, int32_t* cnt_t,
                        cudaStream_t s);
void launch_split_types(const DevGraph& g, const int64_t* up_ptr, const Oriented& up, int packed,
                        const int64_t* t_ptr, const Oriented& t, const int64_t* c_ptr,
                        const Oriented& c, cudaStream_t s);
void launch_sample_adv(const DevGraph& g, const int64_t* set_ptr, const int32_t* set_index,
                       const Oriented& set_ent, uint64_t Wx, int type, int cls, uint32_t stream,
                       const int64_t* full_ptr, const Oriented& full, int packed, uint64_t seed,
                       uint64_t first, uint64_t num, unsigned long long* raw, cudaStream_t s,
                       int nsm);
// single-pattern enumeration over the upper rows
void launch_enumerate(const DevGraph& g, const int64_t* up_ptr, const int32_t* up_index,
                      const Oriented& up, int packed, uint64_t W, int target, int32_t* out,
                      unsigned long long cap, unsigned long long* count, cudaStream_t s, int nsm);
// the sub-hypergraph G' of Algorithms 6-7 (sigma < 1)
void launch_priority(int32_t ne, uint64_t seed, unsigned long long* pr, cudaStream_t s);
void launch_digit_hist(const unsigned long long* pr, int32_t ne, int shift,
                       unsigned long long pmask, unsigned long long prefix, unsigned int* hist,
                       cudaStream_t s);
void launch_equal_flags(const unsigned long long* pr, int32_t ne, unsigned long long T,
                        int32_t* eq, cudaStream_t s);
void launch_keep_flags(const unsigned long long* pr, int32_t ne, unsigned long long T,
                       const int64_t* eq_rank, int64_t need, int32_t* keep, cudaStream_t s);
void launch_compact_kept(const int32_t* keep, const int64_t* pos, const int32_t* esize, int32_t ne,
                         int32_t* ids, int32_t* sizes, cudaStream_t s);
void launch_gather_rows(const int64_t* e_ptr, const int32_t* e_idx, const int32_t* ids, int32_t nk,
                        const int64_t* sub_ptr, int32_t* sub_idx, cudaStream_t s);
size_t wedge_heavy_scratch_bytes(int64_t heavy_max_cand, int nsm);

// k_close.cu
// close team shapes: warp teams (out-degree <= 64, 128, 256), block teams with shared
// tables (<= 1024, <= 2048, and <= kBlockMaxPacked or kBlockMaxUnpacked by the row
// layout), block teams with global scratch (|e_u| > 32 with out-degree <= kWideLargeMin,
// and teams handed over), cluster teams with global scratch (the rest)
constexpr int kCloseBuckets = 8;
constexpr int kWideBucket = 6;
constexpr int kClusterBucket = 7;
constexpr int kWideLargeMin = 4096;
constexpr int kBlockMaxPacked = 6144;     // 4-byte queue entries leave room for 6,144 indices
constexpr int kBlockMaxUnpacked = 4096;
struct CloseBuckets {
  int32_t* lists[kCloseBuckets];
  int32_t* count;     // [kCloseBuckets]
};
// all_block: send every hyperedge to the global-table kernel (bucket 6)
// warp_max: the largest out-degree a warp team takes (64, 128 or 256); larger out-degrees
// (and |e_u| > 32) go to block teams
// sel: NULL, or one byte per hyperedge; then only the hyperedges u with sel[u] != 0
// get a team (the hyper-triangles they own).
// block_max: largest out-degree of the shared-table block teams (kBlockMaxPacked or
// kBlockMaxUnpacked, by the row layout).
void launch_bucket_close(const DevGraph& g, const Oriented& o, CloseBuckets b,
                         unsigned long long* wide_max, bool all_block, int warp_max,
                         int block_max, const uint8_t* sel, cudaStream_t s);
// n: list length (host copy); n_p: the same on the device; counter: zeroed fetch counter;
// work[0] += probes (entries of out(v) streamed), work[1] += E_y entries scanned for masks;
// warp kernels append hyperedges their tables cannot hold (every hyperedge when
// handover is set) to overflow[*n_overflow++]
void launch_close(int bucket, const DevGraph& g, const Oriented& o, int packed,
                  const int32_t* list, int32_t n, const int32_t* n_p, int64_t wide_cap,
                  int64_t wide_words, int64_t wide_dmax, void* scratch, unsigned long long* hist,
                  unsigned long long* work, int32_t* counter, int32_t* overflow,
                  int32_t* n_overflow, int handover, cudaStream_t s, int nsm);
size_t close_wide_scratch_bytes(int64_t cap, int64_t words, int64_t dmax, int nsm);

}  // namespace hg
