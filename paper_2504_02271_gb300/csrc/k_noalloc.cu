// hg_wedge_degrees_noalloc: line-graph degrees and the inclusion-wedge count with
// no device allocation at all.  It is a variant of the count pass of the
// hyperwedge kernels (k_wedge.cu): one block per hyperedge accumulates
// omega_ij over the E_v lists of its vertices in a hash table, but the tables
// live in one file-scope device array instead of memory from an allocator.
//
// Who needs this: a service whose device memory is a fixed arena owned by someone
// else (a serving process that reserved the GPU's memory up front, a plug-in living
// inside another framework's memory pool), where an extra cudaMalloc would either
// fail or stall every other stream on the device while the driver reclaims memory.
// Such a caller can pass device buffers for inputs and outputs, and this entry
// point brings the rest.  It makes ordinary CUDA runtime calls (a memset, a launch,
// copies and a stream synchronisation), so it is called from plain host code -
// never from inside a host function enqueued on a stream, where CUDA calls are not
// allowed at all.
//
// Each row hashes into the first 2^k slots of its block's table, 2^k the smallest
// power of two holding twice the row's gathered incidences (at least 256), so a
// small row clears and scans a small region instead of the whole table.
#include <cuda_runtime.h>

#include <mutex>

#include "hg_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kTableLog2 = 15;                        // 32,768 slots per block table
constexpr int kTables = 128;                          // blocks running at once
constexpr unsigned long long kEmptySlot = ~0ull;

// The whole scratch: kTables tables of (j << 32 | count) slots and a control word
// block.  Every device that loads the library holds it until the process exits.
struct NoallocScratch {
  unsigned long long table[kTables][1 << kTableLog2];   // 32 MiB
  unsigned long long wc;                                // inclusion-type wedges
  int err;                                              // first error (DevErr)
  int next_row;                                         // work counter
};
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__device__ __forceinline__ void add_neighbour(unsigned long long* T, int cap_log2, uint32_t j) {
  const uint32_t mask = (1u << cap_log2) - 1u;
  uint32_t s = (j * 0x9E3779B1u) >> (32 - cap_log2);
  const unsigned long long key = (unsigned long long)j << 32;
  while (true) {
    unsigned long long cur = *((volatile unsigned long long*)&T[s]);
    if (cur == kEmptySlot) {
      cur = atomicCAS(&T[s], kEmptySlot, key | 1ull);
      if (cur == kEmptySlot) return;
    }
    if ((uint32_t)(cur >> 32) == j) {
      atomicAdd(&T[s], 1ull);
      return;
    }
    s = (s + 1u) & mask;
  }
}

// One block per hyperedge i (fetched from a counter): deg[i] = number of distinct
// j != i sharing a vertex with e_i; inclusion wedges (j > i, omega_ij equal to the
// smaller size) are summed into wc.  A row that gathers more than half a table of
// (j, v) incidences is not processed and sets DE_LIMIT.
__global__ void __launch_bounds__(kThreads)
    k_wedge_degrees_noalloc(NoallocScratch* sc, int32_t ne, const int64_t* __restrict__ e_ptr,
                            const int32_t* __restrict__ e_idx, const int64_t* __restrict__ v_ptr,
                            const int32_t* __restrict__ v_idx, int32_t* __restrict__ deg) {
  unsigned long long* T = sc->table[blockIdx.x];
  constexpr uint32_t CAP = 1u << kTableLog2;
  __shared__ int32_t s_row;
  __shared__ unsigned long long s_cand;
  __shared__ int32_t s_distinct;
  __shared__ unsigned long long s_wc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kWarps = kThreads / 32;
  if (threadIdx.x == 0) s_wc = 0;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_row = atomicAdd(&sc->next_row, 1);
      s_cand = 0;
      s_distinct = 0;
    }
    __syncthreads();
    const int32_t i = s_row;
    if (i >= ne) break;
    const int64_t b = e_ptr[i], e = e_ptr[i + 1];
    // gather count of the row: it must fit half a table
    unsigned long long c = 0;
    for (int64_t p = b + threadIdx.x; p < e; p += kThreads) {
      const int32_t v = e_idx[p];
      c += (unsigned long long)(v_ptr[v + 1] - v_ptr[v] - 1);
    }
    atomicAdd(&s_cand, c);
    __syncthreads();
    const unsigned long long cand = s_cand;   // read after a barrier: the same on every thread
    if (cand > (unsigned long long)(CAP / 2)) {
      if (threadIdx.x == 0) atomicCAS(&sc->err, 0, hg::DE_LIMIT);
      continue;
    }
    int cl = 8;   // this row's region: 2^cl >= 2 * cand slots (load factor <= 1/2)
    while (cl < kTableLog2 && (1ull << cl) < 2 * cand) ++cl;
    const uint32_t rcap = 1u << cl;
    for (uint32_t s = threadIdx.x; s < rcap; s += kThreads) T[s] = kEmptySlot;
    __syncthreads();
    for (int64_t p = b + w; p < e; p += kWarps) {
      const int32_t v = e_idx[p];
      for (int64_t q = v_ptr[v] + lane; q < v_ptr[v + 1]; q += 32) {
        const int32_t j = v_idx[q];
        if (j != i) add_neighbour(T, cl, (uint32_t)j);
      }
    }
    __syncthreads();
    const int32_t szi = (int32_t)(e - b);
    int distinct = 0;
    unsigned long long wc = 0;
    for (uint32_t s = threadIdx.x; s < rcap; s += kThreads) {
      const unsigned long long x = T[s];
      if (x == kEmptySlot) continue;
      ++distinct;
      const int32_t j = (int32_t)(x >> 32), om = (int32_t)(x & 0xffffffffu);
      if (j > i) {
        const int32_t szj = (int32_t)(e_ptr[j + 1] - e_ptr[j]);
        if (om == szi && om == szj) atomicCAS(&sc->err, 0, hg::DE_DUPEDGE);
        if (om == (szi < szj ? szi : szj)) ++wc;
      }
    }
    atomicAdd(&s_distinct, distinct);
    if (wc) atomicAdd(&s_wc, wc);
    __syncthreads();
    if (threadIdx.x == 0) deg[i] = s_distinct;
  }
  if (threadIdx.x == 0 && s_wc) atomicAdd(&sc->wc, s_wc);
}

// Device address of the scratch, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
NoallocScratch* g_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" hg_status hg_wedge_degrees_noalloc(int32_t num_edges, const int64_t* edge_ptr,
                                              const int32_t* edge_vtx, const int64_t* vertex_ptr,
                                              const int32_t* vertex_edge, int32_t* degrees,
                                              unsigned long long* inclusion_wedges,
                                              void* cuda_stream) {
  if (num_edges < 0 || !edge_ptr || !vertex_ptr || !degrees || !inclusion_wedges ||
      (num_edges > 0 && (!edge_vtx || !vertex_edge)))
    return HG_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return HG_ERR_NO_DEVICE;
  }
  NoallocScratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return HG_ERR_CUDA;
      }
      g_addr[dev] = static_cast<NoallocScratch*>(p);
    }
    sc = g_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the array keeps the previous call's contents: reset the control words
  if (cudaMemsetAsync(&sc->wc, 0, sizeof(unsigned long long) + 2 * sizeof(int), s) != cudaSuccess)
    return HG_ERR_CUDA;
  if (num_edges > 0) {
    hg::note_launch();
    k_wedge_degrees_noalloc<<<kTables, kThreads, 0, s>>>(sc, num_edges, edge_ptr, edge_vtx,
                                                         vertex_ptr, vertex_edge, degrees);
    if (cudaGetLastError() != cudaSuccess) return HG_ERR_CUDA;   // the launch was refused
  }
  if (cudaMemcpyAsync(inclusion_wedges, &sc->wc, sizeof(unsigned long long),
                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HG_ERR_CUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, &sc->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return HG_ERR_CUDA;
  }
  if (err == hg::DE_LIMIT) return HG_ERR_UNSUPPORTED;
  if (err == hg::DE_DUPEDGE) return HG_ERR_DUPLICATE_HYPEREDGE;
  return err ? HG_ERR_INTERNAL : HG_OK;
}
