// K0: validate the hyperedge->vertex CSR and build the vertex->hyperedge lists E_v
// (the per-vertex lists of Sec. 3.1 / Algorithm 2).  E_v is built by counting
// sort with atomic cursors, so the order inside one E_v is not fixed; no later
// step depends on it.
#include "hg_internal.cuh"

namespace hg {
namespace {

// edge_ptr[0] == 0, edge_ptr[ne] == nnz, non-decreasing, every row non-empty.
__global__ void k_check_ptr(const int64_t* __restrict__ e_ptr, int32_t ne, int64_t nnz,
                            int* __restrict__ err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e_ptr[i];
    if (p < 0 || p > nnz) dev_fail(err, DE_PTR);
    if (i == 0 && p != 0) dev_fail(err, DE_PTR);
    if (i == ne && p != nnz) dev_fail(err, DE_PTR);
    if (i < ne) {
      int64_t q = e_ptr[i + 1];
      if (q < p) dev_fail(err, DE_PTR);
      else if (q == p) dev_fail(err, DE_EMPTY);
    }
  }
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A bounded wait on a flag in device memory: poll with back-off until it is set, give up
// after limit_ns of the global timer or after a poll count that bounds the loop even if
// the timer stalls.
__global__ void k_wait_flag(const int32_t* flag, int64_t limit_ns, int* __restrict__ err) {
  const uint64_t t0 = global_ns();
  const uint64_t max_polls = (uint64_t)(limit_ns / 256) + 1024;
  for (uint64_t it = 0; it < max_polls; ++it) {
    if (*(volatile const int32_t*)flag != 0) return;
    if ((int64_t)(global_ns() - t0) > limit_ns) break;
    __nanosleep(256);
  }
  dev_fail(err, DE_TIMEOUT);
}

// Row checks (ascending, distinct, in range), |e_i| and vertex degrees |E_v|.
// Runs only after k_check_ptr passed, so every row range lies inside [0, nnz).
__global__ void k_validate_rows(DevGraph g, int32_t* __restrict__ esize,
                                int32_t* __restrict__ vdeg, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < g.ne; i += warps) {
    const int64_t b = g.e_ptr[i], e = g.e_ptr[i + 1];
    if (lane == 0) esize[i] = (int32_t)(e - b);
    for (int64_t p = b + lane; p < e; p += 32) {
      const int32_t v = g.e_idx[p];
      bool ok = true;
      if (v < 0 || v >= g.nv) {
        dev_fail(err, DE_RANGE);
        ok = false;
      }
      if (p > b) {
        const int32_t u = g.e_idx[p - 1];
        if (u == v) {
          dev_fail(err, DE_DUPV);
        } else if (u > v) {
          dev_fail(err, DE_UNSORTED);
        }
      }
      if (ok) atomicAdd(&vdeg[v], 1);
    }
  }
}

__global__ void k_scatter(DevGraph g, int32_t* __restrict__ cursor, int32_t* __restrict__ v_idx) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < g.ne; i += warps) {
    const int64_t b = g.e_ptr[i], e = g.e_ptr[i + 1];
    for (int64_t p = b + lane; p < e; p += 32) {
      const int32_t v = g.e_idx[p];
      const int32_t pos = atomicAdd(&cursor[v], 1);
      v_idx[g.v_ptr[v] + pos] = i;
    }
  }
}

// cand[i] = sum_{v in e_i} (|E_v| - 1): how many (j, v) incidences row i gathers.  One
// thread per row (rows are short); maxima reduced per warp before their atomics.
__global__ void k_candidates(DevGraph g, int64_t* __restrict__ cand,
                             unsigned long long* __restrict__ max_cand,
                             int32_t* __restrict__ max_size) {
  const int lane = threadIdx.x & 31;
  unsigned long long my_max = 0;
  int32_t my_size = 0;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < g.ne;
       i0 += (int64_t)gridDim.x * blockDim.x) {   // warp-uniform trip count
    const int64_t i = i0 + threadIdx.x;
    if (i < g.ne) {
      const int64_t b = g.e_ptr[i], e = g.e_ptr[i + 1];
      int64_t c = 0;
      for (int64_t p = b; p < e; ++p) {
        const int32_t v = g.e_idx[p];
        c += g.v_ptr[v + 1] - g.v_ptr[v] - 1;
      }
      cand[i] = c;
      my_max = (unsigned long long)c > my_max ? (unsigned long long)c : my_max;
      my_size = (int32_t)(e - b) > my_size ? (int32_t)(e - b) : my_size;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long om = __shfl_down_sync(0xffffffffu, my_max, d);
    const int32_t os = __shfl_down_sync(0xffffffffu, my_size, d);
    my_max = om > my_max ? om : my_max;
    my_size = os > my_size ? os : my_size;
  }
  if (lane == 0) {
    atomicMax(max_cand, my_max);
    atomicMax(max_size, my_size);
  }
}

int grid_for(int64_t work_items, int per_block) {
  int64_t b = (work_items + per_block - 1) / per_block;
  if (b > 65535) b = 65535;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_check_ptr(const int64_t* e_ptr, int32_t ne, int64_t nnz, int* err, cudaStream_t s) {
  note_launch();
  k_check_ptr<<<grid_for((int64_t)ne + 1, 256), 256, 0, s>>>(e_ptr, ne, nnz, err);
}

void launch_wait_flag(const int32_t* flag, int64_t limit_ns, int* err, cudaStream_t s) {
  note_launch();
  k_wait_flag<<<1, 1, 0, s>>>(flag, limit_ns, err);
}

void launch_validate_rows(const DevGraph& g, int32_t* esize, int32_t* vdeg, int* err,
                          cudaStream_t s) {
  if (g.ne == 0) return;
  note_launch();
  k_validate_rows<<<grid_for(g.ne, 8), 256, 0, s>>>(g, esize, vdeg, err);
}

void launch_scatter(const DevGraph& g, int32_t* cursor, int32_t* v_idx, cudaStream_t s) {
  if (g.ne == 0) return;
  note_launch();
  k_scatter<<<grid_for(g.ne, 8), 256, 0, s>>>(g, cursor, v_idx);
}

void launch_candidates(const DevGraph& g, int64_t* cand, unsigned long long* max_cand,
                       int32_t* max_size, cudaStream_t s) {
  if (g.ne == 0) return;
  note_launch();
  k_candidates<<<grid_for(g.ne, 256), 256, 0, s>>>(g, cand, max_cand, max_size);
}

}  // namespace hg
