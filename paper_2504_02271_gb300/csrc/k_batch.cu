// Batches of independent hypergraphs counted as one disjoint union.
//
// A union of member hypergraphs with disjoint vertex ranges has the disjoint
// union of their line graphs as its line graph, so every hyperwedge and every
// hyper-triangle (Defs. 2.2, 2.4) lies inside one member, and ranking by
// (line-graph degree, id) orders each member's hyperedges as it would alone.
// The kernels here move the members' CSRs into union coordinates and reduce the
// per-row results of step one into per-member statistics.
#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void k_sub_base(int64_t* __restrict__ e_ptr, int32_t ne, int64_t base) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= ne;
       i += (int64_t)gridDim.x * blockDim.x)
    e_ptr[i] -= base;
}

// Members gathered from separate CSRs: e_ptr[i] += noff[member of i] for i in [0, ne]
// (position ne holds the last member's final offset, so it becomes the total).
__global__ void k_add_member_base(int64_t* __restrict__ e_ptr, int32_t ne,
                                  const int32_t* __restrict__ m_eoff, int32_t nm,
                                  const int64_t* __restrict__ noff) {
  DevGraph g{};
  g.m_eoff = m_eoff;
  g.nm = nm;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= ne;
       i += (int64_t)gridDim.x * blockDim.x)
    e_ptr[i] += noff[member_of(g, (int32_t)i)];
}

// Member-local vertex ids -> union ids (v + m_voff[m]); ids outside [0, |V_m|) set DE_RANGE.
// Runs after the row pointers were checked, so every row range lies in [0, nnz).
__global__ void k_localize(DevGraph g, const int32_t* __restrict__ m_voff, int32_t* __restrict__ e_idx,
                           int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < g.ne; i += warps) {
    const int32_t m = member_of(g, i);
    const int32_t vb = m_voff[m], nvm = m_voff[m + 1] - vb;
    const int64_t b = g.e_ptr[i], e = g.e_ptr[i + 1];
    for (int64_t p = b + lane; p < e; p += 32) {
      const int32_t v = e_idx[p];
      if (v < 0 || v >= nvm) dev_fail(err, DE_RANGE);
      else e_idx[p] = v + vb;
    }
  }
}

// One warp per member: out[4m..4m+3] = sum deg (= 2 W_m), sum C(deg, 2), inclusion
// wedges W_c, max deg.
__global__ void k_member_stats(DevGraph g, const int32_t* __restrict__ deg,
                               const int32_t* __restrict__ wcr,
                               unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < g.nm; m += warps) {
    const int32_t b = g.m_eoff[m], e = g.m_eoff[m + 1];
    unsigned long long sd = 0, sc2 = 0, swc = 0, mx = 0;
    for (int32_t i = b + lane; i < e; i += 32) {
      const unsigned long long d = (unsigned long long)deg[i];
      sd += d;
      sc2 += d * (d - (d > 0)) / 2;
      swc += (unsigned long long)wcr[i];
      mx = d > mx ? d : mx;
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
      sd += __shfl_down_sync(kFull, sd, k);
      sc2 += __shfl_down_sync(kFull, sc2, k);
      swc += __shfl_down_sync(kFull, swc, k);
      const unsigned long long o = __shfl_down_sync(kFull, mx, k);
      mx = o > mx ? o : mx;
    }
    if (lane == 0) {
      out[4 * (size_t)m + 0] = sd;
      out[4 * (size_t)m + 1] = sc2;
      out[4 * (size_t)m + 2] = swc;
      out[4 * (size_t)m + 3] = mx;
    }
  }
}

int grid_of(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b > 65535) b = 65535;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_sub_base(int64_t* e_ptr, int32_t ne, int64_t base, cudaStream_t s) {
  if (base == 0) return;
  note_launch();
  k_sub_base<<<grid_of((int64_t)ne + 1, 256), 256, 0, s>>>(e_ptr, ne, base);
}

void launch_add_member_base(int64_t* e_ptr, int32_t ne, const int32_t* m_eoff, int32_t nm,
                            const int64_t* noff, cudaStream_t s) {
  note_launch();
  k_add_member_base<<<grid_of((int64_t)ne + 1, 256), 256, 0, s>>>(e_ptr, ne, m_eoff, nm, noff);
}

void launch_localize(const DevGraph& g, const int32_t* m_voff, int32_t* e_idx, int* err,
                     cudaStream_t s) {
  if (g.ne == 0) return;
  note_launch();
  k_localize<<<grid_of(g.ne, 8), 256, 0, s>>>(g, m_voff, e_idx, err);
}

void launch_member_stats(const DevGraph& g, const int32_t* deg, const int32_t* wcr,
                         unsigned long long* out, cudaStream_t s) {
  if (g.nm == 0) return;
  note_launch();
  k_member_stats<<<grid_of(g.nm, 8), 256, 0, s>>>(g, deg, wcr, out);
}

}  // namespace hg
