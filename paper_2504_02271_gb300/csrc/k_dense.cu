// Dense-tile hyperwedges on the 5th-generation tensor cores (tcgen05).
//
// For the heaviest hyperedges (the largest ones), omega_ij = |e_i cap e_j| for
// every pair is the product A * A^T of their 0/1 incidence matrix A (rows =
// heavy hyperedges, columns = vertices): omega_ij = sum_v A[i][v] A[j][v]
// (Def. 2.2; it is the heavy-heavy block of H * H^T, Sec. 3.1).  sm_103a has no
// tcgen05 8-bit integer MMA, so the 0/1 entries are e4m3 values (1.0 = 0x38) and
// the products accumulate in FP32 in tensor memory; every dot product is an
// integer no larger than the smaller hyperedge.  The heavy set only takes
// hyperedges of at most 65,535 vertices, so every omega fits the uint16 output and
// is far below 2^24, where FP32 stops representing integers exactly: omega is exact.
//
// Kernel shape: persistent, one CTA per SM, each taking 128 x 256 output tiles in a
// grouped raster (consecutive tiles walk down a group of kGroupM tile rows before
// moving one tile column right, so the CTAs working at one time share a few A panels
// (128 rows) and B panels (256 rows) in L2); K runs over the vertices in steps of 128
// bytes.  Warp 0 issues TMA loads (128-byte swizzle) of the A tile (128 rows) and the B
// tile (256 rows, two boxes) into a 4-stage ring that runs on from tile to tile; warp
// 1 allocates 512 TMEM columns (two 256-column accumulators) and one thread issues
// tcgen05.mma (M=128, N=256, K=32 per instruction, 4 per stage), committing each stage
// back to its ring slot and each finished accumulator to the epilogue; warps 2-5 read
// the accumulator rows they own with tcgen05.ld and write omega as uint16 while the next
// tile's MMAs fill the other accumulator.  Every mbarrier wait is bounded: on time-out the kernel raises
// an error word, stops issuing, waits for its own copies and frees its TMEM.
#include <algorithm>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr int kBM = 128, kBN = 256, kBK = 128;   // tile rows (A), rows (B), bytes of K per stage
constexpr int kStages = 4;
constexpr int kThreads = 192;
constexpr uint32_t kStageBytes = (kBM + kBN) * kBK;
constexpr uint32_t kTmemCols = 512;   // two 256-column accumulators
constexpr uint32_t kSpinLimit = 1u << 22;          // bounded waits (~ 1 s with backoff)
constexpr int kGroupM = 16;                        // tile rows per raster group

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// true once the phase with the given parity has completed; false after the spin limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// UMMA shared-memory descriptor: K-major operand staged by TMA with the 128-byte
// swizzle; 8-row groups 1024 bytes apart (stride byte offset), leading offset unused.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address, 16-byte units
  d |= (uint64_t)1 << 16;                          // leading byte offset (ignored here)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f8f6f4: A = B = e4m3, D = f32, both K-major, M=128, N=256.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// tile t of the grouped raster -> (tile_m, tile_n), kGroupM tile rows per group
__device__ __forceinline__ void tile_of(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
  const int per_group = kGroupM * tiles_n;
  const int first_m = (t / per_group) * kGroupM;
  const int gm = min(tiles_m - first_m, kGroupM);
  const int in_group = t % per_group;
  tm = first_m + in_group % gm;
  tn = in_group / gm;
}

// Persistent: each CTA takes tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... in the
// grouped raster.  The TMA ring runs on across tiles (k-block g of the CTA uses stage
// g % kStages); the accumulator alternates between two 256-column halves of TMEM, so
// the epilogue of one tile overlaps the MMAs of the next (tfull[b]: MMAs of buffer b
// done; tempty[b]: its 128 epilogue threads have read it).
__global__ void __launch_bounds__(kThreads, 1)
    k_dense_omega(const __grid_constant__ CUtensorMap amap, int32_t rows, int32_t kblocks,
                  int32_t tiles_m, int32_t tiles_n, uint16_t* __restrict__ omega, int64_t ld,
                  int* __restrict__ err) {
  extern __shared__ unsigned char dyn_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* base = (unsigned char*)(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;                                  // kStages x 16 KiB
  unsigned char* sB = base + kStages * kBM * kBK;            // kStages x 32 KiB
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull[2], tempty[2], tdone;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = tiles_m * tiles_n;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(&tdone, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = tmem_base;

  if (warp == 0) {
    if (lane == 0) {   // producer
      uint32_t g = 0;
      for (int t = blockIdx.x; t < ntiles && !*(volatile int*)&abort_flag; t += gridDim.x) {
        int tm, tn;
        tile_of(t, tiles_m, tiles_n, tm, tn);
        for (int kb = 0; kb < kblocks; ++kb, ++g) {
          const int s = (int)(g % kStages);
          const uint32_t round = g / kStages;
          if (g >= (uint32_t)kStages && !mbar_wait(&empty[s], (round & 1u) ^ 1u)) {
            atomicExch(&abort_flag, 1);
            break;
          }
          if (*(volatile int*)&abort_flag) break;
          mbar_expect_tx(&full[s], kStageBytes);
          tma_load_2d(sA + s * kBM * kBK, &amap, kb * kBK, tm * kBM, &full[s]);
          tma_load_2d(sB + s * kBN * kBK, &amap, kb * kBK, tn * kBN, &full[s]);
          tma_load_2d(sB + s * kBN * kBK + 128 * kBK, &amap, kb * kBK, tn * kBN + 128, &full[s]);
        }
      }
      if (*(volatile int*)&abort_flag) {
        // wait (bounded) for the copies this thread started that may still be landing
        const uint32_t first = g > (uint32_t)kStages ? g - kStages : 0u;
        for (uint32_t k = first; k < g; ++k)
          (void)mbar_wait(&full[k % kStages], (k / kStages) & 1u);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      uint32_t g = 0;
      int li = 0;   // tiles of this CTA so far
      bool issued_any = false;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++li) {
        if (*(volatile int*)&abort_flag) break;
        const int b = li & 1, n = li >> 1;   // accumulator half, its earlier uses
        if (n >= 1 && !mbar_wait(&tempty[b], (uint32_t)(n - 1) & 1u)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_d = tmem_d + (uint32_t)(b * kBN);
        bool ok = true;
        for (int kb = 0; kb < kblocks; ++kb, ++g) {
          const int s = (int)(g % kStages);
          if (!mbar_wait(&full[s], (g / kStages) & 1u)) {
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          if (*(volatile int*)&abort_flag) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * kBM * kBK), b0 = smem_u32(sB + s * kBN * kBK);
#pragma unroll
          for (int kk = 0; kk < kBK / 32; ++kk) {
            const uint64_t ad = umma_desc(a0 + kk * 32), bd = umma_desc(b0 + kk * 32);
            const uint32_t acc = (kb | kk) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_d),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                : "memory");
          }
          issued_any = true;
          umma_commit(&empty[s]);
        }
        if (!ok) break;
        umma_commit(&tfull[b]);
      }
      if (issued_any) {   // every MMA of this CTA has completed before TMEM is released
        umma_commit(&tdone);
        (void)mbar_wait(&tdone, 0);
      }
    }
  } else {   // warps 2-5: epilogue, warp w reads TMEM lanes 32 * (w % 4) ..
    const int q = warp & 3;
    int li = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++li) {
      const int b = li & 1, n = li >> 1;
      const bool ok = mbar_wait(&tfull[b], (uint32_t)n & 1u);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) atomicExch(&abort_flag, 1);
      if (!ok || *(volatile int*)&abort_flag) break;
      int tm, tn;
      tile_of(t, tiles_m, tiles_n, tm, tn);
      const int row = tm * kBM + q * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < kBN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem_d + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kBN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
            "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < rows) {
          // every accumulator is an integer <= 65,535 (heavy hyperedges are capped there)
          uint32_t packed[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const uint32_t lo = (uint32_t)__float2uint_rn(__uint_as_float(r[2 * j]));
            const uint32_t hi = (uint32_t)__float2uint_rn(__uint_as_float(r[2 * j + 1]));
            packed[j] = lo | (hi << 16);
          }
          uint4* dst = reinterpret_cast<uint4*>(omega + (int64_t)row * ld + tn * kBN + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            dst[j] = make_uint4(packed[4 * j], packed[4 * j + 1], packed[4 * j + 2], packed[4 * j + 3]);
        }
      }
      // this half of TMEM is read: the MMAs of the tile after next may overwrite it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&tempty[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicCAS(err, 0, DE_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ------------------------------------------------------------------ heavy set

// heavy_idx[i] = position of i in the heavy list, or -1; ids[pos] = i
__global__ void k_pick_heavy(const int32_t* __restrict__ esize, int32_t ne, int32_t min_size,
                             int32_t max_size, int32_t cap, int32_t* __restrict__ heavy_idx,
                             int32_t* __restrict__ ids, int32_t* __restrict__ count) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
    int32_t pos = -1;
    if (esize[i] >= min_size && esize[i] <= max_size) {
      pos = atomicAdd(count, 1);
      if (pos >= cap) pos = -1;   // beyond the cap: stays on the hash path
      else ids[pos] = i;
    }
    heavy_idx[i] = pos;
  }
}

// A[pos][v] = 1.0 in e4m3 (0x38) for every vertex v of heavy hyperedge ids[pos]
__global__ void k_fill_dense(const int64_t* __restrict__ e_ptr, const int32_t* __restrict__ e_idx,
                             const int32_t* __restrict__ ids, int32_t nh, uint8_t* __restrict__ a,
                             int64_t lda) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t h = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nh; h += warps) {
    const int32_t i = ids[h];
    for (int64_t p = e_ptr[i] + lane; p < e_ptr[i + 1]; p += 32) a[(int64_t)h * lda + e_idx[p]] = 0x38;
  }
}

__global__ void k_size_hist(const int32_t* __restrict__ esize, int32_t ne, int32_t max_bin,
                            unsigned long long* __restrict__ hist) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
    const int32_t s = esize[i] < max_bin ? esize[i] : max_bin;
    atomicAdd(&hist[s], 1ull);
  }
}

}  // namespace

size_t dense_smem_bytes() { return (size_t)kStages * kStageBytes + 1024; }

int64_t dense_round_rows(int64_t n) { return (n + kBN - 1) / kBN * kBN; }
int64_t dense_round_k(int64_t k) { return (k + kBK - 1) / kBK * kBK; }

void launch_size_hist(const int32_t* esize, int32_t ne, int32_t max_bin, unsigned long long* hist,
                      cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_size_hist<<<1024, 256, 0, s>>>(esize, ne, max_bin, hist);
}

void launch_pick_heavy(const int32_t* esize, int32_t ne, int32_t min_size, int32_t max_size,
                       int32_t cap, int32_t* heavy_idx, int32_t* ids, int32_t* count,
                       cudaStream_t s) {
  if (ne == 0) return;
  note_launch();
  k_pick_heavy<<<1024, 256, 0, s>>>(esize, ne, min_size, max_size, cap, heavy_idx, ids, count);
}

void launch_fill_dense(const int64_t* e_ptr, const int32_t* e_idx, const int32_t* ids, int32_t nh,
                       uint8_t* a, int64_t lda, cudaStream_t s) {
  if (nh == 0) return;
  note_launch();
  k_fill_dense<<<(nh + 7) / 8, 256, 0, s>>>(e_ptr, e_idx, ids, nh, a, lda);
}

// omega[rows_pad x rows_pad] (uint16, row stride ld = rows_pad) = A A^T for
// A[rows_pad x k_pad] e4m3.  Returns a CUDA error from the tensor-map encoding or the launch.
cudaError_t launch_dense_omega(const uint8_t* a, int64_t rows, int64_t rows_pad, int64_t k_pad,
                               uint16_t* omega, int* err, cudaStream_t s) {
  // looked up once (thread-safe static initialisation)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess) fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return cudaErrorNotSupported;
  if (rows_pad % kBN || k_pad % kBK || ((uintptr_t)a & 255) || ((uintptr_t)omega & 15))
    return cudaErrorInvalidValue;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows_pad};
  const cuuint64_t gstride[1] = {(cuuint64_t)k_pad};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, 128};
  const cuuint32_t estride[2] = {1, 1};
  CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)a, gdim, gstride, box, estride,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int smem = (int)dense_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_dense_omega, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles_m = rows_pad / kBM, tiles_n = rows_pad / kBN;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return cudaErrorInvalidValue;
  const int64_t ctas = std::min<int64_t>(tiles_m * tiles_n, nsm);   // one per SM, persistent
  note_launch();
  k_dense_omega<<<(unsigned)ctas, kThreads, smem, s>>>(
      map, (int32_t)rows, (int32_t)(k_pad / kBK), (int32_t)tiles_m, (int32_t)tiles_n, omega,
      rows_pad, err);
  return cudaGetLastError();
}

}  // namespace hg
