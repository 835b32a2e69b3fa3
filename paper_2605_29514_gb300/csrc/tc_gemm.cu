// Real GEMM on the fifth-generation tensor cores (tcgen05, sm_103a) with FP32
// accuracy from TF32 operands: C = A B with A (m x k) and B (k x n) row-major
// FP32.  Each operand is split into a TF32 head and a TF32 tail
// (a = a_hi + a_lo, both exactly representable), and
//     A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi
// is accumulated in FP32 in tensor memory (the 3-term split of Ootomo and
// Yokota, 2022); the dropped A_lo B_lo term is below FP32 rounding.  This is
// the contraction the MPS sweeps run as complex GEMMs (four real products
// each); here it stands alone on one CTA so that it can be checked against a
// plain product.
//
// One CTA of 128 threads (4 warps).  Output tiles of 128 x 64: the A tile
// (128 rows x 8 k) and the B tile (64 columns x 8 k) of each k step are
// written to shared memory in the no-swizzle K-major layout of the MMA
// (8 x 16-byte core matrices; the two core matrices along k 128 bytes apart,
// consecutive 8-row groups 256 bytes apart), made visible to the tensor
// cores by a proxy fence, and one thread issues the three MMAs
// (M = 128, N = 64, K = 8, kind::tf32) and commits them to an mbarrier that
// every thread waits on (a bounded wait: on time-out the kernel records an
// error, frees its tensor memory and returns).  The accumulator (128 lanes x
// 64 columns of FP32) is read back with tcgen05.ld, each warp reading its own
// 32 lanes.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/stn.h"

namespace stn {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTileM = 128, kTileN = 64, kTileK = 8;
constexpr uint32_t kTmemCols = 64;
constexpr long long kWaitLimit = 1ll << 22;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// TF32 rounding (round to nearest, ties away) of an FP32 value, returned as
// the FP32 number it represents.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, k) of a row x 8 tile in the no-swizzle
// K-major core-matrix layout.
__device__ __forceinline__ int core_offset(int row, int k) {
  return ((row >> 3) * 2 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// Shared-memory matrix descriptor: start address, leading byte offset (the
// next core matrix along k), stride byte offset (the next 8-row group),
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N = kTileN, M = kTileM.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(kTileN >> 3) << 17) |
                            (static_cast<uint32_t>(kTileM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem_d), "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ bool wait_barrier(uint32_t bar, uint32_t phase) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(int m, int n, int k, const float *A, const float *B, float *C, int *status) {
  __shared__ __align__(128) float a_hi[kTileM * kTileK], a_lo[kTileM * kTileK];
  __shared__ __align__(128) float b_hi[kTileN * kTileK], b_lo[kTileN * kTileK];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    failed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tmem_slot;
  const uint32_t bar_a = smem_addr(&bar);
  uint32_t phase = 0;
  const uint64_t dah = make_desc(smem_addr(a_hi), 128, 256), dal = make_desc(smem_addr(a_lo), 128, 256);
  const uint64_t dbh = make_desc(smem_addr(b_hi), 128, 256), dbl = make_desc(smem_addr(b_lo), 128, 256);
  for (int i0 = 0; i0 < m && !failed; i0 += kTileM) {
    for (int j0 = 0; j0 < n && !failed; j0 += kTileN) {
      for (int k0 = 0; k0 < k; k0 += kTileK) {
        for (int e = t; e < kTileM * kTileK; e += kTcThreads) {
          const int r = e / kTileK, c = e % kTileK;
          const float v = (i0 + r < m && k0 + c < k) ? A[static_cast<int64_t>(i0 + r) * k + k0 + c] : 0.f;
          const float hi = to_tf32(v);
          const int o = core_offset(r, c) >> 2;
          a_hi[o] = hi;
          a_lo[o] = to_tf32(v - hi);
        }
        for (int e = t; e < kTileN * kTileK; e += kTcThreads) {
          const int c = e / kTileN, j = e % kTileN;  // consecutive threads: consecutive columns of B
          const float v = (j0 + j < n && k0 + c < k) ? B[static_cast<int64_t>(k0 + c) * n + j0 + j] : 0.f;
          const float hi = to_tf32(v);
          const int o = core_offset(j, c) >> 2;
          b_hi[o] = hi;
          b_lo[o] = to_tf32(v - hi);
        }
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        if (t == 0) {
          mma_tf32(tmem, dah, dbh, k0 > 0 ? 1u : 0u);
          mma_tf32(tmem, dah, dbl, 1u);
          mma_tf32(tmem, dal, dbh, 1u);
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_a)
                       : "memory");
        }
        if (!wait_barrier(bar_a, phase)) {
          if (lane == 0) atomicExch(&failed, 1);
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        __syncthreads();
        if (failed) break;
      }
      if (failed) break;
      // accumulator rows 32 warp .. 32 warp + 31, 64 columns, 16 at a time
      for (int c0 = 0; c0 < kTileN; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * warp) << 16) + c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        const int row = i0 + 32 * warp + lane;
        if (row < m) {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (j0 + c0 + c < n) C[static_cast<int64_t>(row) * n + j0 + c0 + c] = __uint_as_float(v[c]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n");
    }
  }
  if (failed) {  // give the MMAs in flight a last bounded chance to land
    wait_barrier(bar_a, phase);
    if (t == 0) *status = STN_ETIMEOUT;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace
}  // namespace stn

extern "C" stn_status stn_dense_gemm_tc(int32_t m, int32_t n, int32_t k, const float *d_a, const float *d_b,
                                        float *d_c, int32_t *d_status, void *cuda_stream) {
  if (m < 1 || n < 1 || k < 1 || m > 4096 || n > 4096 || k > 4096 || !d_a || !d_b || !d_c || !d_status)
    return STN_EINVAL;
  stn::tc_gemm_kernel<<<1, stn::kTcThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(m, n, k, d_a, d_b, d_c,
                                                                                       d_status);
  return cudaGetLastError() == cudaSuccess ? STN_OK : STN_ECUDA;
}
