// Arithmetic-peak probes: dense chains of independent FP32 FMAs, FP64 FMAs
// and TF32 tensor-core products (mma.sync m16n8k8, FP32 accumulation), run
// on every SM at full occupancy.  The caller times a launch with CUDA events
// and divides the returned FLOP count by it; the rates are the denominators
// of the roofline of the MPS sweeps (CUDA-core FP32 for the contractions and
// Jacobi rotations, FP64 for the double-precision SVDs, TF32 for what a
// tensor-core path could reach).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/stn.h"

namespace stn {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe(int64_t iters, T seed, int keep, T *out) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + static_cast<T>(threadIdx.x + c);
  const T b = seed * static_cast<T>(0.999), d = static_cast<T>(1e-3);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (keep) out[blockIdx.x] = s;  // keep = 0 from the host: never taken, keeps the chains alive
}

// D = A B + D on m16n8k8 TF32 fragments, four independent accumulators.
__global__ void __launch_bounds__(kProbeThreads) tf32_probe(int64_t iters, float seed, int keep, float *out) {
  uint32_t a[4], b[2];
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = __float_as_uint(seed + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  }
  b[0] = __float_as_uint(seed * 0.5f);
  b[1] = __float_as_uint(seed * 0.25f);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[c][j];
  if (keep) out[blockIdx.x] = s;  // never taken (keep = 0)
}

}  // namespace stn

extern "C" stn_status stn_peak_probe(int32_t kind, int64_t iters, double *h_flops, void *cuda_stream) {
  if (kind < 0 || kind > 2 || iters < 1 || !h_flops) return STN_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
    return STN_ECUDA;
  const int grid = sms * (per_sm / stn::kProbeThreads);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const double threads = static_cast<double>(grid) * stn::kProbeThreads;
  if (kind == 0) {
    stn::fma_probe<float><<<grid, stn::kProbeThreads, 0, s>>>(iters, 1.0001f, 0, nullptr);
    *h_flops = threads * iters * 16 * stn::kChains * 2.0;
  } else if (kind == 1) {
    stn::fma_probe<double><<<grid, stn::kProbeThreads, 0, s>>>(iters, 1.0001, 0, nullptr);
    *h_flops = threads * iters * 16 * stn::kChains * 2.0;
  } else {
    stn::tf32_probe<<<grid, stn::kProbeThreads, 0, s>>>(iters, 1.0001f, 0, nullptr);
    *h_flops = (threads / 32.0) * iters * 16 * (2.0 * 16 * 8 * 8);
  }
  return cudaGetLastError() == cudaSuccess ? STN_OK : STN_ECUDA;
}
