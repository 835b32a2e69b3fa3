// Host side of the simulation kernels: launch dispatch by precision, scratch
// planning, and the small kernels (Philox uniforms, detectors).  The round,
// init and dense-check kernels are instantiated in engine_f32.cu and
// engine_f64.cu; the allocation-free SVD lives in engine_noalloc.cu.
#include "engine_kernels.cuh"

namespace stn {

// Philox uniforms for tests: out[s][e] = u(seed, shot_offset + s, event_offset + e).
__global__ void philox_kernel(uint64_t seed, uint64_t shot_offset, int64_t n_shots,
                              uint32_t event_offset, int n_events, double *out) {
  int64_t total = n_shots * static_cast<int64_t>(n_events);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t s = i / n_events;
    uint32_t e = static_cast<uint32_t>(i % n_events);
    out[i] = philox_uniform(seed, shot_offset + static_cast<uint64_t>(s), event_offset + e);
  }
}

// ---------------------------------------------------------------------------
// Detector bits and the Z_L parity of every shot from its packed record: one
// thread per (shot, detector byte), the last slot of a shot computing Z_L.
__global__ void detector_kernel(const uint8_t *rec, int rec_bytes, int64_t shots, const int32_t *det,
                                int n_det, const int32_t *logical, int n_logical, uint8_t *out_det,
                                uint8_t *out_obs) {
  const int det_bytes = (n_det + 7) / 8;
  const int64_t total = shots * (det_bytes + 1);
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t shot = e / (det_bytes + 1);
    const int j = static_cast<int>(e % (det_bytes + 1));
    const uint8_t *r = rec + shot * rec_bytes;
    if (j < det_bytes) {
      unsigned v = 0;
      for (int b = 0; b < 8 && j * 8 + b < n_det; ++b) {
        const int32_t *row = det + (j * 8 + b) * kDetWidth;
        unsigned par = 0;
        for (int k = 0; k < kDetWidth; ++k)
          if (row[k] >= 0) par ^= (r[row[k] >> 3] >> (row[k] & 7)) & 1u;
        v |= par << b;
      }
      out_det[shot * det_bytes + j] = static_cast<uint8_t>(v);
    } else {
      unsigned par = 0;
      for (int k = 0; k < n_logical; ++k) par ^= (r[logical[k] >> 3] >> (logical[k] & 7)) & 1u;
      out_obs[shot] = static_cast<uint8_t>(par);
    }
  }
}

cudaError_t launch_detectors(const uint8_t *records, int rec_bytes, int64_t shots, const int32_t *det,
                             int n_det, const int32_t *logical, int n_logical, uint8_t *out_det,
                             uint8_t *out_obs, cudaStream_t s) {
  const int64_t total = shots * ((n_det + 7) / 8 + 1);
  if (total <= 0) return cudaSuccess;
  int grid = static_cast<int>((total + 255) / 256);
  if (grid > 4096) grid = 4096;
  detector_kernel<<<grid, 256, 0, s>>>(records, rec_bytes, shots, det, n_det, logical, n_logical, out_det,
                                       out_obs);
  return cudaGetLastError();
}

int svd_smem_elems(int precision) { return precision == 0 ? SvdSmem<double>::elems : SvdSmem<float>::elems; }

// ---------------------------------------------------------------------------
// host side
ScratchPlan plan_scratch(int n, const int *chimax, int chi_cap) {
  ScratchPlan p{};
  int64_t ap = 0, g = 0;
  int cmax = 1;
  for (int k = 0; k < n; ++k) ap += 8ll * chimax[k] * chimax[k + 1];
  for (int k = 1; k < n; ++k) g += 4ll * chimax[k] * chimax[k];
  for (int k = 0; k <= n; ++k) cmax = chimax[k] > cmax ? chimax[k] : cmax;
  (void)chi_cap;
  int64_t c2 = static_cast<int64_t>(cmax) * cmax;
  p.work_c = cmax;
  p.ap_elems = ap;
  p.g_elems = g;
  p.work_elems = 35 * c2 + 4ll * cmax + 1024;
  p.total = ap + g + p.work_elems;
  return p;
}

// Largest SVD buffer (complex elements, at most SvdSmem) that keeps the round
// kernel within the 227 KB of shared memory a CTA may use.
template <typename T>
static int svd_elems_for(int n, int W) {
  const size_t limit = 227 * 1024;
  size_t base = smem_bytes<T>(n, W, 0);
  if (base + 64 >= limit) return 0;
  size_t e = (limit - base - 64) / sizeof(cplx<T>);
  return static_cast<int>(e < static_cast<size_t>(SvdSmem<T>::elems) ? e : SvdSmem<T>::elems);
}

int round_kernel_svd_elems(int precision, int n, int W) {
  return precision == 0 ? svd_elems_for<double>(n, W) : svd_elems_for<float>(n, W);
}

size_t round_kernel_smem(int precision, int n, int W, int svd_elems) {
  return precision == 0 ? smem_bytes<double>(n, W, svd_elems) : smem_bytes<float>(n, W, svd_elems);
}

int jacobi_smem_limit(int precision) {
  return precision == 0 ? SvdSmem<double>::elems : SvdSmem<float>::elems;
}


cudaError_t launch_init(int precision, const EngineParams &p, cudaStream_t s) {
  return precision == 0 ? launch_init_f64(p, s) : launch_init_f32(p, s);
}


cudaError_t launch_round(int precision, const EngineParams &p, int grid, cudaStream_t s) {
  return precision == 0 ? launch_round_f64(p, grid, s) : launch_round_f32(p, grid, s);
}

cudaError_t launch_dense_check(int precision, int what, int m, int n, void *A, void *V, void *sig2,
                               int use_smem, cudaStream_t s) {
  return precision == 0 ? launch_dense_check_f64(what, m, n, A, V, sig2, use_smem, s)
                        : launch_dense_check_f32(what, m, n, A, V, sig2, use_smem, s);
}

cudaError_t launch_philox(uint64_t seed, uint64_t shot_offset, int64_t n_shots, uint32_t event_offset,
                          int n_events, double *out, cudaStream_t s) {
  int64_t total = n_shots * n_events;
  if (total <= 0) return cudaSuccess;
  int grid = static_cast<int>((total + 255) / 256);
  if (grid > 65535) grid = 65535;
  philox_kernel<<<grid, 256, 0, s>>>(seed, shot_offset, n_shots, event_offset, n_events, out);
  return cudaGetLastError();
}

}  // namespace stn
