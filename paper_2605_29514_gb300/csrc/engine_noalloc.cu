#include "engine_kernels.cuh"

#include <mutex>

namespace stn {

// ---------------------------------------------------------------------------
// Allocation-free large-bond SVD.  Some callers cannot allocate device memory
// at the moment they need this routine: code running inside a host callback
// or under a framework's memory pool that forbids cudaMalloc mid-stream, or an
// embedded runtime that hands out only the buffers it owns.  For them the work
// copy of the input lives in this file-scope array instead of a buffer the
// caller or the library would allocate.  Every GPU that loads the library
// holds the array until the process exits.  All calls share it: it keeps the
// last call's contents, and two calls that overlap on the GPU (different
// streams, or different host threads on one stream without ordering) race
// on it.  Each call writes every scratch element it later reads, so nothing
// has to start at zero.
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) svd_noalloc_kernel(int m, int n, const cplx<T> *C,
                                                                  cplx<T> *work, cplx<T> *V, T *sig2) {
  extern __shared__ __align__(16) char smem_raw[];
  tc_disable();
  double *red = reinterpret_cast<double *>(smem_raw);
  double *dm = red + kThreads;
  int *flag = reinterpret_cast<int *>(dm + 16);
  cplx<T> *buf = reinterpret_cast<cplx<T> *>(flag + 16) + kMaxVec;
  float *rv_wrk = reinterpret_cast<float *>(buf + SvdSmem<T>::elems);
  for (int e = tid(); e < m * n; e += kThreads) work[e] = C[e];
  __syncthreads();
  // the large-bond path of the truncation sweep on the work copy: R factor,
  // Jacobi on X = R^dag, V = normalised columns of X
  qr_r_inplace<T>(m, n, work, n, buf, SvdSmem<T>::elems, red, dm);
  const int k = min(m, n);
  const bool regs = sizeof(T) == 4 && k > 16 && n <= kThreads;
  const bool x_smem = !regs && n * k <= SvdSmem<T>::elems;
  cplx<T> *Xc = x_smem ? buf : work;
  for (int e = tid(); e < n * k; e += kThreads) Xc[e] = cconj(work[e]);
  __syncthreads();
  if (x_smem) svd_onesided<T>(n, k, Xc, nullptr, sig2, flag, red);
  else svd_onesided_blocked<T>(n, k, Xc, nullptr, sig2, flag, red, buf, SvdSmem<T>::elems,
                               regs ? rv_wrk : nullptr);
  for (int e = tid(); e < n * n; e += kThreads) {
    const int c = e / n;
    const T l = c < k ? sig2[c] : T(0);
    V[e] = l > T(0) ? cscale(Xc[e], T(1) / sqrt(l)) : cmake<T>(0, 0);
  }
  for (int c = k + tid(); c < n; c += kThreads) sig2[c] = T(0);
}

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

// Device address of the scratch array on the current device.  Host code may
// not pass g_noalloc_scratch itself: on the host that name is a stand-in, not
// a device address.  The address is looked up once per device, with that
// device current, on the first call made there.
static cudaError_t noalloc_scratch_ptr(void **out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static void *ptr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (ptr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    ptr[dev] = p;
  }
  *out = ptr[dev];
  return cudaSuccess;
}

template <typename T>
static cudaError_t launch_svd_noalloc_t(int m, int n, const void *C, void *V, void *sig2, cudaStream_t s) {
  void *work = nullptr;
  cudaError_t e = noalloc_scratch_ptr(&work);
  if (e != cudaSuccess) return e;
  size_t smem = sizeof(double) * (kThreads + 16) + sizeof(int) * 16 + sizeof(cplx<T>) * kMaxVec +
                sizeof(cplx<T>) * SvdSmem<T>::elems + sizeof(float) * kRvWrkFloats;
  e = cudaFuncSetAttribute(svd_noalloc_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  svd_noalloc_kernel<T><<<1, kThreads, smem, s>>>(m, n, static_cast<const cplx<T> *>(C),
                                                  static_cast<cplx<T> *>(work), static_cast<cplx<T> *>(V),
                                                  static_cast<T *>(sig2));
  return cudaGetLastError();
}

cudaError_t launch_svd_noalloc(int precision, int m, int n, const void *C, void *V, void *sig2,
                               cudaStream_t s) {
  return precision == 0 ? launch_svd_noalloc_t<double>(m, n, C, V, sig2, s)
                        : launch_svd_noalloc_t<float>(m, n, C, V, sig2, s);
}

}  // namespace stn
