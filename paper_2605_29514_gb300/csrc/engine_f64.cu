// Complex128 instantiations of the round, init and dense-check kernels.
#include "engine_kernels.cuh"

namespace stn {

cudaError_t launch_round_f64(const EngineParams &p, int grid, cudaStream_t s) {
  return launch_round_t<double>(p, grid, s);
}

cudaError_t launch_init_f64(const EngineParams &p, cudaStream_t s) { return launch_init_t<double>(p, s); }

cudaError_t launch_dense_check_f64(int what, int m, int n, void *A, void *V, void *sig2, int use_smem,
                                     cudaStream_t s) {
  return launch_dense_check_t<double>(what, m, n, A, V, sig2, use_smem, s);
}

cudaError_t launch_dense_gemm_f64(int ta, int tb, int m, int n, int k, const double *alpha, const void *A, int lda,
                                  const void *B, int ldb, const double *beta, void *C, int ldc, int use_tc,
                                  int *status, cudaStream_t s) {
  return launch_dense_gemm_t<double>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, use_tc, status, s);
}

cudaError_t launch_diag_f64(const EngineParams &p, int what, int target, int cut, const int32_t *lq, int nl,
                            int letter, double *out, int *count, int grid, cudaStream_t s) {
  return launch_diag_t<double>(p, what, target, cut, lq, nl, letter, out, count, grid, s);
}

cudaError_t launch_adjoint_f64(const EngineParams &p, double *grad, int grid, cudaStream_t s) {
  return launch_adjoint_t<double>(p, grad, grid, s);
}

}  // namespace stn
