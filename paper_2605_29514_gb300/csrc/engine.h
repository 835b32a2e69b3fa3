// Device-side parameter block and host launchers of the simulation kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "program.h"

namespace stn {

constexpr int kThreads = 512;   // threads per CTA of the round kernel (16 warps)
constexpr double kNearThreshold = 1e-5;
// Phase counters (SM clock cycles of the CTA, summed over ops): left sweep,
// right-sweep SVDs, the rest of the right sweep, expectation values, the whole
// op loop; counts of small (shared-memory) and large-bond SVDs; gauge-move
// cycles and the number of sites they crossed; the cycles of the small SVDs
// (a part of the SVD cycles); the Jacobi sweeps of the large-bond SVDs and
// the cycles of their Householder R factors (a part of the SVD cycles).
constexpr int kProfSlots = 15;
enum ProfSlot { PROF_LEFT = 0, PROF_SVD, PROF_RIGHT, PROF_EXPECT, PROF_OPS, PROF_NSVD_SMALL,
                PROF_NSVD_LARGE, PROF_GAUGE, PROF_NGAUGE, PROF_SVD_SMALL, PROF_JSWEEPS, PROF_SVD_QR,
                PROF_JROWS, PROF_JCOLS, PROF_JAC_ROWS256 };

// Everything one segment launch needs.  Per-shot arrays are indexed by the
// shot's position in the batch; per-CTA scratch by blockIdx.x.
struct EngineParams {
  const Op *ops;
  int op_begin, op_end;
  const double *theta;  // [K]
  int n, W, n_meas, rec_bytes;
  int chi_cap;
  double cutoff, delta;
  double p1, p2, pR, pM;
  uint64_t seed, shot_offset;
  const uint64_t *shot_offset_dev;  // when set, the offset is read here (captured graphs)
  int shots;
  // frame: inverse tableau rows X_0..X_{n-1}, Z_0..Z_{n-1}
  uint64_t *tab_x, *tab_z;  // [shot][2n][W]
  uint8_t *tab_m;           // [shot][2n]
  // MPS: site k of a shot at slab + site_off[k], shape (chi[k], 2, chi[k+1])
  void *mps;
  const int64_t *site_off;  // [n+1]
  const int *chimax;        // [n+1] largest possible bond (cap and 2^min(k, n-k))
  int64_t slab_elems;
  int *chi;                 // [shot][n+1], chi[0] = chi[n] = 1
  int *center;              // [shot]
  double *logp, *disc;      // [shot]
  int *maxchi, *near, *status;  // [shot]
  uint8_t *records;         // [shot][rec_bytes]
  double *born;             // [shot][n_meas]
  double *flops;            // [shot] algorithmic FLOPs, cumulative over batches
  double *prof;             // [shot][kProfSlots] SM cycles per phase, cumulative
  // per-CTA scratch, complex elements of the path's precision
  void *scratch;
  int64_t scratch_elems, ap_elems, g_elems;
  int work_c;               // largest bond of the plan (sizes the work area)
  int svd_elems;            // complex elements of the shared-memory SVD buffer
  int svd64_all;            // complex64 path: every bond SVD in double precision
  int use_tc;               // complex64 and gemm_units = STN_GEMM_TENSOR: large contractions on tcgen05
  int *err;                 // first error code seen on the device
  int *ticket;              // shot queue of a launch (zeroed before it), or null: grid-stride
  // Adjoint of log P(record) (all null in an ordinary run).  forced: records
  // to reproduce, [shot][rec_bytes]; a measurement's outcome is then its
  // record bit XOR its record-flip event.  With tape_info set, rotations and
  // measurements write what the backward pass needs: the conjugated Pauli
  // (tape_px/pz [shot][op][W]), tape_info [shot][op][kTapeInts], and after
  // each rotation the state (phi_* [shot][rotation ordinal]).
  const uint8_t *forced;
  uint64_t *tape_px, *tape_pz;
  int32_t *tape_info;
  void *phi_store;          // [shot][n_rot][slab_elems] complex of the precision
  int *phi_chi;             // [shot][n_rot][n + 1]
  const int32_t *rot_ord;   // [op] ordinal of a rotation among the shot's rotations, -1 otherwise
  int n_ops_total, n_rot;
};

// tape_info entries of an op: [0] phase m of P' | case B << 2 | outcome << 3
// | lidx << 4 | sign(P') < 0 << 6, [1] lo, [2] hi, [3] j
constexpr int kTapeInts = 4;

struct ScratchPlan {
  int64_t ap_elems, g_elems, work_elems, total;
  int work_c;
};

ScratchPlan plan_scratch(int n, const int *chimax, int chi_cap);
size_t round_kernel_smem(int precision, int n, int W, int svd_elems);
int round_kernel_svd_elems(int precision, int n, int W);
int jacobi_smem_limit(int precision);

cudaError_t launch_init(int precision, const EngineParams &p, cudaStream_t s);
// per-precision instantiations (engine_f32.cu, engine_f64.cu)
cudaError_t launch_round_f32(const EngineParams &p, int grid, cudaStream_t s);
cudaError_t launch_round_f64(const EngineParams &p, int grid, cudaStream_t s);
cudaError_t launch_init_f32(const EngineParams &p, cudaStream_t s);
cudaError_t launch_init_f64(const EngineParams &p, cudaStream_t s);
cudaError_t launch_dense_check_f32(int what, int m, int n, void *A, void *V, void *sig2, int use_smem,
                                   cudaStream_t s);
cudaError_t launch_dense_check_f64(int what, int m, int n, void *A, void *V, void *sig2, int use_smem,
                                   cudaStream_t s);
cudaError_t launch_round(int precision, const EngineParams &p, int grid, cudaStream_t s);
cudaError_t launch_adjoint_f32(const EngineParams &p, double *grad, int grid, cudaStream_t s);
cudaError_t launch_adjoint_f64(const EngineParams &p, double *grad, int grid, cudaStream_t s);
cudaError_t launch_diag_f32(const EngineParams &p, int what, int target, int cut, const int32_t *lq, int nl,
                            int letter, double *out, int *count, int grid, cudaStream_t s);
cudaError_t launch_diag_f64(const EngineParams &p, int what, int target, int cut, const int32_t *lq, int nl,
                            int letter, double *out, int *count, int grid, cudaStream_t s);
cudaError_t launch_dense_check(int precision, int what, int m, int n, void *A, void *V, void *sig2,
                               int use_smem, cudaStream_t s);
// C = alpha op(A) op(B) + beta C on one CTA through the sweeps' cgemm
// (alpha, beta: host re/im pairs); use_tc: complex64 on the tensor cores
cudaError_t launch_dense_gemm_f32(int ta, int tb, int m, int n, int k, const double *alpha, const void *A, int lda,
                                  const void *B, int ldb, const double *beta, void *C, int ldc, int use_tc,
                                  int *status, cudaStream_t s);
cudaError_t launch_dense_gemm_f64(int ta, int tb, int m, int n, int k, const double *alpha, const void *A, int lda,
                                  const void *B, int ldb, const double *beta, void *C, int ldc, int use_tc,
                                  int *status, cudaStream_t s);
int svd_smem_elems(int precision);
size_t noalloc_scratch_bytes();
cudaError_t launch_svd_noalloc(int precision, int m, int n, const void *C, void *V, void *sig2,
                               cudaStream_t s);
cudaError_t launch_detectors(const uint8_t *records, int rec_bytes, int64_t shots, const int32_t *det,
                             int n_det, const int32_t *logical, int n_logical, uint8_t *out_det,
                             uint8_t *out_obs, cudaStream_t s);
cudaError_t launch_philox(uint64_t seed, uint64_t shot_offset, int64_t n_shots,
                          uint32_t event_offset, int n_events, double *out, cudaStream_t s);

}  // namespace stn
