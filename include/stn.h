/*
 * stn.h — C ABI of a GB300 (sm_103a) stabilizer-tensor-network simulator of
 * noisy rotated-surface-code syndrome extraction under coherent crosstalk.
 *
 * Method (Harper, Nakhl, Sevior, Usman, "Non-Clifford Crosstalk Noise in
 * Surface Codes Using Hybrid Stabilizer-Tensor Network Methods"):
 *   - each shot is |psi> = C |MPS> (Eq. 7): a Clifford frame C held as an
 *     inverse tableau, times a matrix product state;
 *   - Clifford gates and Pauli noise (Eq. 2-3, Table I) update C only;
 *   - a crosstalk rotation exp(-i theta P) (Eq. 4) and a Pauli measurement are
 *     pushed through C (Sec. IV A) and applied to the MPS as a bond-2 Pauli
 *     MPO, followed by truncation to a bond-dimension cap (Sec. IV B, Eq. 8);
 *   - the surface code layout and the Z/X syndrome circuits are those of
 *     Sec. II and Fig. 1, repeated for `rounds` rounds.
 *
 * Conventions shared by every call:
 *   - All pointers named h_* are host memory owned by the caller; d_* are
 *     device memory owned by the caller.  The context owns all other device
 *     memory (tableaux, MPS arenas, scratch) and frees it in stn_destroy.
 *   - Every call returns a stn_status and never aborts.  On failure the
 *     reason is kept in the context (stn_last_error).  Device-side failures
 *     (arena overflow, non-finite numbers) are recorded on the device and
 *     reported by the next call that synchronises (stn_sync, stn_read_*).
 *   - A context is bound to one CUDA stream (given at creation) and is not
 *     thread-safe.  Work is enqueued on that stream; calls that return host
 *     data synchronise it.
 *   - Shot s of a batch started at `shot_offset` draws every random number
 *     from Philox4x32-10 (Salmon et al., SC'11) with key = seed and counter =
 *     (global shot index, event id), so batches and shards are reproducible
 *     and independent of batch size.
 */
#ifndef STN_H
#define STN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stn_ctx stn_ctx;

typedef enum {
  STN_OK = 0,
  STN_EINVAL = 1,   /* invalid argument or configuration */
  STN_ENOMEM = 2,   /* device allocation failed */
  STN_ECUDA = 3,    /* CUDA runtime error */
  STN_ETIMEOUT = 4, /* a bounded device wait ran out */
  STN_ENUMERIC = 5, /* non-finite or vanishing norm in the MPS */
  STN_ENOTIMPL = 6, /* entry point not implemented */
  STN_EOVERFLOW = 7 /* a device arena was too small */
} stn_status;

enum { STN_PAIRS_ADJACENT_IDLE = 0, STN_PAIRS_ADJACENT_IDLE_DIAG_XX = 1 };
/* Arithmetic of the MPS path.  C128: complex128 throughout.  C64: complex64
 * contractions; norms, Born probabilities and log P in double; the SVDs of
 * bonds whose complex128 copy fits shared memory (about 75 columns) in double
 * precision, larger bonds by single-precision Jacobi on the R factor.
 * C64_SVD64: as C64 with every bond SVD (R factor and Jacobi) in double
 * precision, at the FP64 rate of the GPU. */
enum { STN_PRECISION_C128 = 0, STN_PRECISION_C64 = 1, STN_PRECISION_C64_SVD64 = 2 };
enum { STN_BASIS_Z = 0, STN_BASIS_X = 1 };
enum { STN_LAYERS_IDLE = 0xFF }; /* pair_layer_mask entry: use the idle rule */
enum { STN_GEMM_FMA = 0, STN_GEMM_TENSOR = 1 }; /* stn_config.gemm_units */

/* Simulation parameters: the problem statement of Sec. II-III (code
 * distance, rounds, CNOT schedule, crosstalk pairs and angles, Pauli noise
 * rates) and the truncation of Sec. IV B.  Rates follow Table I:
 * p1 = p1_scale*p after each single-qubit gate (Eq. 2), p2 = p2_scale*p
 * after each CNOT (Eq. 3), pR = pR_scale*p X flip after each reset,
 * pM = pM_scale*p flip of each recorded bit.
 *
 * Qubits are numbered 0..n-1 in row-major (y, x) order of the layout
 * (stn_layout gives coordinates and kinds): data qubit (column i, row j) at
 * (2i+1, 2j+1), face (i, j) at (2i, 2j), X type when i + j is odd.  The
 * ancillas, in ascending qubit order, index the rows of cnot_schedule.
 * stn_create deep-copies every array; the caller keeps ownership. */
typedef struct {
  int32_t distance;      /* code distance d >= 3, odd; n = 2 d^2 - 1 qubits */
  int32_t rounds;        /* syndrome rounds >= 1 (Sec. II: d rounds) */
  int32_t pair_rule;     /* STN_PAIRS_*: which pairs get crosstalk (Sec. III B)
                            when n_pairs = 0 */
  int32_t chi_cap;       /* bond-dimension cap chi_max (Sec. IV B), 1..256 */
  double p, p1_scale, p2_scale, pR_scale, pM_scale;
  double svd_cutoff;     /* drop Schmidt values <= svd_cutoff * s_1 */
  double degeneracy_tol; /* at the cap, kept values exceed the first dropped
                            one by more than degeneracy_tol * s_1 */
  int32_t precision;     /* STN_PRECISION_*: arithmetic of the MPS path */
  uint64_t seed;         /* Philox key */
  int32_t memory_basis;  /* STN_BASIS_Z: data prepared and read out in Z,
                            detectors on Z faces, logical Z_L on the top data
                            row; STN_BASIS_X: H after the data reset and
                            before the readout, X faces, X_L on the left
                            data column */
  int32_t n_pairs;       /* K > 0: the explicit pairs below replace pair_rule */
  const int32_t *cnot_schedule;  /* [d^2 - 1][4] (ancillas in ascending qubit
                            order): the data qubit each ancilla's CNOT gates in
                            layers 0..3 of Fig. 1, or -1 for an idle layer;
                            every face qubit exactly once, no qubit twice in a
                            layer.  NULL: the hook-avoiding default (Z faces
                            NW, SW, NE, SE; X faces NW, NE, SW, SE) */
  const int32_t *pairs;           /* [K][2] qubits of crosstalk pair k (Eq. 4) */
  const uint8_t *pair_pauli;      /* [K] 0: exp(-i theta Z Z), 1: X X; NULL = ZZ */
  const uint8_t *pair_layer_mask; /* [K] bit l: the rotation acts after CNOT
                            layer l; STN_LAYERS_IDLE (or a NULL array) = after
                            every layer in which no CNOT acts on exactly that
                            pair (Sec. III B, Fig. 1) */
  int64_t arena_cap_bytes; /* 0: each resident shot's stack of doubled span
                            tensors and R factors is sized for the largest
                            span the cap allows; > 0: that stack is capped at
                            this many bytes, and a sweep that needs more stops
                            its shot with STN_EOVERFLOW (reported by the next
                            synchronising call) */
  int32_t gemm_units;      /* STN_GEMM_FMA (0, the default): every contraction
                            on the CUDA cores (FP32 FMA for complex64);
                            STN_GEMM_TENSOR (1): complex64 contractions of at
                            least 64 x 32 x 16 on the tcgen05 tensor cores
                            (TF32 operands split into head and tail, about 22
                            bits each, FP32 accumulation).  The split's
                            products are a few times less accurate than FP32
                            FMA ones, and the sweeps carry that into the Born
                            probabilities.  Complex128 always uses the CUDA
                            cores */
} stn_config;

/* Per-shot diagnostics of the last batch (Sec. IV B: truncation). */
typedef struct {
  int32_t max_chi;   /* largest bond dimension reached */
  int32_t near_draws; /* Born draws with |u - p0| < 1e-5 */
  double discarded;  /* sum over truncations of the discarded weight */
  double logp;       /* log-probability of the realised outcomes */
} stn_shot_stats;

/* Host-only layout of the distance-d rotated code (Sec. II, Fig. 1; no GPU
 * needed): h_xy[2n] the (x, y) coordinates of qubit q at h_xy[2q], h_kind[n]
 * 'D' (data), 'X' or 'Z' (ancilla of that face type); either may be NULL.
 * Returns n, or -1 for a distance that is not odd and in 3..11. */
int32_t stn_layout(int32_t distance, int32_t *h_xy, char *h_kind);

/* Compile the program (Sec. II-III: layout, CNOT schedule, crosstalk pairs,
 * noise events, measurement records) and allocate device state for up to
 * max_shots shots per batch.  `cuda_stream` is a cudaStream_t (NULL = legacy
 * default stream).  On success *out owns the context.  Errors: STN_EINVAL
 * (bad config: distance, rounds, rates, a schedule that does not gate every
 * face qubit once or gates a qubit twice in a layer, a pair out of range),
 * STN_ENOMEM, STN_ECUDA. */
stn_status stn_create(const stn_config *cfg, int64_t max_shots, void *cuda_stream,
                      stn_ctx **out);
void stn_destroy(stn_ctx *ctx);
const char *stn_last_error(const stn_ctx *ctx);

/* Sizes of the compiled program: qubits, crosstalk pairs K (the length of
 * every theta table), measurement records per shot, random events per shot,
 * ops per shot. */
int32_t stn_num_qubits(const stn_ctx *ctx);
int32_t stn_num_pairs(const stn_ctx *ctx);
int32_t stn_num_meas(const stn_ctx *ctx);
int32_t stn_num_events(const stn_ctx *ctx);
int32_t stn_num_ops(const stn_ctx *ctx);

/* Copy the compiled program to the host: ops[i] = {kind, a, b, pauli, ev, idx}
 * as six int32 per op (kinds: 1 reset flip, 2 H, 3 1q noise, 4 CNOT,
 * 5 2q noise, 6 rotation, 7 Z measurement; for 7, pauli = 1 when the qubit
 * is reset afterwards), and pairs[k] = {a, b, pauli(0 ZZ, 1 XX), layer_mask}.
 * Either pointer may be NULL. */
stn_status stn_get_program(const stn_ctx *ctx, int32_t *h_ops, int32_t *h_pairs);

/* Host-only (no GPU needed): compile the program of `cfg` and report its
 * sizes h_counts[5] = {qubits, pairs K, measurements, events, ops}; when
 * h_ops / h_pairs are not NULL, also copy the ops and pairs as in
 * stn_get_program (the caller sizes them from a first call with NULL).
 * Errors: STN_EINVAL for a bad config. */
stn_status stn_compile_program(const stn_config *cfg, int32_t *h_counts, int32_t *h_ops,
                               int32_t *h_pairs);

/* Start a batch of `shots` shots (<= max_shots) with global indices
 * shot_offset .. shot_offset+shots-1: every tableau is reset to the identity
 * frame and every MPS to |0...0>.  Asynchronous. */
stn_status stn_begin_batch(stn_ctx *ctx, int64_t shots, uint64_t shot_offset);

/* Apply program segment `round` to every shot of the batch, with per-pair
 * crosstalk angles h_theta[K] (host, radians).  Segments are 0..rounds:
 * segment 0 holds the initial resets and syndrome round 0, segment r the
 * syndrome round r, segment `rounds` the final Z readout of the data qubits.
 * One persistent kernel launch per segment.  Asynchronous. */
stn_status stn_apply_round(stn_ctx *ctx, int32_t round, const double *h_theta);

/* Same, with the angles already in device memory (d_theta[K], doubles). */
stn_status stn_apply_round_device(stn_ctx *ctx, int32_t round, const double *d_theta);

/* The same program in finer launches: layer step s (0 .. 4 rounds - 1) is
 * CNOT layer s % 4 of syndrome round s / 4 (Fig. 1) with the crosstalk
 * rotations after it (Sec. III B); the first layer of a round also holds the
 * round's opening H gates (round 0: the initial resets too), the last layer
 * its closing H gates and ancilla measurements, and the last step the final
 * data readout.  Running steps 0..4 rounds - 1 in order does exactly what
 * running rounds 0..rounds does.  stn_num_steps returns 4 rounds.  One
 * persistent kernel launch per step, angles d_theta[K] in device memory.
 * Asynchronous.  Errors: STN_EINVAL for a bad step or no batch. */
int32_t stn_num_steps(const stn_ctx *ctx);
stn_status stn_apply_step_device(stn_ctx *ctx, int32_t step, const double *d_theta);

/* A whole batch as one CUDA graph (the persistent scheduler's launches
 * captured once and replayed): stn_capture_batch records, on the context's
 * stream (it must not be the legacy default stream), the batch start and one
 * launch per layer step for `shots` shots with the angles d_theta[K] (device,
 * read at replay, so the caller may change their values between replays);
 * stn_launch_captured replays it for the global shots shot_offset..
 * shot_offset + shots - 1, equivalent to stn_begin_batch followed by every
 * layer step.  Asynchronous; results are read with stn_read_records as
 * usual.  The shot offset is copied from the context (host) to the device
 * before each replay.  Errors: STN_EINVAL (no capture yet, bad shots, the
 * default stream), STN_ECUDA. */
stn_status stn_capture_batch(stn_ctx *ctx, int64_t shots, const double *d_theta);
stn_status stn_launch_captured(stn_ctx *ctx, uint64_t shot_offset);

/* Wait for the stream and report any device-side failure of the batch. */
stn_status stn_sync(stn_ctx *ctx);

/* Copy results of the current batch to the host (synchronises).
 * h_records: [shots][ceil(n_meas/8)] bytes, bit i of record j at byte i/8,
 * bit i%8; h_born: [shots][n_meas] realised Born probabilities (or NULL);
 * h_stats: [shots] (or NULL). */
stn_status stn_read_records(stn_ctx *ctx, uint8_t *h_records, double *h_born,
                            stn_shot_stats *h_stats);

/* Device pointer to the packed records of the current batch
 * ([shots][ceil(n_meas/8)] bytes, owned by the context). */
const uint8_t *stn_device_records(const stn_ctx *ctx);

/* Number of detectors of the program (Z-memory: the Z faces in round 0, every
 * face from round 1 on, every Z face again at the final data readout). */
int32_t stn_num_detectors(const stn_ctx *ctx);

/* Detector bits and logical Z_L parity of the current batch, computed on the
 * device from the packed records (Sec. II: a detector is the XOR of a face's
 * outcome with its previous round's; the final data readout closes each Z
 * face; Z_L is the parity of the top row of data qubits), then copied to
 * caller-owned host memory (synchronises).  h_det: [shots][ceil(n_det/8)]
 * bytes, detector i of a shot in byte i/8, bit i%8; h_logical: [shots] bytes
 * (0/1).  Either may be NULL.  Errors: STN_EINVAL without a batch. */
stn_status stn_read_detectors(stn_ctx *ctx, uint8_t *h_det, uint8_t *h_logical);

/* Host-only: the detector table of `cfg`.  h_counts[2] = {n_det, n_logical};
 * h_det (or NULL): [n_det][6] record indices whose XOR is the detector, -1
 * padded; h_logical (or NULL): [n_logical] record indices of Z_L. */
stn_status stn_compile_detectors(const stn_config *cfg, int32_t *h_counts, int32_t *h_det,
                                 int32_t *h_logical);

/* Algorithmic FLOPs of all MPS work since creation, summed over shot slots
 * (synchronises): textbook counts of the GEMMs, Householder R factors and
 * SVDs the sweeps perform (Sec. IV B), independent of the kernels' actual
 * instruction mix.  Used to place measured throughput on a roofline. */
stn_status stn_algorithmic_flops(stn_ctx *ctx, double *h_total);

/* Phase counters of all round launches since creation, summed over shot
 * slots (synchronises).  h_out[15]: SM clock cycles spent by the CTAs in
 * [0] the left (R-factor) sweep, [1] the right sweep's SVDs, [2] the rest of
 * the right sweep (contractions, sorting, new sites), [3] expectation values,
 * [4] the whole op loop (so [4] - [0..3] - [7] is the tableau and
 * bookkeeping); counts of [5] shared-memory SVDs and [6] large-bond SVDs
 * (Householder R factor plus Jacobi on R^dag); [7] cycles of the gauge steps
 * that move the orthogonality centre into an operator's support and [8] the
 * number of sites they crossed; [9] the cycles of the shared-memory SVDs
 * (a part of [1]); [10] the Jacobi sweeps of the large-bond SVDs and [11]
 * the cycles of their Householder R factors (a part of [1]); [12] and [13]
 * the summed rows and columns of the matrices those Jacobi runs rotate, and
 * [14] the cycles of the runs on at most 256 rows (a part of [1]).
 * Diagnostics only: they explain
 * where a round's time goes, they are not part of the path. */
stn_status stn_profile_counters(stn_ctx *ctx, double *h_out);

/* Inverse tableau of one shot of the current batch (synchronises): rows
 * X_0..X_{n-1}, Z_0..Z_{n-1}; row r is i^phase[r] X^x Z^z with x bits in
 * h_x[r*W .. r*W+W-1] (W = ceil(n/64) words, qubit q at bit q%64 of word
 * q/64), likewise h_z.  h_phase[r] in 0..3. */
stn_status stn_read_tableau(stn_ctx *ctx, int64_t shot, uint64_t *h_x, uint64_t *h_z,
                            uint8_t *h_phase);

/* Bond dimensions chi_0..chi_{n-2} of one shot's MPS (synchronises). */
stn_status stn_read_bonds(stn_ctx *ctx, int64_t shot, int32_t *h_bonds);

/* Site tensor k of one shot's MPS (synchronises): chi_k x 2 x chi_{k+1}
 * complex elements of the path's precision, row-major, copied to h_site
 * (caller-owned, sized from stn_read_bonds; chi_0 = chi_n = 1).  With the
 * tableau this gives the full state |psi> = C |MPS> (Eq. 7) of small cases.
 * Errors: STN_EINVAL for a bad shot or site. */
stn_status stn_read_site(stn_ctx *ctx, int64_t shot, int32_t k, void *h_site);

/* Expectation of the memory's logical operator on every shot of the current
 * batch (synchronises): Z_L (Z on the top data row) for a Z-memory, X_L (X
 * on the left data column) for an X-memory, evaluated on the present state
 * C|MPS> (Eq. 7) by pushing it through the frame and contracting the MPS over
 * its support.  Called after the syndrome rounds and before the final
 * readout, it gives the logical angle behind the P_L estimator of Sec. II,
 * Eq. 1: with the decoder's correction c, sin^2(theta/2) = (1 - (-1)^c <L>)/2.
 * h_out[shots] (host, caller-owned); NaN for a shot stopped by an error.
 * Moves each shot's orthogonality centre by exact gauge steps only.
 * Errors: STN_EINVAL without a batch. */
stn_status stn_logical_expectation(stn_ctx *ctx, double *h_out);

/* Squared Schmidt coefficients of one shot's MPS across the cut between sites
 * `cut` and `cut` + 1 (Sec. IV B, Fig. 2 shows them at the centre cut),
 * largest first, into h_sig2 (host, caller-owned, room for chi_cap values);
 * *h_count receives their number.  The shot's orthogonality centre is moved
 * to site `cut` by exact gauge steps (synchronises).  Errors: STN_EINVAL for a
 * bad shot or cut. */
stn_status stn_schmidt_values(stn_ctx *ctx, int64_t shot, int32_t cut, double *h_sig2, int32_t *h_count);

/* Whole job: begin_batch, every segment with h_theta, read_records. */
stn_status stn_sample_shots(stn_ctx *ctx, int64_t shots, uint64_t shot_offset,
                            const double *h_theta, uint8_t *h_records, double *h_born,
                            stn_shot_stats *h_stats);

/* Log-likelihood of fixed measurement records and its gradient with respect
 * to the K per-pair crosstalk angles (the rotation of Eq. 4 in the stabilizer
 * tensor network of Eq. 7), by the adjoint method.  Record r (h_records
 * [n_rec][ceil(n_meas/8)], packed as in stn_read_records) belongs to global
 * shot shot_offset + r, whose Pauli-noise and record-flip events stay the
 * shot's own Philox draws: P(record) is the probability of the record with
 * that noise realisation held fixed, so each measurement's outcome is forced
 * to the record bit XOR its flip event.  Forward pass: the forced shot on
 * the GPU, keeping the state after every rotation and each op's conjugated
 * Pauli; h_logp[r] = sum of the log Born probabilities of the forced
 * outcomes (-inf with STN_ENUMERIC for a record of probability zero).
 * Backward pass: from the final state mu, op by op to the first, rotation j
 * of pair k adds 2 Re <mu|(-i P'_j)|phi_j> / <mu|phi_j> to h_grad[k] and then
 * mu <- exp(+i theta P'_j) mu; a case-A measurement projector is applied
 * again, a case-B measurement applies U |v><0|_j; each application is
 * followed by the same truncating sweep (Sec. IV B), so the result is the
 * gradient of the truncated simulation, exact when nothing is truncated.
 * h_grad[K] is summed over the n_rec records (host, caller-owned).  Uses the
 * context's shot slots (n_rec <= max_shots): the current batch is replaced.
 * Allocates device memory for one state per rotation and record for the
 * duration of the call (STN_ENOMEM when it does not fit).  Errors:
 * STN_EINVAL, STN_ENOMEM, STN_ENUMERIC, STN_ECUDA. */
stn_status stn_logprob_grad(stn_ctx *ctx, uint64_t shot_offset, int64_t n_rec, const uint8_t *h_records,
                            const double *h_theta, double *h_logp, double *h_grad);

/* Philox4x32-10 uniforms u = ((w0<<21) ^ (w1>>11)) * 2^-53 for shots
 * shot_offset.. (n_shots) and events event_offset.. (n_events), written to
 * device memory d_out[n_shots][n_events] on `cuda_stream`.  Stateless. */
stn_status stn_philox_uniforms(uint64_t seed, uint64_t shot_offset, int64_t n_shots,
                               uint32_t event_offset, int32_t n_events, double *d_out,
                               void *cuda_stream);

/* Dense building blocks of the truncation sweep (Sec. IV B, Eq. 8), run alone
 * on one CTA for checking.  precision: STN_PRECISION_*; complex elements are
 * interleaved (re, im) of that precision, all device memory.
 * stn_dense_qr: Householder QR of d_b (m x n, row-major, m <= 1024), in
 *   place; rows 0..min(m,n)-1 then hold R, the rest is zero.
 * stn_dense_svd: one-sided Jacobi SVD of d_c (m x n, column-major, n <= 512):
 *   d_c becomes U diag(sigma), d_v (n x n, column-major) the right singular
 *   vectors, d_sig2[n] (real, of the precision) sigma^2, unsorted.
 *   in_shared = 1 runs it in shared memory (requires m n + n^2 to fit);
 *   in_shared = 2 runs the blocked variant (column-block pairs in shared
 *   memory, C and V in global memory).
 *   in_shared = 3 runs the large-bond path of the truncation sweep instead:
 *   d_c is then ROW-major m x n (m <= 1024) and is overwritten; its
 *   Householder R factor is formed and one-sided Jacobi runs on R^dag, so
 *   column c < min(m,n) of d_v is the right singular vector (the normalised
 *   rotated column of R^dag) for sigma_c^2 = d_sig2[c]; later columns and
 *   entries are zero.
 * Errors: STN_EINVAL on bad sizes, STN_ECUDA on launch failure. */
stn_status stn_dense_qr(int32_t precision, int32_t m, int32_t n, void *d_b, void *cuda_stream);
/* Explicit-Q Householder QR, as the gauge steps that move the orthogonality
 * centre use it (Sec. IV B): d_b (m x n, row-major, m <= 1024) becomes R as
 * for stn_dense_qr, d_q (m x min(m,n), row-major) receives Q with A = Q R,
 * and d_work (m x min(m,n) complex) holds the reflectors.  Errors: STN_EINVAL
 * on bad sizes, STN_ECUDA on launch failure. */
stn_status stn_dense_qr_q(int32_t precision, int32_t m, int32_t n, void *d_b, void *d_q, void *d_work,
                          void *cuda_stream);
stn_status stn_dense_svd(int32_t precision, int32_t m, int32_t n, void *d_c, void *d_v, void *d_sig2,
                         int32_t in_shared, void *cuda_stream);

/* Allocation-free variant of stn_dense_svd with in_shared = 3 (the large-bond
 * SVD of the truncation sweep).  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * the decomposition (a host callback, a framework pool that forbids cudaMalloc
 * while work is queued, an embedded runtime that owns every buffer).  It
 * allocates nothing, neither through the CUDA runtime nor any library: its
 * work copy of the input lives in one static device array of 1 MiB per GPU,
 * held from library load until process exit.
 *   d_c: input, ROW-major m x n complex of the precision (device), left
 *        unchanged.  d_v (n x n, column-major), d_sig2[n]: outputs as for
 *        stn_dense_svd with in_shared = 3.  m <= 1024, n <= 512 (the sizes
 *        of the truncation sweep's bond matrices).
 *   Limit: m n complex elements must fit 1 MiB (m n <= 131072 for
 *   complex64, 65536 for complex128); larger requests return STN_EOVERFLOW
 *   and launch nothing.  Errors: STN_EINVAL for bad sizes or null pointers,
 *   STN_ECUDA for a runtime failure.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture begins.  Every call shares the array and it keeps the last call's
 * contents; calls that overlap on the GPU race on it, so callers must order
 * them (one stream, or events between streams). */
stn_status stn_dense_svd_noalloc(int32_t precision, int32_t m, int32_t n, const void *d_c, void *d_v,
                                 void *d_sig2, void *cuda_stream);

/* Real GEMM on the tcgen05 tensor cores with FP32 accuracy from TF32
 * operands (the 3-term split a = a_hi + a_lo: A_hi B_hi + A_hi B_lo +
 * A_lo B_hi accumulated in FP32 in tensor memory), one CTA, for checking the
 * tensor-core form of the sweep's contractions (Sec. IV A-B: the MPO and
 * truncation contractions are products of such matrices, four real ones per
 * complex one).  d_c (m x n) = d_a (m x k) d_b (k x n), row-major FP32 device
 * memory, each dimension 1..4096.  *d_status (device int, caller-zeroed) is
 * set to STN_ETIMEOUT if a bounded wait for the tensor cores ran out (the
 * kernel then frees its tensor memory and returns).  Asynchronous.
 * Errors: STN_EINVAL on bad sizes or null pointers, STN_ECUDA on launch
 * failure. */
stn_status stn_dense_gemm_tc(int32_t m, int32_t n, int32_t k, const float *d_a, const float *d_b, float *d_c,
                             int32_t *d_status, void *cuda_stream);

/* The complex contraction of the MPS sweeps (R_k A'_k, C = R_k M_k,
 * M_k V_keep, A'_{k-1} W, the transfer products; Sec. IV A-B) alone on one
 * CTA, through the same device routine the round kernel calls:
 *   C = alpha op(A) op(B) + beta C
 * row-major complex of the precision (0: complex128, 1: complex64; device
 * memory), op = identity (0) or conjugate transpose (1), op(A) m x k, op(B)
 * k x n, lda / ldb / ldc the row strides of A, B, C as stored (lda >= k for
 * op_a = 0, >= m for op_a = 1; likewise ldb; ldc >= n); each of m, n, k in
 * 1..4096.  alpha and beta: host (re, im) pairs, rounded to the precision.
 * gemm_units as in stn_config: STN_GEMM_FMA (and complex128) on the CUDA
 * cores, STN_GEMM_TENSOR runs complex64 products of at least 64 x 32 x 16 on
 * the tcgen05 tensor cores (TF32 3-term split, FP32 accumulation).
 * *d_status (device int, caller-zeroed) becomes STN_ETIMEOUT if a bounded
 * wait for the tensor cores ran out.  Asynchronous on cuda_stream.
 * Errors: STN_EINVAL on bad sizes, strides, ops or null pointers, STN_ECUDA
 * on launch failure. */
stn_status stn_dense_cgemm(int32_t precision, int32_t gemm_units, int32_t op_a, int32_t op_b, int32_t m,
                           int32_t n, int32_t k, const double *alpha, const void *d_a, int32_t lda,
                           const void *d_b, int32_t ldb, const double *beta, void *d_c, int32_t ldc,
                           int32_t *d_status, void *cuda_stream);

/* Arithmetic-peak probe (the paper has no counterpart: it measures the
 * denominators of the roofline the kernels are placed on).  Launches on
 * `cuda_stream`, on every SM at full occupancy, a kernel of independent
 * kind 0: FP32 FMA chains, kind 1: FP64 FMA chains, kind 2: TF32 tensor-core
 * products (mma.sync m16n8k8, FP32 accumulation), `iters` loop trips each,
 * and stores in *h_flops the floating-point operations it performs (an FMA
 * counts 2).  Asynchronous: the caller times the launch (CUDA events on the
 * same stream) and divides.  Allocates nothing.  Errors: STN_EINVAL for a bad
 * kind, iters < 1 or a null h_flops; STN_ECUDA for a launch failure. */
stn_status stn_peak_probe(int32_t kind, int64_t iters, double *h_flops, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* STN_H */
