"""GB300 (sm_103a) stabilizer-tensor-network simulator of noisy surface-code
syndrome extraction under coherent crosstalk.

Python binding of the C ABI in include/stn.h.  The binding marshals arguments
only; tableau updates, Pauli conjugation, MPS apply/compress, Born sampling and
Philox draws all run in the library's CUDA kernels.  There is no CPU fallback:
without the built library every call raises.
"""

import ctypes

import numpy as np

from ._native import Config, ShotStats, build, load

STN_OK, STN_EINVAL, STN_ENOMEM, STN_ECUDA, STN_ETIMEOUT, STN_ENUMERIC, STN_ENOTIMPL, STN_EOVERFLOW = range(8)
GEMM_FMA, GEMM_TENSOR = 0, 1  # stn_config.gemm_units
PAIR_RULES = {"adjacent_idle": 0, "adjacent_idle+diag_xx": 1}
OP_KINDS = {1: "RN", 2: "H", 3: "D1", 4: "CX", 5: "D2", 6: "ROT", 7: "M"}


class StnError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"stn status {status}: {message}")
        self.status = status


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def config_from_workload(w):
    """stn_config of a workload.  The arrays of an explicit CNOT schedule or
    explicit pairs stay referenced by the returned object (stn_create copies
    them)."""
    cfg = Config(
        distance=w.distance, rounds=w.rounds, pair_rule=PAIR_RULES[w.pair_rule], chi_cap=w.chi_cap,
        p=w.p, p1_scale=w.p1_scale, p2_scale=w.p2_scale, pR_scale=w.pR_scale, pM_scale=w.pM_scale,
        svd_cutoff=w.svd_cutoff, degeneracy_tol=w.degeneracy_tol, precision=w.precision,
        seed=w.seed, memory_basis={"Z": 0, "X": 1}[getattr(w, "memory_basis", "Z")])
    keep = []
    schedule = getattr(w, "cnot_schedule", None)
    if schedule is not None:
        sch = np.ascontiguousarray([[(-1 if q is None else q) for q in row] for row in schedule], dtype=np.int32)
        keep.append(sch)
        cfg.cnot_schedule = sch.ctypes.data
    pairs = getattr(w, "pairs", None)
    if pairs is not None:
        ab = np.ascontiguousarray([[a, b] for a, b, _, _ in pairs], dtype=np.int32).reshape(-1, 2)
        pauli = np.ascontiguousarray([{"ZZ": 0, "XX": 1}[pp] for _, _, pp, _ in pairs], dtype=np.uint8)
        keep += [ab, pauli]
        cfg.n_pairs = len(pairs)
        cfg.pairs = ab.ctypes.data
        cfg.pair_pauli = pauli.ctypes.data
        if any(m is not None for _, _, _, m in pairs):  # None: the idle rule (STN_LAYERS_IDLE)
            mask = np.ascontiguousarray([0xFF if m is None else int(m) & 0xF for _, _, _, m in pairs],
                                        dtype=np.uint8)
            keep.append(mask)
            cfg.pair_layer_mask = mask.ctypes.data
    cfg._keep = keep
    return cfg


def layout(distance):
    """Host-only layout (stn_layout): (xy[n, 2] coordinates, kinds 'D'/'X'/'Z')."""
    lib = load()
    n = lib.stn_layout(int(distance), None, None)
    if n < 0:
        raise StnError(STN_EINVAL, "bad distance")
    xy = np.zeros((n, 2), dtype=np.int32)
    kind = ctypes.create_string_buffer(n)
    lib.stn_layout(int(distance), _ptr(xy), kind)
    return xy, [chr(c) for c in kind.raw[:n]]


class Simulator:
    """One stn_ctx: a compiled program plus device state for max_shots shots.
    arena_cap_bytes > 0 caps each resident shot's stack of span tensors;
    gemm_units picks the complex64 contraction units (GEMM_FMA, the default:
    CUDA cores; GEMM_TENSOR: tcgen05 tensor cores; see stn_config)."""

    def __init__(self, workload, max_shots, stream=0, arena_cap_bytes=0, gemm_units=GEMM_FMA):
        self.lib = load()
        self.cfg = config_from_workload(workload)
        self.cfg.arena_cap_bytes = int(arena_cap_bytes)
        self.cfg.gemm_units = int(gemm_units)
        ctx = ctypes.c_void_p()
        st = self.lib.stn_create(ctypes.byref(self.cfg), int(max_shots), ctypes.c_void_p(stream),
                                 ctypes.byref(ctx))
        if st != STN_OK:
            raise StnError(st, "stn_create failed")
        self.ctx = ctx
        self.max_shots = int(max_shots)
        self.n_qubits = self.lib.stn_num_qubits(ctx)
        self.n_pairs = self.lib.stn_num_pairs(ctx)
        self.n_meas = self.lib.stn_num_meas(ctx)
        self.n_events = self.lib.stn_num_events(ctx)
        self.n_ops = self.lib.stn_num_ops(ctx)
        self.n_det = self.lib.stn_num_detectors(ctx)
        self.rounds = workload.rounds
        self.rec_bytes = (self.n_meas + 7) // 8
        self.words = (self.n_qubits + 63) // 64
        self.shots = 0

    def _check(self, st):
        if st != STN_OK:
            msg = self.lib.stn_last_error(self.ctx)
            raise StnError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.stn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def program(self):
        ops = np.zeros((self.n_ops, 6), dtype=np.int32)
        pairs = np.zeros((max(self.n_pairs, 1), 4), dtype=np.int32)
        self._check(self.lib.stn_get_program(self.ctx, _ptr(ops), _ptr(pairs)))
        return ops, pairs[: self.n_pairs]

    def begin_batch(self, shots, shot_offset=0):
        self._check(self.lib.stn_begin_batch(self.ctx, int(shots), int(shot_offset)))
        self.shots = int(shots)

    def apply_round(self, r, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        assert theta.shape == (self.n_pairs,)
        self._check(self.lib.stn_apply_round(self.ctx, int(r), _ptr(theta)))

    def apply_round_device(self, r, d_theta_ptr):
        self._check(self.lib.stn_apply_round_device(self.ctx, int(r), ctypes.c_void_p(d_theta_ptr)))

    @property
    def n_steps(self):
        """Layer steps of the program (4 per round, see stn_apply_step_device)."""
        return self.lib.stn_num_steps(self.ctx)

    def apply_step_device(self, step, d_theta_ptr):
        self._check(self.lib.stn_apply_step_device(self.ctx, int(step), ctypes.c_void_p(d_theta_ptr)))

    def capture_batch(self, shots, d_theta_ptr):
        """Capture a whole batch (batch start and every layer step) as one
        CUDA graph (stn_capture_batch); the simulator needs its own stream."""
        self._check(self.lib.stn_capture_batch(self.ctx, int(shots), ctypes.c_void_p(d_theta_ptr)))
        self._graph_shots = int(shots)

    def launch_captured(self, shot_offset):
        """Replay the captured batch for global shots shot_offset.. ."""
        self._check(self.lib.stn_launch_captured(self.ctx, int(shot_offset)))
        self.shots = self._graph_shots

    def sync(self):
        self._check(self.lib.stn_sync(self.ctx))

    def read_records(self, born=True, stats=True):
        rec = np.zeros((self.shots, self.rec_bytes), dtype=np.uint8)
        b = np.zeros((self.shots, self.n_meas), dtype=np.float64) if born else None
        s = (ShotStats * self.shots)() if stats else None
        self._check(self.lib.stn_read_records(self.ctx, _ptr(rec), _ptr(b),
                                              ctypes.cast(s, ctypes.c_void_p) if stats else None))
        out = {"records": rec, "bits": unpack_records(rec, self.n_meas)}
        if born:
            out["born"] = b
        if stats:
            out["max_chi"] = np.array([x.max_chi for x in s])
            out["near_draws"] = np.array([x.near_draws for x in s])
            out["discarded"] = np.array([x.discarded for x in s])
            out["logp"] = np.array([x.logp for x in s])
        return out

    def read_detectors(self):
        """Detector bits [shots][n_det] and Z_L parities [shots] of the batch,
        computed on the device from its records."""
        det = np.zeros((self.shots, (self.n_det + 7) // 8), dtype=np.uint8)
        obs = np.zeros(self.shots, dtype=np.uint8)
        self._check(self.lib.stn_read_detectors(self.ctx, _ptr(det), _ptr(obs)))
        return unpack_records(det, self.n_det), obs

    def algorithmic_flops(self):
        v = ctypes.c_double()
        self._check(self.lib.stn_algorithmic_flops(self.ctx, ctypes.byref(v)))
        return v.value

    PROFILE_KEYS = ("left_sweep_cycles", "svd_cycles", "right_sweep_rest_cycles", "expectation_cycles",
                    "op_loop_cycles", "svd_count_shared", "svd_count_large", "gauge_cycles",
                    "gauge_sites", "svd_small_cycles", "jacobi_sweeps_large", "svd_qr_cycles",
                    "jacobi_rows_large", "jacobi_cols_large", "jacobi_rows256_cycles")

    def profile_counters(self):
        """Per-phase SM cycles and SVD counts summed over shot slots since
        creation (see stn_profile_counters)."""
        buf = (ctypes.c_double * len(self.PROFILE_KEYS))()  # the library writes one value per key
        self._check(self.lib.stn_profile_counters(self.ctx, ctypes.cast(buf, ctypes.c_void_p)))
        return dict(zip(self.PROFILE_KEYS, list(buf)))

    def logical_expectation(self):
        """<L> of the memory's logical operator on every shot of the batch
        (stn_logical_expectation); call after the syndrome rounds."""
        out = np.zeros(self.shots, dtype=np.float64)
        self._check(self.lib.stn_logical_expectation(self.ctx, _ptr(out)))
        return out

    def schmidt_values(self, shot, cut):
        """Squared Schmidt coefficients across the cut after site `cut`
        (stn_schmidt_values), largest first."""
        out = np.zeros(max(512, self.cfg.chi_cap), dtype=np.float64)
        cnt = ctypes.c_int32()
        self._check(self.lib.stn_schmidt_values(self.ctx, int(shot), int(cut), _ptr(out), ctypes.byref(cnt)))
        return out[: cnt.value]

    def read_records_into(self, h_records_ptr):
        """Packed records of the batch into caller-owned host memory
        ([shots][rec_bytes] bytes, e.g. pinned)."""
        self._check(self.lib.stn_read_records(self.ctx, ctypes.c_void_p(h_records_ptr), None, None))

    def device_records_ptr(self):
        return self.lib.stn_device_records(self.ctx)

    def read_tableau(self, shot):
        rows = 2 * self.n_qubits
        x = np.zeros((rows, self.words), dtype=np.uint64)
        z = np.zeros((rows, self.words), dtype=np.uint64)
        m = np.zeros(rows, dtype=np.uint8)
        self._check(self.lib.stn_read_tableau(self.ctx, int(shot), _ptr(x), _ptr(z), _ptr(m)))
        return x, z, m

    def read_bonds(self, shot):
        b = np.zeros(self.n_qubits - 1, dtype=np.int32)
        self._check(self.lib.stn_read_bonds(self.ctx, int(shot), _ptr(b)))
        return b

    def read_mps(self, shot):
        """Site tensors of one shot's MPS as complex numpy arrays (chi_k, 2, chi_k+1)."""
        bonds = [1] + list(self.read_bonds(shot)) + [1]
        dt = np.complex128 if self.cfg.precision == 0 else np.complex64
        sites = []
        for k in range(self.n_qubits):
            a = np.zeros((bonds[k], 2, bonds[k + 1]), dtype=dt)
            self._check(self.lib.stn_read_site(self.ctx, int(shot), int(k), _ptr(a)))
            sites.append(a)
        return sites

    def sample_shots(self, shots, shot_offset, theta, born=True, stats=True):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        self.begin_batch(shots, shot_offset)
        for r in range(self.rounds + 1):
            self.apply_round(r, theta)
        return self.read_records(born=born, stats=stats)

    def logprob_grad(self, records, theta, shot_offset=0):
        """(log P[r], d sum_r log P[r] / d theta[K]) of packed records
        [n_rec][rec_bytes] of global shots shot_offset.. (stn_logprob_grad)."""
        rec = np.ascontiguousarray(records, dtype=np.uint8)
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        logp = np.zeros(len(rec), dtype=np.float64)
        grad = np.zeros(self.n_pairs, dtype=np.float64)
        self._check(self.lib.stn_logprob_grad(self.ctx, int(shot_offset), len(rec), _ptr(rec), _ptr(theta),
                                              _ptr(logp), _ptr(grad)))
        self.shots = len(rec)
        return logp, grad


def compile_program(workload):
    """Host-only compile of the op program (no GPU): (counts, ops[N,6], pairs[K,4])."""
    lib = load()
    cfg = config_from_workload(workload)
    counts = np.zeros(5, dtype=np.int32)
    st = lib.stn_compile_program(ctypes.byref(cfg), _ptr(counts), None, None)
    if st != STN_OK:
        raise StnError(st, "stn_compile_program failed")
    ops = np.zeros((counts[4], 6), dtype=np.int32)
    pairs = np.zeros((max(counts[1], 1), 4), dtype=np.int32)
    st = lib.stn_compile_program(ctypes.byref(cfg), _ptr(counts), _ptr(ops), _ptr(pairs))
    if st != STN_OK:
        raise StnError(st, "stn_compile_program failed")
    return counts, ops, pairs[: counts[1]]


def compile_detectors(workload):
    """Host-only detector table (no GPU): (det[n_det, 6] record indices, -1
    padded, whose XOR is each detector; logical[n] record indices of Z_L)."""
    lib = load()
    cfg = config_from_workload(workload)
    counts = np.zeros(2, dtype=np.int32)
    st = lib.stn_compile_detectors(ctypes.byref(cfg), _ptr(counts), None, None)
    if st != STN_OK:
        raise StnError(st, "stn_compile_detectors failed")
    det = np.zeros((counts[0], 6), dtype=np.int32)
    logical = np.zeros(counts[1], dtype=np.int32)
    st = lib.stn_compile_detectors(ctypes.byref(cfg), _ptr(counts), _ptr(det), _ptr(logical))
    if st != STN_OK:
        raise StnError(st, "stn_compile_detectors failed")
    return det, logical


def unpack_records(rec, n_meas):
    bits = np.unpackbits(rec, axis=1, bitorder="little")
    return bits[:, :n_meas].astype(np.uint8)


def philox_uniforms(seed, shot_offset, n_shots, event_offset, n_events, d_out_ptr, stream=0):
    st = load().stn_philox_uniforms(int(seed), int(shot_offset), int(n_shots), int(event_offset),
                                    int(n_events), ctypes.c_void_p(d_out_ptr), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_philox_uniforms failed")


def dense_gemm_tc(m, n, k, d_a, d_b, d_c, d_status, stream=0):
    """stn_dense_gemm_tc: d_c = d_a @ d_b (row-major FP32) on the tcgen05
    tensor cores with the 3-term TF32 split."""
    st = load().stn_dense_gemm_tc(int(m), int(n), int(k), ctypes.c_void_p(d_a), ctypes.c_void_p(d_b),
                                  ctypes.c_void_p(d_c), ctypes.c_void_p(d_status), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_dense_gemm_tc failed")


def dense_cgemm(precision, op_a, op_b, m, n, k, d_a, lda, d_b, ldb, d_c, ldc, d_status, alpha=1.0, beta=0.0,
                gemm_units=GEMM_FMA, stream=0):
    """stn_dense_cgemm: d_c = alpha op(A) op(B) + beta d_c (row-major complex
    device buffers, op 0 = identity, 1 = conjugate transpose) on one CTA
    through the sweeps' contraction routine."""
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
    st = load().stn_dense_cgemm(int(precision), int(gemm_units), int(op_a), int(op_b), int(m), int(n), int(k),
                                al, ctypes.c_void_p(d_a), int(lda), ctypes.c_void_p(d_b), int(ldb), be,
                                ctypes.c_void_p(d_c), int(ldc), ctypes.c_void_p(d_status), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_dense_cgemm failed")


def peak_probe(kind, iters, stream=0):
    """Launch the arithmetic-peak probe (kind 0 FP32 FMA, 1 FP64 FMA, 2 TF32
    mma.sync) on `stream`; returns the FLOPs it performs.  The caller times
    the launch."""
    flops = ctypes.c_double()
    st = load().stn_peak_probe(int(kind), int(iters), ctypes.byref(flops), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_peak_probe failed")
    return flops.value


def dense_qr_q(precision, m, n, d_b, d_q, d_work, stream=0):
    st = load().stn_dense_qr_q(int(precision), int(m), int(n), ctypes.c_void_p(d_b), ctypes.c_void_p(d_q),
                               ctypes.c_void_p(d_work), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_dense_qr_q failed")


def dense_qr(precision, m, n, d_b, stream=0):
    st = load().stn_dense_qr(int(precision), int(m), int(n), ctypes.c_void_p(d_b), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_dense_qr failed")


def dense_svd(precision, m, n, d_c, d_v, d_sig2, in_shared, stream=0):
    st = load().stn_dense_svd(int(precision), int(m), int(n), ctypes.c_void_p(d_c), ctypes.c_void_p(d_v),
                              ctypes.c_void_p(d_sig2), int(in_shared), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_dense_svd failed")


def dense_svd_noalloc(precision, m, n, d_c, d_v, d_sig2, stream=0):
    """stn_dense_svd_noalloc: the large-bond SVD with no device allocation
    (its work copy lives in the library's static 1 MiB array); d_c is kept."""
    st = load().stn_dense_svd_noalloc(int(precision), int(m), int(n), ctypes.c_void_p(d_c),
                                      ctypes.c_void_p(d_v), ctypes.c_void_p(d_sig2), ctypes.c_void_p(stream))
    if st != STN_OK:
        raise StnError(st, "stn_dense_svd_noalloc failed")


__all__ = ["Simulator", "StnError", "build", "load", "philox_uniforms", "unpack_records",
           "config_from_workload", "compile_program", "compile_detectors", "dense_qr", "dense_svd",
           "dense_svd_noalloc", "peak_probe", "layout", "dense_gemm_tc"]
