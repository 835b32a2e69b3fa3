"""CPU checks of the native library: it loads, exports every entry point that
include/stn.h declares, and its host-side circuit compiler emits exactly the
program the oracle builds (no GPU needed)."""

import os
import re

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from oracle.shot import make_program
from workloads import D3_EXACT, D5_BENCH

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    stn.build()
    return stn.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "stn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stn_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


KIND = {"RN": 1, "H": 2, "D1": 3, "CX": 4, "D2": 5, "ROT": 6, "M": 7}


def oracle_rows(prog):
    rows = []
    for op in prog.ops:
        k = op[0]
        if k in ("RN", "D1"):
            rows.append([KIND[k], op[1], 0, 0, op[2], 0])
        elif k == "H":
            rows.append([2, op[1], 0, 0, 0, 0])
        elif k == "CX":
            rows.append([4, op[1], op[2], 0, 0, 0])
        elif k == "D2":
            rows.append([5, op[1], op[2], 0, op[3], 0])
        elif k == "ROT":
            p = prog.pairs[op[1]]
            rows.append([6, p.a, p.b, 0 if p.pauli == "ZZ" else 1, 0, op[1]])
        elif k == "M":
            q, evb, evf, rec, reset, evr = op[1:]
            assert evf == evb + 1 and (not reset or evr == evb + 2)
            rows.append([7, q, 0, int(reset), evb, rec])
    return np.array(rows, dtype=np.int32)


@pytest.mark.parametrize("d", [3, 5, 7, 9])
@pytest.mark.parametrize("rule", ["adjacent_idle", "adjacent_idle+diag_xx"])
def test_native_program_matches_oracle(lib, d, rule):
    w = D3_EXACT.with_(distance=d, rounds=d, pair_rule=rule)
    counts, ops, pairs = stn.compile_program(w)
    prog = make_program(w)
    assert counts[0] == prog.layout.n
    assert counts[1] == len(prog.pairs)
    assert counts[2] == prog.n_meas == w.n_meas
    assert counts[3] == prog.n_events
    assert np.array_equal(ops, oracle_rows(prog))
    ref_pairs = np.array([[p.a, p.b, 0 if p.pauli == "ZZ" else 1, p.layer_mask] for p in prog.pairs])
    assert np.array_equal(pairs, ref_pairs)


def test_bench_program_sizes(lib):
    counts, ops, _ = stn.compile_program(D5_BENCH)
    n, K, n_meas, n_events, n_ops = counts
    assert (n, K, n_meas) == (49, 80, 145)
    assert int(np.sum(ops[:, 0] == 6)) == 5 * 3 * 80  # 1200 rotations
    assert int(np.sum(ops[:, 0] == 7)) == 145


@pytest.mark.parametrize("bad", [dict(distance=4), dict(distance=1), dict(rounds=0), dict(chi_cap=0),
                                 dict(chi_cap=1000), dict(p=-1.0), dict(p=0.5, pM_scale=5.0),
                                 dict(svd_cutoff=1.5), dict(precision=7)])
def test_invalid_configs_rejected(lib, bad):
    with pytest.raises(stn.StnError) as e:
        stn.compile_program(D3_EXACT.with_(**bad))
    assert e.value.status == stn.STN_EINVAL


@pytest.mark.parametrize("w", [D3_EXACT, D5_BENCH, D3_EXACT.with_(rounds=1), D5_BENCH.with_(distance=7, rounds=2)])
def test_detector_table_matches_oracle(lib, w):
    """The compiled detector table, applied to arbitrary records, gives the
    oracle's detector bits and Z_L parity (Sec. II)."""
    from oracle.circuit import detectors, logical_z
    det, logical = stn.compile_detectors(w)
    prog = make_program(w)
    rng = np.random.default_rng(w.distance * 10 + w.rounds)
    n_meas = w.n_meas
    for _ in range(8):
        rec = rng.integers(0, 2, size=n_meas)
        ext = np.append(rec, 0)  # index -1 reads the appended zero
        got = np.bitwise_xor.reduce(ext[det], axis=1)
        assert list(got) == detectors(prog, list(rec))
        assert int(np.bitwise_xor.reduce(rec[logical])) == logical_z(prog, list(rec))


def _schedule_and_pairs():
    from test_oracle_shot import transposed_schedule
    from oracle.circuit import build_layout, build_pairs
    lay = build_layout(3)
    rule = build_pairs(lay, "adjacent_idle")
    pairs = tuple((p.a, p.b, p.pauli, None) for p in rule[::3]) + ((lay.data[0], lay.data[1], "XX", None),)
    return transposed_schedule(3), pairs, rule


@pytest.mark.parametrize("variant", ["x_memory", "schedule", "pairs_idle_rule", "pairs_masks", "all"])
def test_problem_statement_fields_compile_like_the_oracle(lib, variant):
    """The boundary's problem statement (memory basis, CNOT schedule, explicit
    pairs with or without layer masks) compiles to the oracle's program, pairs
    and detector table."""
    from oracle.circuit import detectors, logical_z
    schedule, pairs, rule = _schedule_and_pairs()
    w = D3_EXACT.with_(rounds=2, p=0.01)
    if variant in ("x_memory", "all"):
        w = w.with_(memory_basis="X")
    if variant in ("schedule", "all"):
        w = w.with_(cnot_schedule=schedule)
    if variant in ("pairs_idle_rule", "all"):
        w = w.with_(pairs=pairs)
    if variant == "pairs_masks":
        w = w.with_(pairs=tuple((p.a, p.b, "XX" if k % 5 == 0 else "ZZ", (k * 7) % 16)
                                for k, p in enumerate(rule)))
    counts, ops, got_pairs = stn.compile_program(w)
    prog = make_program(w)
    assert counts[3] == prog.n_events and counts[2] == prog.n_meas
    rows = oracle_rows(prog)
    assert np.array_equal(ops, rows)
    ref_pairs = np.array([[p.a, p.b, 0 if p.pauli == "ZZ" else 1, p.layer_mask] for p in prog.pairs])
    assert np.array_equal(got_pairs, ref_pairs)
    det, logical = stn.compile_detectors(w)
    rng = np.random.default_rng(3)
    for _ in range(4):
        rec = rng.integers(0, 2, size=w.n_meas)
        ext = np.append(rec, 0)
        assert list(np.bitwise_xor.reduce(ext[det], axis=1)) == detectors(prog, list(rec))
        assert int(np.bitwise_xor.reduce(rec[logical])) == logical_z(prog, list(rec))


def test_explicit_default_pairs_give_the_default_program(lib):
    _, _, rule = _schedule_and_pairs()
    base = stn.compile_program(D3_EXACT)
    for masks in (True, False):
        w = D3_EXACT.with_(pairs=tuple((p.a, p.b, p.pauli, p.layer_mask if masks else None) for p in rule))
        got = stn.compile_program(w)
        assert all(np.array_equal(x, y) for x, y in zip(got, base))


def test_invalid_schedule_and_pairs_rejected(lib):
    schedule, pairs, _ = _schedule_and_pairs()
    bad_schedule = [list(r) for r in schedule]
    bad_schedule[0] = [bad_schedule[0][0]] * 4
    for w in (D3_EXACT.with_(cnot_schedule=tuple(map(tuple, bad_schedule))),
              D3_EXACT.with_(pairs=((0, 0, "ZZ", None),)),
              D3_EXACT.with_(pairs=((0, 99, "ZZ", None),))):
        with pytest.raises(stn.StnError) as e:
            stn.compile_program(w)
        assert e.value.status == stn.STN_EINVAL


def test_layout_entry_point(lib):
    from oracle.circuit import build_layout
    for d in (3, 5):
        xy, kind = stn.layout(d)
        lay = build_layout(d)
        assert [tuple(v) for v in xy] == lay.coords
        assert [k for k in kind] == ["D" if q in lay.data else lay.kind[q] for q in range(lay.n)]


def test_gemm_units_validated(lib):
    """stn_config.gemm_units accepts STN_GEMM_TENSOR and STN_GEMM_FMA only."""
    import ctypes
    counts = np.zeros(5, dtype=np.int32)
    for units, ok in ((stn.GEMM_TENSOR, True), (stn.GEMM_FMA, True), (2, False), (-1, False)):
        cfg = stn.config_from_workload(D3_EXACT)
        cfg.gemm_units = units
        st = lib.stn_compile_program(ctypes.byref(cfg), counts.ctypes.data_as(ctypes.c_void_p), None, None)
        assert (st == stn.STN_OK) == ok, (units, st)


def test_dense_cgemm_rejects_bad_arguments(lib):
    """stn_dense_cgemm validates sizes, strides, ops and units before any
    launch (no GPU needed)."""
    import ctypes
    one = (ctypes.c_double * 2)(1.0, 0.0)
    p = ctypes.c_void_p(16)  # never dereferenced: every call below is rejected first
    good = dict(precision=1, units=0, op_a=0, op_b=0, m=8, n=8, k=8, lda=8, ldb=8, ldc=8)
    bad = [dict(precision=2), dict(units=3), dict(op_a=2), dict(m=0), dict(k=5000), dict(lda=7),
           dict(op_a=1, m=9, lda=8), dict(ldb=4), dict(ldc=7)]
    for b in bad:
        a = {**good, **b}
        st = lib.stn_dense_cgemm(a["precision"], a["units"], a["op_a"], a["op_b"], a["m"], a["n"], a["k"], one, p,
                                 a["lda"], p, a["ldb"], one, p, a["ldc"], p, None)
        assert st == stn.STN_EINVAL, b
    st = lib.stn_dense_cgemm(1, 0, 0, 0, 8, 8, 8, one, None, 8, p, 8, one, p, 8, p, None)
    assert st == stn.STN_EINVAL
