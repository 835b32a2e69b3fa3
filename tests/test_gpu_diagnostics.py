"""Device diagnostics through the C ABI against the oracle: the squared
Schmidt coefficients at a cut (Sec. IV B, Fig. 2) and the logical operator's
expectation before the final readout (Sec. II, Eq. 1)."""

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from oracle.circuit import build_layout
from oracle.diagnostics import logical_expectation, schmidt_values
from oracle.shot import ShotSim, make_program
from workloads import D3_EXACT, D5_BENCH, PRECISION_C64, theta_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stn.build()


def oracle_after_rounds(w, shot, theta, rounds_done):
    prog = make_program(w)
    stop = max(i for i, op in enumerate(prog.ops) if op[0] == "M" and op[5] and prog.meas_round[op[4]] < rounds_done)
    sim = ShotSim(w, shot, theta, prog)
    for op in prog.ops[: stop + 1]:
        sim.step(op)
    return sim


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-5)])
def test_schmidt_values_match_oracle(precision, tol):
    w = D3_EXACT.with_(rounds=2, theta=0.12, precision=precision,
                       svd_cutoff=1e-12 if precision == 0 else D5_BENCH.svd_cutoff,
                       degeneracy_tol=1e-12 if precision == 0 else D5_BENCH.degeneracy_tol)
    shots = 3
    sim = stn.Simulator(w, max_shots=shots)
    theta = theta_table(w, sim.n_pairs)
    sim.begin_batch(shots, 0)
    for r in range(w.rounds):
        sim.apply_round(r, theta)
    for s in range(shots):
        ref = oracle_after_rounds(w, s, theta, w.rounds)
        for cut in (3, 8, 12):
            got = sim.schmidt_values(s, cut)
            want = schmidt_values(ref.mps, cut)
            k = min(len(got), len(want))
            assert np.abs(got[:k] - want[:k]).max() < tol, (s, cut)
            assert abs(got.sum() - 1.0) < 10 * tol
    out = sim.read_records()  # the gauge moves left the batch's state and records intact
    for s in range(shots):
        assert np.all(np.isfinite(out["born"][s]))


@pytest.mark.parametrize("basis", ["Z", "X"])
def test_logical_expectation_matches_oracle(basis):
    w = D3_EXACT.with_(rounds=2, theta=0.15, p=0.01, memory_basis=basis)
    shots = 4
    sim = stn.Simulator(w, max_shots=shots)
    theta = theta_table(w, sim.n_pairs)
    sim.begin_batch(shots, 0)
    for r in range(w.rounds):
        sim.apply_round(r, theta)
    got = sim.logical_expectation()
    lay = build_layout(3)
    qubits = [q for q in lay.data if (lay.coords[q][1] == 1 if basis == "Z" else lay.coords[q][0] == 1)]
    for s in range(shots):
        ref = oracle_after_rounds(w, s, theta, w.rounds)
        want = logical_expectation(ref.T, ref.mps, qubits, basis)
        assert abs(got[s] - want) < 1e-11, (s, got[s], want)
    # the readout segment still runs on the state the diagnostics left
    sim.apply_round(w.rounds, theta)
    out = sim.read_records()
    from oracle.shot import run_shot
    for s in range(shots):
        assert list(out["bits"][s]) == run_shot(w, s, theta).record
