"""Pins of the oracle's diagnostics (Sec. IV B Fig. 2: Schmidt values at a
cut; Sec. II Eq. 1: the logical expectation behind the P_L estimator) against
dense linear algebra on the same states."""

import numpy as np
import pytest

from oracle.circuit import build_layout
from oracle.diagnostics import eq1_term, logical_expectation, schmidt_values
from oracle.shot import ShotSim, make_program
from statevector import run_dense
from workloads import D3_EXACT, theta_table


def readout_start(prog):
    """Index of the first op of the final data readout."""
    last = max(i for i, op in enumerate(prog.ops) if op[0] == "M" and op[5])
    return last + 1


def run_to(w, shot, stop):
    prog = make_program(w)
    theta = theta_table(w.with_(theta_sigma=0.02), len(prog.pairs))
    sim = ShotSim(w, shot, theta, prog)
    for op in prog.ops[:stop]:
        sim.step(op)
    return prog, theta, sim


@pytest.mark.parametrize("cut", [0, 5, 8, 12, 15])
def test_schmidt_values_match_dense_svd(cut):
    w = D3_EXACT.with_(rounds=1, theta=0.12, chi_cap=256, svd_cutoff=1e-14, degeneracy_tol=0.0, p=0.02)
    prog, _, sim = run_to(w, 2, readout_start(make_program(w)))
    got = schmidt_values(sim.mps, cut)
    amp = sim.mps.amplitudes()
    n = sim.n
    ref = np.linalg.svd(amp.reshape(2 ** (cut + 1), 2 ** (n - cut - 1)), compute_uv=False) ** 2
    k = len(got)
    assert abs(got.sum() - 1.0) < 1e-12
    assert np.abs(got - ref[:k]).max() < 1e-12 and ref[k:].sum() < 1e-20
    assert np.all(np.diff(got) <= 0)


@pytest.mark.parametrize("basis", ["Z", "X"])
def test_logical_expectation_matches_dense_state(basis):
    """<L> on C|MPS> before the final readout equals <psi|L|psi> of the dense
    statevector run with the same uniforms (L = Z on the top row for a Z
    memory, X on the left column for an X memory)."""
    w = D3_EXACT.with_(rounds=2, theta=0.15, chi_cap=256, svd_cutoff=1e-14, degeneracy_tol=0.0,
                       memory_basis=basis)
    prog = make_program(w)
    stop = readout_start(prog)
    lay = build_layout(3)
    qubits = [q for q in lay.data if (lay.coords[q][1] == 1 if basis == "Z" else lay.coords[q][0] == 1)]
    for shot in range(3):
        _, theta, sim = run_to(w, shot, stop)
        got = logical_expectation(sim.T, sim.mps, qubits, basis)
        _, _, st = run_dense(w, prog, theta, shot, max_ops=stop, return_state=True)
        psi = st.psi
        lpsi = psi.copy()
        for q in qubits:
            v = lpsi.reshape((2,) * st.n)
            if basis == "Z":
                sgn = 1 - 2 * st.bits(q)
                lpsi = lpsi * sgn
            else:
                lpsi = np.flip(v, axis=q).reshape(-1)
        ref = float(np.real(np.vdot(psi, lpsi)))
        assert abs(got - ref) < 1e-12
        assert abs(got) <= 1.0 + 1e-12


def test_eq1_term_limits():
    assert eq1_term(1.0, 0) == 0.0 and eq1_term(-1.0, 1) == 0.0
    assert abs(eq1_term(-1.0, 0) - 1.0) < 1e-15
    assert abs(eq1_term(np.cos(0.3), 0) - abs(np.sin(0.15))) < 1e-15
