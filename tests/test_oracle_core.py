"""Pins of the oracle's building blocks against definitions that do not come
from the oracle itself: published Philox known answers, dense matrices, and
brute-force conjugation."""

import itertools
import os

import numpy as np
import pytest

from oracle.mps import MPS, keep_count
from oracle.pauli import (CNOT, CY, CZ, H2, S2, X2, Y2, Z2, Pauli, conjugation_table,
                          conjugate_by_gate, local_xz_matrix)
from oracle.philox import philox4x32_10, uniform
from oracle.tableau import InverseTableau

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert philox4x32_10(r[0:4], r[4:6]) == tuple(r[6:10])


def test_uniform_range_and_independence():
    us = np.array([uniform(0, s, e) for s in range(40) for e in range(50)])
    assert us.min() >= 0.0 and us.max() < 1.0
    # mean and variance of U[0,1) within 5 sigma for 2000 draws
    assert abs(us.mean() - 0.5) < 5 * np.sqrt(1 / 12 / us.size)
    assert abs(us.var() - 1 / 12) < 0.01
    # different seeds, shots and events give different streams
    assert uniform(0, 1, 2) != uniform(1, 1, 2) != uniform(0, 2, 2)
    assert uniform(0, 1 << 33, 2) != uniform(0, 1, 2)


def dense_pauli(p):
    mat = np.ones((1, 1), dtype=complex)
    for k in range(p.n):
        mat = np.kron(mat, p.site_matrix(k))
    return (1j ** p.m) * mat


def random_pauli(rng, n):
    return Pauli(rng.integers(4), rng.integers(0, 2, n).astype(bool), rng.integers(0, 2, n).astype(bool))


def test_pauli_product_and_commutation_match_dense():
    rng = np.random.default_rng(1)
    for _ in range(200):
        n = int(rng.integers(1, 4))
        a, b = random_pauli(rng, n), random_pauli(rng, n)
        assert np.allclose(dense_pauli(a * b), dense_pauli(a) @ dense_pauli(b))
        da, db = dense_pauli(a), dense_pauli(b)
        assert a.commutes(b) == np.allclose(da @ db, db @ da)


def test_hermitian_letters_and_sign():
    rng = np.random.default_rng(2)
    for _ in range(100):
        n = 3
        p = random_pauli(rng, n)
        d = dense_pauli(p)
        assert p.is_hermitian() == np.allclose(d, d.conj().T)
        if p.is_hermitian():
            mats = {"I": np.eye(2), "X": X2, "Y": Y2, "Z": Z2}
            ref = np.ones((1, 1))
            for ch in p.letters():
                ref = np.kron(ref, mats[ch])
            assert np.allclose(d, p.sign() * ref)


@pytest.mark.parametrize("gate", [H2, S2, CNOT, CZ, CY])
def test_conjugation_table_matches_dense(gate):
    k = int(np.log2(gate.shape[0]))
    tab = conjugation_table(gate)
    for bits, (m, bits2) in tab.items():
        lhs = gate.conj().T @ local_xz_matrix(bits) @ gate
        assert np.allclose(lhs, (1j ** m) * local_xz_matrix(bits2))
    assert len(tab) == 4 ** k


def embed(gate, qubits, n):
    """Dense n-qubit operator of a gate on `qubits` (qubit 0 most significant)."""
    k = len(qubits)
    full = np.zeros((2 ** n, 2 ** n), dtype=complex)
    others = [q for q in range(n) if q not in qubits]
    for col in range(2 ** n):
        bits = [(col >> (n - 1 - q)) & 1 for q in range(n)]
        sub = 0
        for q in qubits:
            sub = sub * 2 + bits[q]
        for out_sub in range(2 ** k):
            amp = gate[out_sub, sub]
            if amp == 0:
                continue
            ob = list(bits)
            for i, q in enumerate(qubits):
                ob[q] = (out_sub >> (k - 1 - i)) & 1
            row = 0
            for q in range(n):
                row = row * 2 + ob[q]
            full[row, col] += amp
    return full


def test_inverse_tableau_tracks_dense_clifford():
    """Random Clifford circuits (left gates, Pauli errors, right gates): every
    row must equal C^dag g C computed from the dense unitary."""
    rng = np.random.default_rng(3)
    n = 3
    tables = {"H": conjugation_table(H2), "S": conjugation_table(S2), "CX": conjugation_table(CNOT),
              "CZ": conjugation_table(CZ), "CY": conjugation_table(CY)}
    mats = {"H": H2, "S": S2, "CX": CNOT, "CZ": CZ, "CY": CY}
    for trial in range(20):
        t = InverseTableau(n)
        c = np.eye(2 ** n, dtype=complex)
        for _ in range(25):
            r = rng.integers(4)
            name = ["H", "S", "CX", "CZ", "CY"][rng.integers(5)]
            qs = [int(rng.integers(n))] if name in "HS" else list(rng.choice(n, 2, replace=False))
            qs = [int(q) for q in qs]
            g = embed(mats[name], qs, n)
            if r == 0:
                t.left_gate(tables[name], qs)
                c = g @ c
            elif r == 1:
                letter = "XYZ"[rng.integers(3)]
                q = int(rng.integers(n))
                t.left_pauli(letter, [q])
                c = embed({"X": X2, "Y": Y2, "Z": Z2}[letter], [q], n) @ c
            else:
                t.right_gate(tables[name], qs)
                c = c @ g
        for q in range(n):
            for letter, row in (("X", t.tx[q]), ("Z", t.tz[q])):
                gq = embed({"X": X2, "Z": Z2}[letter], [q], n)
                assert np.allclose(dense_pauli(row), c.conj().T @ gq @ c)
        assert t.is_symplectic()
        # conjugate(): a random physical Pauli
        p = random_pauli(rng, n)
        assert np.allclose(dense_pauli(t.conjugate(p)), c.conj().T @ dense_pauli(p) @ c)


def random_mps(rng, n, chi):
    m = MPS(n)
    dims = [1] + [min(chi, 2 ** min(k, n - k)) for k in range(1, n)] + [1]
    for k in range(n):
        m.A[k] = rng.normal(size=(dims[k], 2, dims[k + 1])) + 1j * rng.normal(size=(dims[k], 2, dims[k + 1]))
    m.center = 0
    # bring to canonical form with the centre at 0 by sweeping from the right
    m.center = n - 1
    m.move_center(0)
    m.A[0] /= np.linalg.norm(m.A[0])
    return m


def test_mps_two_branch_and_compress_exact():
    """Without truncation, MPO apply + QR/SVD compression must equal the dense
    operator applied to the dense vector."""
    rng = np.random.default_rng(4)
    n = 7
    for trial in range(10):
        m = random_mps(rng, n, 8)
        psi = m.amplitudes()
        lo, hi = sorted(rng.choice(n, 2, replace=False).tolist())
        ops0 = {k: rng.normal(size=(2, 2)) + 0j for k in range(lo, hi + 1) if rng.random() < 0.5}
        ops1 = {k: rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)) for k in range(lo, hi + 1)}
        w0, w1 = 0.7, -0.3j
        dense = np.zeros((2 ** n, 2 ** n), dtype=complex)
        for branch, w in ((ops0, w0), (ops1, w1)):
            op = np.ones((1, 1))
            for k in range(n):
                op = np.kron(op, branch.get(k, np.eye(2)))
            dense += w * op
        target = dense @ psi
        target /= np.linalg.norm(target)
        m.move_center_into(lo, hi)
        m.apply_two_branch(lo, hi, ops0, ops1, w0, w1)
        disc, _ = m.compress(lo, hi, chi_cap=1 << 20, cutoff=0.0, delta=0.0)
        got = m.amplitudes()
        assert abs(abs(np.vdot(target, got)) - 1.0) < 1e-12
        assert disc < 1e-20
        # canonical form: centre at lo, left sites left-canonical, right sites right-canonical
        for k in range(lo):
            a = m.A[k].reshape(-1, m.A[k].shape[2])
            assert np.allclose(a.conj().T @ a, np.eye(a.shape[1]))
        for k in range(lo + 1, n):
            a = m.A[k].reshape(m.A[k].shape[0], -1)
            assert np.allclose(a @ a.conj().T, np.eye(a.shape[0]))


def test_truncation_is_optimal_at_one_bond():
    """Eq. 8: keeping the chi largest Schmidt values is the best rank-chi
    approximation; discarded weight equals the sum of dropped squared values
    (Eckart-Young)."""
    rng = np.random.default_rng(5)
    n = 6
    m = random_mps(rng, n, 8)
    psi = m.amplitudes()
    mat = psi.reshape(2 ** 3, 2 ** 3)
    s = np.linalg.svd(mat, compute_uv=False)
    m.move_center(2)
    # identity two-branch operator on [2, 3]: doubles bond 2-3, then truncate to 4
    m.apply_two_branch(2, 3, {}, {}, 0.5, 0.5)
    disc, chi = m.compress(2, 3, chi_cap=4, cutoff=0.0, delta=0.0)
    assert abs(disc - np.sum(s[4:] ** 2) / np.sum(s ** 2)) < 1e-12
    assert m.A[2].shape[2] == 4


def test_keep_count_rules():
    s = np.array([1.0, 0.5, 0.1, 0.1, 0.1, 1e-9, 1e-16])
    assert keep_count(s, 10, 1e-14, 0.0) == 6
    assert keep_count(s, 10, 1e-8, 0.0) == 5
    assert keep_count(s, 2, 0.0, 1e-12) == 2
    # cap inside a degenerate cluster: the whole cluster is dropped
    assert keep_count(s, 3, 0.0, 1e-12) == 2
    assert keep_count(s, 4, 0.0, 1e-12) == 2
    # cap right after the cluster keeps it
    assert keep_count(s, 5, 0.0, 1e-12) == 5


def test_oracle_matches_its_stored_records():
    """Regression guard: the oracle still produces the records and Born
    probabilities stored by tests/golden/make_oracle_golden.py (a change to
    the oracle's arithmetic must regenerate them and say why)."""
    import os
    from oracle.shot import make_program, run_shot
    from workloads import D3_EXACT, theta_table
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_d3_records.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    w = D3_EXACT
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    for row in rows:
        s, bits, born = int(row[0]), row[1], np.array([float(x) for x in row[2:]])
        res = run_shot(w, s, theta, prog)
        assert "".join(str(b) for b in res.record) == bits
        assert np.abs(np.array(res.born) - born).max() < 1e-13


def test_gauge_moves_are_exact_and_canonical():
    """The QR gauge steps that move the orthogonality centre into an
    operator's support (Sec. IV B sweep, reading R7) leave the state unchanged
    and every site left of the centre a left isometry, every site right of it
    a right isometry."""
    rng = np.random.default_rng(5)
    n = 6
    m = MPS(n)
    # entangle with a few random two-branch operators, compressing exactly
    for lo, hi in [(0, 3), (2, 5), (1, 4), (0, 5)]:
        m.move_center_into(lo, hi)
        ops1 = {k: (rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))) for k in range(lo, hi + 1)}
        m.apply_two_branch(lo, hi, {}, ops1, 0.8, 0.6j)
        m.compress(lo, hi, chi_cap=64, cutoff=0.0, delta=0.0)
    psi = m.amplitudes()
    for target in [5, 0, 3, 1, 4, 2]:
        m.move_center(target)
        assert m.center == target
        assert np.abs(m.amplitudes() - psi).max() < 1e-12
        for k, a in enumerate(m.A):
            l, _, r = a.shape
            if k < target:
                mat = a.reshape(l * 2, r)
                assert np.abs(mat.conj().T @ mat - np.eye(r)).max() < 1e-12
            elif k > target:
                mat = a.reshape(l, 2 * r)
                assert np.abs(mat @ mat.conj().T - np.eye(l)).max() < 1e-12
