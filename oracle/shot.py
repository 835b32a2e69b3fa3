"""One shot of noisy surface-code syndrome extraction with coherent crosstalk,
simulated as a stabilizer tensor network |psi> = C |MPS> (Eq. 7).

Test infrastructure only: the CUDA path never imports this module.

Per op of the program (`oracle.circuit.build_program`):
  * Clifford gate G:  C <- G C  (Sec. IV A: Clifford gates update C only).
  * Pauli noise E (Eq. 2-3, Table I): C <- E C, one uniform per event: the
    event fires when u < p; the Pauli is number floor(k u / p) (clamped)
    among the k = 3 (one qubit, X, Y, Z) or 15 (two qubits, base-4 digits
    (control, target) over I, X, Y, Z, skipping II) non-identity Paulis.
  * Crosstalk exp(-i theta Q) (Eq. 4, sign reading exp(-i theta Q)):
    P' = C^dag Q C, then cos(theta) I - i sin(theta) P' on the MPS as a
    bond-2 MPO, then compression (Sec. IV B) over the support [lo, hi] of P'
    (`prepare_span`: the orthogonality centre is first moved into [lo, hi]
    by exact QR gauge steps, so only the bonds the MPO doubled are
    truncated).
  * Z measurement of qubit q (Sec. IV A: a Pauli pushed through C and applied
    to the tensor network): P' = C^dag Z_q C, e = <phi|P'|phi>,
    p0 = (1 + e)/2, outcome b = 0 iff u < p0.
      - P' without X or Y (case A): project with (I + (-1)^b P')/2.
      - Otherwise (case B): j = first site where P' has X or Y; the
        controlled-Pauli product U (control j, target P'_k on every other
        site of the support) satisfies P' = s U P'_j U^dag, so the projector is
        U (I + lambda P'_j)/2 U^dag with lambda = (-1)^b s.  The MPS becomes
        L |v><v|_j U^dag |phi> with |v> the lambda eigenvector of P'_j and L a
        one-qubit Clifford taking |v> to |0>, and C <- C U L^dag.  This keeps
        a measured stabilizer as a single Z on the MPS, so the MPS holds only
        the non-Clifford part of the state (Sec. IV A, last paragraphs).
    The record bit is b flipped with probability pM; an ancilla is then reset
    (X when b = 1) and flipped with probability pR.
"""

import math
from dataclasses import dataclass, field

import numpy as np

from .circuit import build_layout, build_pairs, build_program, detectors, logical_z
from .mps import MPS
from .pauli import (CNOT, CY, CZ, H2, I2, S2, TABLE_CNOT, TABLE_CY, TABLE_CZ, TABLE_H,
                    X2, Y2, Z2, Pauli, conjugation_table)
from .philox import uniform
from .tableau import InverseTableau

LETTER = {"X": X2, "Y": Y2, "Z": Z2}
CTRL_TABLE = {"X": TABLE_CNOT, "Y": TABLE_CY, "Z": TABLE_CZ}
SQ2 = 1.0 / math.sqrt(2.0)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)
SDG = S2.conj().T

# lambda-eigenvector v of X or Y and the Clifford L with L v = |0>.
EIGVEC = {
    ("X", 1): np.array([SQ2, SQ2], dtype=complex),
    ("X", -1): np.array([SQ2, -SQ2], dtype=complex),
    ("Y", 1): np.array([SQ2, 1j * SQ2], dtype=complex),
    ("Y", -1): np.array([SQ2, -1j * SQ2], dtype=complex),
}
LMAT = {
    ("X", 1): H2,
    ("X", -1): X2 @ H2,
    ("Y", 1): H2 @ SDG,
    ("Y", -1): X2 @ H2 @ SDG,
}
LDAG_TABLE = {key: conjugation_table(m.conj().T) for key, m in LMAT.items()}

NEAR_THRESHOLD = 1e-5


@dataclass
class ShotResult:
    record: list
    born: list  # probability of the realised outcome, per measurement
    logp: float
    max_chi: int
    discarded: float
    near_draws: int  # Born draws with |u - p0| < NEAR_THRESHOLD
    tableau: object = None
    mps: object = None
    trace: list = field(default_factory=list)


class ShotSim:
    """The state of one shot and the ops acting on it."""

    def __init__(self, w, shot, theta, program, trace=False):
        self.w = w
        self.shot = shot
        self.theta = np.asarray(theta, dtype=np.float64)
        self.prog = program
        n = program.layout.n
        self.n = n
        self.T = InverseTableau(n)
        self.mps = MPS(n)
        p = w.p
        self.p1, self.p2 = p * w.p1_scale, p * w.p2_scale
        self.pR, self.pM = p * w.pR_scale, p * w.pM_scale
        self.record = [0] * program.n_meas
        self.born = [0.0] * program.n_meas
        self.logp = 0.0
        self.max_chi = 1
        self.discarded = 0.0
        self.near = 0
        self.want_trace = trace
        self.trace = []
        # forced outcomes (the adjoint's forward pass): record bits to
        # reproduce, each outcome being the record bit XOR its record flip
        self.forced = None
        # with a list here, rotations and measurements append what the
        # adjoint's backward pass needs (see oracle.adjoint)
        self.tape = None

    def u(self, ev):
        return uniform(self.w.seed, self.shot, ev)

    def _compress(self, lo, hi, kind):
        before = self.mps.bonds()[lo:hi] if self.want_trace else None
        disc, chi = self.mps.compress(lo, hi, self.w.chi_cap, self.w.svd_cutoff, self.w.degeneracy_tol)
        self.discarded += disc
        self.max_chi = max(self.max_chi, chi)
        if self.want_trace:
            self.trace.append((kind, lo, hi, before, self.mps.bonds()[lo - 1 if lo else 0:hi + 1]))

    # -- noise ----------------------------------------------------------------
    def dep1(self, q, ev):
        u = self.u(ev)
        if u < self.p1:
            idx = min(2, int(3.0 * u / self.p1))
            self.T.left_pauli("XYZ"[idx], [q])

    def dep2(self, c, t, ev):
        u = self.u(ev)
        if u < self.p2:
            idx = min(14, int(15.0 * u / self.p2)) + 1
            lc, lt = "IXYZ"[idx // 4], "IXYZ"[idx % 4]
            if lc != "I":
                self.T.left_pauli(lc, [c])
            if lt != "I":
                self.T.left_pauli(lt, [t])

    def reset_flip(self, q, ev):
        if self.u(ev) < self.pR:
            self.T.left_pauli("X", [q])

    # -- non-Clifford and measurement ------------------------------------------
    def prepare_span(self, lo, hi):
        """Sites swept by the compression after an operator on [lo, hi].
        Sec. IV B truncates the bonds the operator's MPO enlarged, and leaves
        the rest of the sweep open; here the orthogonality centre is moved
        into [lo, hi] first by exact QR gauge steps (no truncation), so the
        sites left of lo are left-canonical, those right of hi
        right-canonical, and the sweep covers exactly the support."""
        self.mps.move_center_into(lo, hi)
        return lo, hi

    def rotation(self, k):
        pair = self.prog.pairs[k]
        q = Pauli.identity(self.n)
        for site in (pair.a, pair.b):
            if pair.pauli == "ZZ":
                q.z[site] = True
            else:
                q.x[site] = True
        pp = self.T.conjugate(q)
        th = float(self.theta[k])
        supp = pp.support()
        lo, hi = int(supp.min()), int(supp.max())
        a, b = self.prepare_span(lo, hi)
        ops1 = {int(s): pp.site_matrix(s) for s in supp}
        w1 = -1j * math.sin(th) * (1j ** pp.m)
        self.mps.apply_two_branch(lo, hi, {}, ops1, math.cos(th), w1)
        self._compress(a, b, "rot")
        if self.tape is not None:
            self.tape.append(("rot", k, pp, lo, hi, self.mps.copy()))

    def measure(self, q, ev_b, ev_f, rec, reset, ev_r):
        zq = Pauli.single(self.n, q, "Z")
        pp = self.T.conjugate(zq)
        supp = pp.support()
        lo, hi = int(supp.min()), int(supp.max())
        ops = {int(s): pp.site_matrix(s) for s in supp}
        e = float(np.real(self.mps.expect(ops, 1j ** pp.m)))
        p0 = min(1.0, max(0.0, 0.5 * (1.0 + e)))
        u = self.u(ev_b)
        b = 0 if u < p0 else 1
        if self.forced is not None:
            b = self.forced[rec] ^ (1 if self.u(ev_f) < self.pM else 0)
        if abs(u - p0) < NEAR_THRESHOLD:
            self.near += 1
        pb = p0 if b == 0 else 1.0 - p0
        self.born[rec] = pb
        self.logp += math.log(pb) if pb > 0 else -math.inf
        sa, sb = self.prepare_span(lo, hi)
        if not pp.x.any():
            w1 = (1 if b == 0 else -1) * (1j ** pp.m) * 0.5
            self.mps.apply_two_branch(lo, hi, {}, ops, 0.5, w1)
            self._compress(sa, sb, "measA")
            if self.tape is not None:
                self.tape.append(("measA", ops, lo, hi, w1))
        else:
            j = int(np.flatnonzero(pp.x)[0])
            letters = pp.letters()
            lam = (1 if b == 0 else -1) * pp.sign()
            key = (letters[j], lam)
            ops0 = {j: P0}
            ops1 = {j: P1}
            for s in supp:
                s = int(s)
                if s != j:
                    ops1[s] = LETTER[letters[s]]
            self.mps.apply_two_branch(lo, hi, ops0, ops1, 1.0, 1.0)
            v = EIGVEC[key]
            self.mps.apply_site(j, np.outer(np.array([1, 0], dtype=complex), v.conj()))
            self._compress(sa, sb, "measB")
            if self.tape is not None:
                self.tape.append(("measB", ops1, lo, hi, j, v))
            for s in supp:
                s = int(s)
                if s != j:
                    self.T.right_gate(CTRL_TABLE[letters[s]], (j, s))
            self.T.right_gate(LDAG_TABLE[key], (j,))
        flip = 1 if self.u(ev_f) < self.pM else 0
        self.record[rec] = b ^ flip
        if reset:
            if b:
                self.T.left_pauli("X", [q])
            self.reset_flip(q, ev_r)
        return b

    # -- driver -----------------------------------------------------------------
    def step(self, op):
        kind = op[0]
        if kind == "RN":
            self.reset_flip(op[1], op[2])
        elif kind == "H":
            self.T.left_gate(TABLE_H, [op[1]])
        elif kind == "D1":
            self.dep1(op[1], op[2])
        elif kind == "CX":
            self.T.left_gate(TABLE_CNOT, [op[1], op[2]])
        elif kind == "D2":
            self.dep2(op[1], op[2], op[3])
        elif kind == "ROT":
            self.rotation(op[1])
        elif kind == "M":
            self.measure(*op[1:])
        else:
            raise ValueError(kind)

    def result(self):
        return ShotResult(self.record, self.born, self.logp, self.max_chi, self.discarded,
                          self.near, self.T, self.mps, self.trace)


def make_program(w):
    layout = build_layout(w.distance, w.cnot_schedule)
    pairs = build_pairs(layout, w.pair_rule, w.pairs)
    return build_program(layout, pairs, w.rounds, w.memory_basis)


def run_shot(w, shot, theta=None, program=None, trace=False, max_ops=None):
    """Simulate shot `shot` of workload `w`; theta is the per-pair angle table
    (default: workloads.theta_table)."""
    if program is None:
        program = make_program(w)
    if theta is None:
        from workloads import theta_table
        theta = theta_table(w, len(program.pairs))
    sim = ShotSim(w, shot, theta, program, trace=trace)
    for i, op in enumerate(program.ops):
        if max_ops is not None and i >= max_ops:
            break
        sim.step(op)
    return sim.result()


def shot_detectors(program, result):
    return detectors(program, result.record), logical_z(program, result.record)
