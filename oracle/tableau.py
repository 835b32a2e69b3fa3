"""Inverse Clifford tableau of a stabilizer tensor network state.

Test infrastructure only: the CUDA path never imports this module.

The state is |psi> = C |MPS> (Eq. 7).  C is kept through its inverse
tableau: for every physical generator g in {X_q, Z_q} the row
    T[g] = C^dagger g C
as an exact Pauli string (`oracle.pauli.Pauli`).  This gives directly what the
method needs (Sec. IV A, the Pauli-sum update after Eq. 7):
  * a Clifford gate G acting on the state:  C <- G C        (left_gate)
  * a Pauli error E (depolarising noise, Eq. 2-3; reset flips): C <- E C
  * a physical Pauli Q pushed into the MPS frame:  C^dagger Q C  (conjugate)
  * a Clifford W absorbed from the MPS side (measurement):  C <- C W
"""

import numpy as np

from .pauli import Pauli, conjugation_table, conjugate_by_gate


class InverseTableau:
    def __init__(self, n):
        self.n = n
        self.tx = [Pauli.single(n, q, "X") for q in range(n)]
        self.tz = [Pauli.single(n, q, "Z") for q in range(n)]

    def copy(self):
        t = InverseTableau.__new__(InverseTableau)
        t.n = self.n
        t.tx = [p.copy() for p in self.tx]
        t.tz = [p.copy() for p in self.tz]
        return t

    # -- pushing a physical Pauli string into the MPS frame ------------------
    def conjugate(self, q_phys):
        """C^dagger Q C for Q = i^m X^x Z^z: the image of each generator factor,
        multiplied in the same order (all X factors, then all Z factors)."""
        out = Pauli(q_phys.m, np.zeros(self.n, bool), np.zeros(self.n, bool))
        for k in np.flatnonzero(q_phys.x):
            out = out * self.tx[k]
        for k in np.flatnonzero(q_phys.z):
            out = out * self.tz[k]
        return out

    # -- C <- G C ---------------------------------------------------------------
    def left_gate(self, table, qubits):
        """G^dagger g G is i^m' X^x' Z^z' on `qubits`; its image under C is the
        ordered product of the old rows."""
        new_rows = {}
        for i, q in enumerate(qubits):
            for letter in "XZ":
                bits = [0] * (2 * len(qubits))
                bits[2 * i + (0 if letter == "X" else 1)] = 1
                m2, bits2 = table[tuple(bits)]
                row = Pauli(m2, np.zeros(self.n, bool), np.zeros(self.n, bool))
                for j, qj in enumerate(qubits):
                    if bits2[2 * j]:
                        row = row * self.tx[qj]
                    if bits2[2 * j + 1]:
                        row = row * self.tz[qj]
                new_rows[(q, letter)] = row
        for (q, letter), row in new_rows.items():
            if letter == "X":
                self.tx[q] = row
            else:
                self.tz[q] = row

    def left_pauli(self, letters, qubits):
        """C <- E C for a Hermitian Pauli E: T[g] -> C^dag E g E C = -T[g] when
        E anticommutes with g."""
        for letter, q in zip(letters, qubits):
            if letter in "XY":  # anticommutes with Z_q
                self.tz[q].m = (self.tz[q].m + 2) % 4
            if letter in "ZY":  # anticommutes with X_q
                self.tx[q].m = (self.tx[q].m + 2) % 4

    # -- C <- C W ---------------------------------------------------------------
    def right_gate(self, table, qubits):
        """Every row R -> W^dagger R W."""
        self.tx = [conjugate_by_gate(r, table, qubits) for r in self.tx]
        self.tz = [conjugate_by_gate(r, table, qubits) for r in self.tz]

    def right_unitary(self, matrix, qubits):
        self.right_gate(conjugation_table(matrix), qubits)

    # -- invariants -------------------------------------------------------------
    def is_symplectic(self):
        """Rows are images of the Pauli group generators under conjugation, so
        they must keep the canonical commutation relations, and be Hermitian."""
        rows = self.tx + self.tz
        for r in rows:
            if not r.is_hermitian():
                return False
        n = self.n
        for i in range(n):
            for j in range(n):
                if not self.tx[i].commutes(self.tx[j]):
                    return False
                if not self.tz[i].commutes(self.tz[j]):
                    return False
                anti = not self.tx[i].commutes(self.tz[j])
                if anti != (i == j):
                    return False
        return True

    def snapshot(self):
        """(x bits, z bits, phase) as arrays: rows X_0..X_{n-1}, Z_0..Z_{n-1}."""
        rows = self.tx + self.tz
        xs = np.array([r.x for r in rows], dtype=bool)
        zs = np.array([r.z for r in rows], dtype=bool)
        ms = np.array([r.m for r in rows], dtype=np.int64)
        return xs, zs, ms
