"""Pauli strings with an exact phase, and Clifford conjugation tables built by
brute force from gate matrices.

Test infrastructure only: the CUDA path never imports this module.

A Pauli string on n qubits is held as (m, x, z): the operator
    i**m * X**x * Z**z,   X**x Z**z = prod_k X_k**x_k Z_k**z_k,
with m in Z4 and x, z boolean vectors.  The Hermitian string with Y on a site
where x_k = z_k = 1 is i**popcount(x & z) X**x Z**z, since Y = iXZ.

The stabilizer-tensor-network method (Sec. IV A, Eq. 7 and the Pauli-sum
update after it) conjugates Pauli strings through a Clifford operator C; the
phase of each product is what decides the sign of every later rotation and
the outcome of every later measurement, so it is tracked exactly here.
"""

import itertools

import numpy as np

I2 = np.eye(2, dtype=complex)
X2 = np.array([[0, 1], [1, 0]], dtype=complex)
Z2 = np.array([[1, 0], [0, -1]], dtype=complex)
Y2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
H2 = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2.0)
S2 = np.array([[1, 0], [0, 1j]], dtype=complex)


class Pauli:
    """i**m X**x Z**z on n qubits."""

    __slots__ = ("m", "x", "z")

    def __init__(self, m, x, z):
        self.m = int(m) % 4
        self.x = np.asarray(x, dtype=bool).copy()
        self.z = np.asarray(z, dtype=bool).copy()

    @staticmethod
    def identity(n):
        return Pauli(0, np.zeros(n, bool), np.zeros(n, bool))

    @staticmethod
    def single(n, q, letter):
        """Hermitian single-qubit Pauli letter ('I','X','Y','Z') on qubit q."""
        p = Pauli.identity(n)
        if letter in "XY":
            p.x[q] = True
        if letter in "ZY":
            p.z[q] = True
        if letter == "Y":
            p.m = 1  # Y = i X Z
        return p

    def copy(self):
        return Pauli(self.m, self.x, self.z)

    @property
    def n(self):
        return len(self.x)

    def __mul__(self, other):
        """(i^m1 X^x1 Z^z1)(i^m2 X^x2 Z^z2) = i^(m1+m2+2 z1.x2) X^(x1^x2) Z^(z1^z2).

        Moving Z^z1 past X^x2 gives (-1)**(z1.x2); X's commute with X's and
        Z's with Z's.
        """
        swap = int(np.count_nonzero(self.z & other.x))
        return Pauli(self.m + other.m + 2 * swap, self.x ^ other.x, self.z ^ other.z)

    def commutes(self, other):
        s = np.count_nonzero(self.x & other.z) + np.count_nonzero(self.z & other.x)
        return s % 2 == 0

    def is_hermitian(self):
        return (self.m - np.count_nonzero(self.x & self.z)) % 2 == 0

    def sign(self):
        """+1 or -1 for a Hermitian string: i^m X^x Z^z = sign * (tensor of I,X,Y,Z)."""
        assert self.is_hermitian()
        r = (self.m - np.count_nonzero(self.x & self.z)) % 4
        return 1 if r == 0 else -1

    def letters(self):
        out = []
        for xk, zk in zip(self.x, self.z):
            out.append("IZXY"[int(xk) * 2 + int(zk)])
        return "".join(out)

    def support(self):
        return np.flatnonzero(self.x | self.z)

    def site_matrix(self, k):
        """X^x_k Z^z_k as a 2x2 matrix (the per-site factor, phase excluded)."""
        m = I2
        if self.x[k]:
            m = m @ X2
        if self.z[k]:
            m = m @ Z2
        return m

    def key(self):
        return (self.m, self.x.tobytes(), self.z.tobytes())

    def __eq__(self, other):
        return self.m == other.m and np.array_equal(self.x, other.x) and np.array_equal(self.z, other.z)

    def __repr__(self):
        return f"Pauli(i^{self.m} X^{self.x.astype(int)} Z^{self.z.astype(int)})"


def local_xz_matrix(bits):
    """X^x Z^z on len(bits)//2 qubits, bits = (x0, z0, x1, z1, ...), qubit 0 the
    most significant kron factor."""
    mat = np.ones((1, 1), dtype=complex)
    for k in range(len(bits) // 2):
        f = I2
        if bits[2 * k]:
            f = f @ X2
        if bits[2 * k + 1]:
            f = f @ Z2
        mat = np.kron(mat, f)
    return mat


def conjugation_table(gate):
    """Table of G^dagger (X^x Z^z) G for every local X^x Z^z of a k-qubit gate.

    Keys and values are bit tuples (x0, z0, x1, z1, ...); the value also holds
    the phase exponent m' with G^dag (X^x Z^z) G = i^m' X^x' Z^z'.
    Found by comparing dense matrices, so it is correct for any Clifford G.
    """
    gate = np.asarray(gate, dtype=complex)
    k = int(round(np.log2(gate.shape[0])))
    table = {}
    candidates = []
    for bits in itertools.product((0, 1), repeat=2 * k):
        candidates.append((bits, local_xz_matrix(bits)))
    for bits, mat in candidates:
        target = gate.conj().T @ mat @ gate
        found = None
        for bits2, mat2 in candidates:
            for m in range(4):
                if np.allclose(target, (1j ** m) * mat2, atol=1e-12):
                    found = (m, bits2)
                    break
            if found:
                break
        if found is None:
            raise ValueError("gate is not a Clifford")
        table[bits] = found
    return table


def conjugate_by_gate(p, table, qubits):
    """G^dag P G for a Pauli string P and a gate G on `qubits` (table from
    `conjugation_table`).  The local factor on `qubits` is replaced; factors on
    other qubits commute with it, so X^x Z^z splits per qubit with no phase."""
    bits = []
    for q in qubits:
        bits += [int(p.x[q]), int(p.z[q])]
    m2, bits2 = table[tuple(bits)]
    out = p.copy()
    out.m = (out.m + m2) % 4
    for i, q in enumerate(qubits):
        out.x[q] = bool(bits2[2 * i])
        out.z[q] = bool(bits2[2 * i + 1])
    return out


def controlled(u):
    """|0><0| (x) I + |1><1| (x) u, control first."""
    u = np.asarray(u, dtype=complex)
    return np.block([[np.eye(2), np.zeros((2, 2))], [np.zeros((2, 2)), u]])


CNOT = controlled(X2)
CZ = controlled(Z2)
CY = controlled(Y2)

TABLE_H = conjugation_table(H2)
TABLE_S = conjugation_table(S2)
TABLE_SDG = conjugation_table(S2.conj().T)
TABLE_X = conjugation_table(X2)
TABLE_CNOT = conjugation_table(CNOT)
TABLE_CZ = conjugation_table(CZ)
TABLE_CY = conjugation_table(CY)
