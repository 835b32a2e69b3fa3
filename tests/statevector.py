"""Dense statevector simulation of the same physical program, used only to pin
the oracle: no tableau, no MPS, no Pauli conjugation.  Every gate, rotation
and measurement acts on the full 2^n amplitude vector (qubit 0 the most
significant bit), with the same event uniforms and noise rules.

Exact (no truncation), so for n <= ~20 it gives the Born probabilities and
records the stabilizer tensor network must reproduce when nothing is
truncated (Sec. IV A: the representation C|MPS> is exact).
"""

import math

import numpy as np

from oracle.philox import uniform

_H = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2.0)
_PAULI = {
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


class Dense:
    def __init__(self, n):
        self.n = n
        self.psi = np.zeros(2 ** n, dtype=complex)
        self.psi[0] = 1.0

    def _view(self):
        return self.psi.reshape((2,) * self.n)

    def apply1(self, q, mat):
        v = np.moveaxis(self._view(), q, 0)
        v = np.tensordot(mat, v, axes=([1], [0]))
        self.psi = np.moveaxis(v, 0, q).reshape(-1)

    def cnot(self, c, t):
        v = self._view().copy()
        idx = [slice(None)] * self.n
        idx[c] = 1
        sub = v[tuple(idx)]
        tt = t if t < c else t - 1
        v[tuple(idx)] = np.flip(sub, axis=tt)
        self.psi = v.reshape(-1)

    def bits(self, q):
        return (np.arange(2 ** self.n) >> (self.n - 1 - q)) & 1

    def rotation(self, a, b, theta, pauli):
        """exp(-i theta P_a P_b) for P in {Z, X}."""
        if pauli == "ZZ":
            s = (1 - 2 * self.bits(a)) * (1 - 2 * self.bits(b))
            self.psi = self.psi * np.exp(-1j * theta * s)
        else:
            flip = self.psi.copy()
            v = flip.reshape((2,) * self.n)
            v = np.flip(np.flip(v, axis=a), axis=b)
            self.psi = math.cos(theta) * self.psi - 1j * math.sin(theta) * v.reshape(-1)

    def measure_z(self, q, u):
        mask = self.bits(q)
        p0 = float(np.sum(np.abs(self.psi[mask == 0]) ** 2))
        p0 = min(1.0, max(0.0, p0))
        b = 0 if u < p0 else 1
        pb = p0 if b == 0 else 1.0 - p0
        self.psi = np.where(mask == b, self.psi, 0.0) / math.sqrt(pb)
        return b, pb


def run_dense(w, program, theta, shot, max_ops=None, return_state=False):
    """Records and realised Born probabilities of one shot (and the dense
    state after the first max_ops ops when return_state)."""
    n = program.layout.n
    st = Dense(n)
    p = w.p
    p1, p2, pR, pM = p * w.p1_scale, p * w.p2_scale, p * w.pR_scale, p * w.pM_scale
    record = [0] * program.n_meas
    born = [0.0] * program.n_meas

    def u(ev):
        return uniform(w.seed, shot, ev)

    for i, op in enumerate(program.ops):
        if max_ops is not None and i >= max_ops:
            break
        kind = op[0]
        if kind == "RN":
            if u(op[2]) < pR:
                st.apply1(op[1], _PAULI["X"])
        elif kind == "H":
            st.apply1(op[1], _H)
        elif kind == "D1":
            x = u(op[2])
            if x < p1:
                st.apply1(op[1], _PAULI["XYZ"[min(2, int(3 * x / p1))]])
        elif kind == "CX":
            st.cnot(op[1], op[2])
        elif kind == "D2":
            x = u(op[3])
            if x < p2:
                idx = min(14, int(15 * x / p2)) + 1
                lc, lt = "IXYZ"[idx // 4], "IXYZ"[idx % 4]
                if lc != "I":
                    st.apply1(op[1], _PAULI[lc])
                if lt != "I":
                    st.apply1(op[2], _PAULI[lt])
        elif kind == "ROT":
            pair = program.pairs[op[1]]
            st.rotation(pair.a, pair.b, float(theta[op[1]]), pair.pauli)
        elif kind == "M":
            q, evb, evf, rec, reset, evr = op[1:]
            b, pb = st.measure_z(q, u(evb))
            born[rec] = pb
            record[rec] = b ^ (1 if u(evf) < pM else 0)
            if reset:
                if b:
                    st.apply1(q, _PAULI["X"])
                if u(evr) < pR:
                    st.apply1(q, _PAULI["X"])
    if return_state:
        return record, born, st
    return record, born
