"""Matrix product state with an orthogonality centre, in complex128.

Test infrastructure only: the CUDA path never imports this module.

Site k holds A[k] with shape (chi_{k-1}, 2, chi_k).  The operations are the
ones the stabilizer tensor network needs (Sec. IV A and IV B):

  * `apply_two_branch`: a sum of two Pauli-string-like products,
        O = w0 * (x)_k B0_k + w1 * (x)_k B1_k     on sites lo..hi,
    as a bond-dimension-2 MPO.  A rotation exp(-i theta P') is
    cos(theta) I - i sin(theta) P'; a projector (I + s P')/2 and the
    controlled-Pauli unitary of a measurement have the same form.
  * `compress`: after an MPO on [lo, hi], a left-to-right QR sweep over the
    span followed by a right-to-left SVD sweep that keeps the largest
    singular values at every bond (Eq. 8 and the chi_max truncation after it).
  * `expect`: <phi| O |phi> by a plain transfer-matrix sweep over all sites.
"""

import numpy as np


def keep_count(s, chi_cap, cutoff, delta):
    """Number of singular values kept at one bond.

    s is sorted in decreasing order.  Values at or below cutoff * s[0] are
    dropped.  If more than chi_cap remain, the chi_cap largest are kept
    (Eq. 8 discards the smallest Schmidt terms), except that every kept value
    must exceed the first discarded one by more than delta * s[0]: with
    degenerate Schmidt values at the cap the kept subspace would otherwise
    not be unique.
    """
    if s.size == 0 or s[0] <= 0.0:
        return 1
    s1 = s[0]
    k = int(np.count_nonzero(s > cutoff * s1))
    k = max(k, 1)
    if k > chi_cap:
        threshold = s[chi_cap] + delta * s1
        k = int(np.count_nonzero(s[:chi_cap] > threshold))
        k = max(k, 1)
    return k


class MPS:
    def __init__(self, n):
        self.n = n
        self.A = []
        for _ in range(n):
            t = np.zeros((1, 2, 1), dtype=np.complex128)
            t[0, 0, 0] = 1.0
            self.A.append(t)
        self.center = 0

    def copy(self):
        m = MPS.__new__(MPS)
        m.n = self.n
        m.A = [a.copy() for a in self.A]
        m.center = self.center
        return m

    def bonds(self):
        return [self.A[k].shape[2] for k in range(self.n - 1)]

    # -- exact gauge moves ------------------------------------------------------
    def _shift_right(self, k):
        l, _, r = self.A[k].shape
        q, rr = np.linalg.qr(self.A[k].reshape(l * 2, r))
        self.A[k] = q.reshape(l, 2, q.shape[1])
        self.A[k + 1] = np.einsum("ab,bsc->asc", rr, self.A[k + 1])

    def _shift_left(self, k):
        l, _, r = self.A[k].shape
        q, rr = np.linalg.qr(self.A[k].reshape(l, 2 * r).conj().T)
        self.A[k] = q.conj().T.reshape(q.shape[1], 2, r)
        self.A[k - 1] = np.einsum("asb,bc->asc", self.A[k - 1], rr.conj().T)

    def move_center(self, target):
        while self.center < target:
            self._shift_right(self.center)
            self.center += 1
        while self.center > target:
            self._shift_left(self.center)
            self.center -= 1

    def move_center_into(self, lo, hi):
        if self.center < lo:
            self.move_center(lo)
        elif self.center > hi:
            self.move_center(hi)

    # -- operators --------------------------------------------------------------
    def apply_site(self, k, op):
        self.A[k] = np.einsum("st,atb->asb", op, self.A[k])

    def apply_two_branch(self, lo, hi, ops0, ops1, w0, w1):
        """O = w0 (x)_k ops0[k] + w1 (x)_k ops1[k] over sites lo..hi; a missing
        entry is the identity.  Bonds strictly inside the span double."""
        eye = np.eye(2, dtype=np.complex128)
        if lo == hi:
            op = w0 * ops0.get(lo, eye) + w1 * ops1.get(lo, eye)
            self.apply_site(lo, op)
            return
        for k in range(lo, hi + 1):
            a = self.A[k]
            b0 = np.einsum("st,atb->asb", ops0.get(k, eye), a)
            b1 = np.einsum("st,atb->asb", ops1.get(k, eye), a)
            l, _, r = a.shape
            if k == lo:
                new = np.zeros((l, 2, 2 * r), dtype=np.complex128)
                new[:, :, :r] = w0 * b0
                new[:, :, r:] = w1 * b1
            elif k == hi:
                new = np.zeros((2 * l, 2, r), dtype=np.complex128)
                new[:l] = b0
                new[l:] = b1
            else:
                new = np.zeros((2 * l, 2, 2 * r), dtype=np.complex128)
                new[:l, :, :r] = b0
                new[l:, :, r:] = b1
            self.A[k] = new

    def compress(self, lo, hi, chi_cap, cutoff, delta):
        """QR sweep lo -> hi, then SVD truncation sweep hi -> lo; the centre
        ends at lo and the state is renormalised.  Requires sites < lo to be
        left-canonical and sites > hi right-canonical (centre was in [lo, hi]
        when the operator was applied).  Returns (discarded weight, max bond)."""
        for k in range(lo, hi):
            self._shift_right(k)
        discarded = 0.0
        for k in range(hi, lo, -1):
            l, _, r = self.A[k].shape
            u, s, vh = np.linalg.svd(self.A[k].reshape(l, 2 * r), full_matrices=False)
            keep = keep_count(s, chi_cap, cutoff, delta)
            total = float(np.sum(s * s))
            if total > 0.0:
                discarded += float(np.sum(s[keep:] ** 2)) / total
            self.A[k] = vh[:keep].reshape(keep, 2, r)
            self.A[k - 1] = np.einsum("asb,bc->asc", self.A[k - 1], u[:, :keep] * s[:keep])
        self.center = lo
        nrm = np.linalg.norm(self.A[lo])
        self.A[lo] = self.A[lo] / nrm
        return discarded, max(self.bonds()) if self.n > 1 else 1

    def expect(self, ops, phase=1.0):
        """phase * <phi| (x)_k ops[k] |phi> by a full transfer-matrix sweep."""
        env = np.ones((1, 1), dtype=np.complex128)
        eye = np.eye(2, dtype=np.complex128)
        for k in range(self.n):
            a = self.A[k]
            oa = np.einsum("st,atb->asb", ops.get(k, eye), a)
            env = np.einsum("ac,asb,csd->bd", env, a.conj(), oa)
        return phase * env[0, 0]

    def norm2(self):
        return float(np.real(self.expect({})))

    def amplitudes(self):
        """Dense vector (qubit 0 most significant); for small n only."""
        v = self.A[0].reshape(2, -1)
        for k in range(1, self.n):
            v = np.einsum("pa,asb->psb", v, self.A[k]).reshape(-1, self.A[k].shape[2])
        return v.reshape(-1)
