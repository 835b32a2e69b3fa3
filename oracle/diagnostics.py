"""Diagnostics of a shot's stabilizer tensor network (test infrastructure
only: the CUDA path never imports this module).

* `schmidt_values(mps, cut)`: the squared Schmidt coefficients of the MPS
  across the cut between sites `cut` and `cut + 1` (Sec. IV B, Fig. 2 plots
  them at the centre cut), largest first.  With the orthogonality centre at
  site `cut`, they are the squared singular values of that site's tensor as
  a (chi_{cut-1} * 2) x chi_cut matrix.
* `logical_expectation(tableau, mps, qubits, letter)`: <psi| L |psi> of the
  logical operator L = (x)_q letter_q on the physical state C|MPS> (Eq. 7):
  L is pushed through the frame, P' = C^dag L C, and <MPS| P' |MPS> is
  contracted.  Sec. II, Eq. 1 averages |sin(theta_i/2)| over syndromes,
  where the post-syndrome state has its logical operator at angle theta_i:
  with the decoder's correction c, (-1)^c <L> = cos theta_i, so
  sin^2(theta_i/2) = (1 - (-1)^c <L>) / 2.
"""

import numpy as np

from .pauli import Pauli


def schmidt_values(mps, cut):
    m = mps.copy()
    m.move_center(cut)
    a = m.A[cut]
    l, _, r = a.shape
    s = np.linalg.svd(a.reshape(l * 2, r), compute_uv=False)
    return np.sort(s * s)[::-1]


def logical_expectation(tableau, mps, qubits, letter="Z"):
    n = mps.n
    p = Pauli.identity(n)
    for q in qubits:
        if letter == "Z":
            p.z[q] = True
        else:
            p.x[q] = True
    pp = tableau.conjugate(p)
    ops = {int(s): pp.site_matrix(s) for s in pp.support()}
    return float(np.real(mps.expect(ops, 1j ** pp.m)))


def eq1_term(expectation, correction):
    """|sin(theta_i / 2)| of one syndrome from <L> and the decoder's
    correction bit c: sqrt((1 - (-1)^c <L>) / 2), clipped at rounding."""
    q = 0.5 * (1.0 - (-1.0) ** int(correction) * expectation)
    return float(np.sqrt(min(1.0, max(0.0, q))))
