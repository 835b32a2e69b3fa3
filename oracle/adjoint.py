"""Gradient of log P(fixed record) with respect to the per-pair crosstalk
angles, by the adjoint method on the stabilizer tensor network (test
infrastructure only: the CUDA path never imports this module).

P(record) is the probability of the given measurement record with the
shot's Pauli-noise events held fixed (they are the shot's own counter-based
draws), so every measurement outcome is forced: the record bit XOR the
record's flip event.  The unnormalised final state is
    psi = O_N ... O_1 |0>,  P(record) = <psi|psi> = prod_m p_m,
with O_j a Clifford gate, a Pauli, a rotation U_j = exp(-i theta_k(j) Q_j)
(Eq. 4) or a measurement projector.  Since dU_j/dtheta = -i Q_j U_j,

    d log P / d theta_k = sum over rotations j of pair k of
                          2 Re <lambda_j| (-i Q_j) |psi_j> / <lambda_j|psi_j>,

with psi_j the state after O_j and lambda_j = O_{j+1}^dag ... O_N^dag psi.
The ratio does not depend on how either state is normalised, because
<lambda_j|psi_j> = <psi|psi> for every j.  In the frame C_j of Eq. 7 both are
MPSs, psi_j = C_j phi_j and lambda_j = C_j mu_j, and the terms become
<mu_j| (-i P'_j) |phi_j> / <mu_j|phi_j> with P'_j = C_j^dag Q_j C_j.  The
backward pass starts from mu = phi_N and steps back through the ops:
Clifford gates and Paulis leave mu alone (they only change the frame), a
rotation maps mu to exp(+i theta P') mu, a case-A projector applies itself
again, and a case-B measurement (frame C_{j-1} = C_j L U, phi_j =
|0><v|_j U phi_{j-1}) maps mu to U |v><0|_j mu.  Every application is
followed by the same truncating sweep as the forward pass (Sec. IV B), so
the gradient is that of the truncated simulation, exact when nothing is
truncated.
"""

import math

import numpy as np

from .mps import MPS
from .shot import P0, P1, ShotSim, make_program


def overlap(mu, phi, ops=None, phase=1.0):
    """phase * <mu| (x)_k ops[k] |phi> of two MPSs on the same sites (a
    missing op is the identity), by a transfer-matrix sweep."""
    ops = ops or {}
    env = np.ones((1, 1), dtype=np.complex128)
    for k in range(mu.n):
        a, b = mu.A[k], phi.A[k]
        if k in ops:
            b = np.einsum("st,atb->asb", ops[k], b)
        env = np.einsum("ac,asb,csd->bd", env, a.conj(), b)
    return phase * env[0, 0]


def _compress(w, m, lo, hi):
    m.compress(lo, hi, w.chi_cap, w.svd_cutoff, w.degeneracy_tol)


def logprob_and_grad(w, shot, theta, record, program=None):
    """(log P(record), d log P / d theta[K]) of one shot index and record."""
    prog = make_program(w) if program is None else program
    theta = np.asarray(theta, dtype=np.float64)
    sim = ShotSim(w, shot, theta, prog)
    sim.forced = list(record)
    sim.tape = []
    for op in prog.ops:
        sim.step(op)
    grad = np.zeros(len(theta))
    mu = sim.mps.copy()
    for entry in reversed(sim.tape):
        kind = entry[0]
        if kind == "rot":
            _, k, pp, lo, hi, phi = entry
            ops1 = {int(s): pp.site_matrix(s) for s in pp.support()}
            num = overlap(mu, phi, ops1, -1j * (1j ** pp.m))
            den = overlap(mu, phi)
            grad[k] += 2.0 * float(np.real(num / den))
            th = float(theta[k])
            mu.move_center_into(lo, hi)
            mu.apply_two_branch(lo, hi, {}, ops1, math.cos(th), 1j * math.sin(th) * (1j ** pp.m))
            _compress(w, mu, lo, hi)
        elif kind == "measA":
            _, ops, lo, hi, w1 = entry
            mu.move_center_into(lo, hi)
            mu.apply_two_branch(lo, hi, {}, ops, 0.5, w1)
            _compress(w, mu, lo, hi)
        else:
            _, ops1, lo, hi, j, v = entry
            mu.move_center_into(lo, hi)
            mu.apply_site(j, np.outer(v, np.array([1, 0], dtype=complex)))
            mu.apply_two_branch(lo, hi, {j: P0}, ops1, 1.0, 1.0)
            _compress(w, mu, lo, hi)
    return sim.logp, grad


def forced_logprob(w, shot, theta, record, program=None):
    """log P(record) alone (the forward pass with forced outcomes)."""
    prog = make_program(w) if program is None else program
    sim = ShotSim(w, shot, np.asarray(theta, dtype=np.float64), prog)
    sim.forced = list(record)
    for op in prog.ops:
        sim.step(op)
    return sim.logp
