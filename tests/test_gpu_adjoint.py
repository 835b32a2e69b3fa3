"""The adjoint gradient of log P(fixed record) (stn_logprob_grad) on the GPU
against the oracle's FP64 adjoint (oracle.adjoint), against central finite
differences (h = 1e-4) of the GPU's own forced-record log-likelihood, through
the torch.autograd wrapper, and used to fit a crosstalk angle to synthetic
records generated at a known angle."""

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from oracle.adjoint import logprob_and_grad
from oracle.shot import make_program
from workloads import D3_EXACT, D5_BENCH, PRECISION_C64, theta_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stn.build()


EXACT = D3_EXACT.with_(rounds=2, chi_cap=256, svd_cutoff=1e-14, degeneracy_tol=0.0, p=0.01, theta=0.2,
                       theta_sigma=0.05)


def sampled_records(w, shots, offset, theta):
    sim = stn.Simulator(w, max_shots=shots)
    out = sim.sample_shots(shots, offset, theta)
    sim.close()
    return out["records"], out["bits"]


@pytest.mark.parametrize("basis", ["Z", "X"])
def test_gpu_adjoint_matches_oracle_fp64(basis):
    w = EXACT.with_(memory_basis=basis, rounds=2 if basis == "Z" else 1)
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    recs, bits = sampled_records(w, 3, 5, theta)
    sim = stn.Simulator(w, max_shots=3)
    logp, grad = sim.logprob_grad(recs, theta, shot_offset=5)
    g_ref = np.zeros(len(theta))
    for r in range(3):
        lp_ref, g = logprob_and_grad(w, 5 + r, theta, list(bits[r]), prog)
        g_ref += g
        assert abs(logp[r] - lp_ref) < 1e-10 * max(1.0, abs(lp_ref))
    assert np.abs(grad - g_ref).max() < 1e-8 * max(1.0, np.abs(g_ref).max()), np.abs(grad - g_ref).max()
    assert np.abs(g_ref).max() > 0.1  # the records do depend on the angles


def test_gpu_adjoint_matches_central_differences():
    w = EXACT
    sim = stn.Simulator(w, max_shots=2)
    theta = theta_table(w, sim.n_pairs)
    recs, _ = sampled_records(w, 2, 0, theta)
    _, grad = sim.logprob_grad(recs, theta)
    h = 1e-4
    for k in range(0, len(theta), 5):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (sim.logprob_grad(recs, tp)[0].sum() - sim.logprob_grad(recs, tm)[0].sum()) / (2 * h)
        assert abs(grad[k] - fd) < 1e-6 * max(1.0, abs(fd)), (k, grad[k], fd)


def test_gpu_adjoint_complex64_against_oracle():
    """The complex64 path at its own cutoff against the FP64 oracle at the
    same cutoff: gradients within 1e-3 of the largest component."""
    w = D3_EXACT.with_(rounds=2, p=0.01, theta=0.2, theta_sigma=0.05, precision=PRECISION_C64,
                       svd_cutoff=D5_BENCH.svd_cutoff, degeneracy_tol=D5_BENCH.degeneracy_tol)
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    recs, bits = sampled_records(w, 2, 0, theta)
    sim = stn.Simulator(w, max_shots=2)
    logp, grad = sim.logprob_grad(recs, theta)
    g_ref = sum(logprob_and_grad(w, r, theta, list(bits[r]), prog)[1] for r in range(2))
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-3 * scale, (np.abs(grad - g_ref).max(), scale)


def test_autograd_wrapper_and_angle_fit():
    """Records of a d = 3 one-round X-memory generated at a shared angle
    theta* = 0.15; the score d/dtheta sum_r log P(r | theta), from the
    autograd wrapper, changes sign within 0.03 of theta*, and the wrapper's
    gradient equals the adjoint's summed over the pairs."""
    from scipy.optimize import brentq
    from paper_2605_29514_gb300.autograd import record_log_likelihood
    w = D3_EXACT.with_(rounds=1, chi_cap=16, memory_basis="X", theta=0.15)
    n = 600
    sim = stn.Simulator(w, max_shots=300)
    recs, _ = sampled_records(w, n, 0, theta_table(w, sim.n_pairs))

    def score(t):
        th = torch.full((sim.n_pairs,), float(t), dtype=torch.float64, requires_grad=True)
        ll = record_log_likelihood(th, sim, recs)
        ll.backward()
        return float(th.grad.sum())

    s_lo, s_hi = score(0.08), score(0.25)
    assert s_lo > 0 > s_hi
    t_hat = brentq(score, 0.08, 0.25, xtol=2e-3)
    assert abs(t_hat - 0.15) < 0.03, t_hat
    th = torch.full((sim.n_pairs,), 0.15, dtype=torch.float64, requires_grad=True)
    ll = record_log_likelihood(th, sim, recs[:100])
    ll.backward()
    _, g = sim.logprob_grad(recs[:100], np.full(sim.n_pairs, 0.15))
    assert np.allclose(th.grad.numpy(), g, rtol=1e-12, atol=1e-12)
