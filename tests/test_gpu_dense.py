"""Kernel-level checks of the truncation sweep's dense routines (Sec. IV B):
the Householder R factor and the one-sided Jacobi SVD, each run alone on one
CTA through the C ABI and compared with numpy (LAPACK) in float64."""

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CDT = {0: torch.complex128, 1: torch.complex64}
RDT = {0: torch.float64, 1: torch.float32}
TOL = {0: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stn.build()


def rand(rng, m, n, decay=0.0):
    a = rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    if decay:
        u, s, vh = np.linalg.svd(a, full_matrices=False)
        s = np.exp(-decay * np.arange(len(s)))
        a = (u * s) @ vh
    return a


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n", [(2, 1), (8, 4), (64, 32), (33, 47), (96, 48), (300, 120), (1024, 512),
                                 (40, 300)])
def test_qr_r_factor(precision, m, n):
    rng = np.random.default_rng(m * 1000 + n)
    a = rand(rng, m, n, decay=0.05)
    d = torch.tensor(a, dtype=CDT[precision], device="cuda")
    stn.dense_qr(precision, m, n, d.data_ptr())
    torch.cuda.synchronize()
    r = d.cpu().numpy().astype(np.complex128)
    k = min(m, n)
    assert np.allclose(r[k:], 0)
    assert np.allclose(np.tril(r[:k, :k], -1), 0)
    # R^dag R = A^dag A  (R is a QR factor up to a diagonal phase)
    g = a.conj().T @ a
    err = np.abs(r[:k].conj().T @ r[:k] - g).max() / np.abs(g).max()
    assert err < TOL[precision], err


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,smem,decay", [(4, 4, 1, 0.1), (32, 32, 1, 0.1), (16, 40, 1, 0.1),
                                            (60, 24, 1, 0.1), (64, 64, 0, 0.1), (130, 70, 0, 0.1),
                                            (64, 64, 2, 0.1), (200, 150, 2, 0.5), (120, 256, 2, 0.5),
                                            (512, 512, 2, 0.5)])
def test_onesided_svd(precision, m, n, smem, decay):
    """Clustered spectra (decay 0.1: neighbours within 10%) on the small cases;
    the large, blocked cases use the strongly graded spectra of MPS bonds
    (Schmidt values falling by orders of magnitude, Sec. IV B)."""
    if smem == 1 and precision == 0 and m * n + n * n > 8192:
        pytest.skip("does not fit shared memory in complex128")
    rng = np.random.default_rng(7 * m + n)
    a = rand(rng, m, n, decay=decay)
    dc = torch.tensor(a.T.copy(), dtype=CDT[precision], device="cuda")  # column-major
    dv = torch.zeros((n, n), dtype=CDT[precision], device="cuda")
    ds = torch.zeros(n, dtype=RDT[precision], device="cuda")
    stn.dense_svd(precision, m, n, dc.data_ptr(), dv.data_ptr(), ds.data_ptr(), smem)
    torch.cuda.synchronize()
    us = dc.cpu().numpy().T.astype(np.complex128)
    v = dv.cpu().numpy().T.astype(np.complex128)
    sig2 = ds.cpu().numpy().astype(np.float64)
    s_ref = np.linalg.svd(a, compute_uv=False)
    got = np.sort(np.sqrt(np.maximum(sig2, 0)))[::-1][: len(s_ref)]
    assert np.abs(got - s_ref).max() < TOL[precision] * 10 * s_ref[0]
    assert np.abs(v.conj().T @ v - np.eye(n)).max() < TOL[precision] * 10
    assert np.abs(a @ v - us).max() < TOL[precision] * 10 * s_ref[0]
    gram = us.conj().T @ us
    off = gram - np.diag(np.diag(gram))
    assert np.abs(off).max() < TOL[precision] * 10 * s_ref[0] ** 2


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,decay", [(40, 24, 0.3), (64, 128, 0.1), (200, 150, 0.05), (256, 512, 0.05),
                                       (512, 512, 0.03)])
def test_large_bond_svd(precision, m, n, decay):
    """The large-bond path of the truncation sweep (Householder R factor,
    then one-sided Jacobi on R^dag): singular values, and the truncation of
    A to its leading right singular vectors, on graded MPS-like spectra."""
    rng = np.random.default_rng(11 * m + n)
    a = rand(rng, m, n, decay=decay)
    dc = torch.tensor(a, dtype=CDT[precision], device="cuda")  # row-major
    dv = torch.zeros((n, n), dtype=CDT[precision], device="cuda")
    ds = torch.zeros(n, dtype=RDT[precision], device="cuda")
    stn.dense_svd(precision, m, n, dc.data_ptr(), dv.data_ptr(), ds.data_ptr(), 3)
    torch.cuda.synchronize()
    v = dv.cpu().numpy().T.astype(np.complex128)  # columns = right vectors
    sig2 = ds.cpu().numpy().astype(np.float64)
    k = min(m, n)
    assert np.all(sig2[k:] == 0)
    u_ref, s_ref, vh_ref = np.linalg.svd(a, full_matrices=False)
    order = np.argsort(-sig2)
    got = np.sqrt(np.maximum(sig2[order], 0))[:k]
    assert np.abs(got - s_ref).max() < TOL[precision] * 10 * s_ref[0]
    # the kept right vectors: orthonormal where sigma is well above rounding,
    # and A projected on the leading `keep` of them is the optimal truncation
    keep = max(1, int(np.sum(s_ref > 1e-3 * s_ref[0])))
    vk = v[:, order[:keep]]
    assert np.abs(vk.conj().T @ vk - np.eye(keep)).max() < TOL[precision] * 1e3
    best = (u_ref[:, :keep] * s_ref[:keep]) @ vh_ref[:keep]
    q, _ = np.linalg.qr(vk)  # the sweep re-orthonormalises the kept vectors
    err = np.abs(a @ q @ q.conj().T - best).max()
    assert err < TOL[precision] * 10 * s_ref[0], err


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n", [(2, 1), (4, 8), (8, 4), (16, 16), (64, 32), (33, 47), (40, 64), (128, 64),
                                 (512, 256)])
def test_explicit_q_factor(precision, m, n):
    """The gauge step's explicit-Q Householder QR: Q has orthonormal columns
    and Q R reproduces A."""
    rng = np.random.default_rng(3 * m + n)
    a = rand(rng, m, n, decay=0.2)
    k = min(m, n)
    db = torch.tensor(a, dtype=CDT[precision], device="cuda")
    dq = torch.zeros((m, k), dtype=CDT[precision], device="cuda")
    dw = torch.zeros((m, k), dtype=CDT[precision], device="cuda")
    stn.dense_qr_q(precision, m, n, db.data_ptr(), dq.data_ptr(), dw.data_ptr())
    torch.cuda.synchronize()
    r = db.cpu().numpy().astype(np.complex128)[:k]
    q = dq.cpu().numpy().astype(np.complex128)
    assert np.abs(q.conj().T @ q - np.eye(k)).max() < TOL[precision] * 10
    assert np.abs(q @ r - a).max() < TOL[precision] * 10 * np.abs(a).max()
