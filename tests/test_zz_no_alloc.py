"""The allocation-free SVD entry point (stn_dense_svd_noalloc), for callers
that cannot allocate device memory when they need the decomposition, checked
through the C ABI against the allocating-caller entry point (stn_dense_svd,
large-bond mode) on two calls in a row.  This file is collected last."""

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CDT = {0: torch.complex128, 1: torch.complex64}
RDT = {0: torch.float64, 1: torch.float32}
TOL = {0: 1e-12, 1: 2e-5}
# Within the 1 MiB scratch: shapes whose R^dag fits shared memory (complex128
# 64 x 64, complex64 16 x 64: the unblocked Jacobi), blocked shapes, and one
# request of exactly 1 MiB (complex128 256 x 256, complex64 512 x 256).
SIZES = {0: [(64, 64), (128, 256), (200, 96), (256, 256)], 1: [(16, 64), (256, 256), (300, 200), (512, 256)]}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stn.build()


def graded(rng, m, n):
    a = rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    u, _, vh = np.linalg.svd(a, full_matrices=False)
    return (u * np.exp(-0.04 * np.arange(min(m, n)))) @ vh


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_allocating_entry_point(precision):
    rng = np.random.default_rng(5 + precision)
    for m, n in SIZES[precision]:  # two calls in a row, different shapes and data
        a = graded(rng, m, n)
        dc = torch.tensor(a, dtype=CDT[precision], device="cuda")
        keep = dc.clone()
        v1 = torch.zeros((n, n), dtype=CDT[precision], device="cuda")
        s1 = torch.zeros(n, dtype=RDT[precision], device="cuda")
        stn.dense_svd_noalloc(precision, m, n, dc.data_ptr(), v1.data_ptr(), s1.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(dc, keep), "the input must be left unchanged"
        v2 = torch.zeros((n, n), dtype=CDT[precision], device="cuda")
        s2 = torch.zeros(n, dtype=RDT[precision], device="cuda")
        stn.dense_svd(precision, m, n, keep.data_ptr(), v2.data_ptr(), s2.data_ptr(), 3)
        torch.cuda.synchronize()
        g1 = s1.cpu().numpy().astype(np.float64)
        g2 = s2.cpu().numpy().astype(np.float64)
        smax = g2.max()
        assert np.abs(g1 - g2).max() <= TOL[precision] * smax
        # and both against LAPACK: the singular values of the input
        s_ref = np.linalg.svd(a, compute_uv=False)
        got = np.sort(np.sqrt(np.maximum(g1, 0)))[::-1][: len(s_ref)]
        assert np.abs(got - s_ref).max() <= TOL[precision] * 10 * s_ref[0]
        # right vectors of the well-separated leading values agree
        lead = np.argsort(-g2)[:16]
        x1 = v1.cpu().numpy().T.astype(np.complex128)[:, lead]
        x2 = v2.cpu().numpy().T.astype(np.complex128)[:, lead]
        assert np.abs(x1 - x2).max() <= TOL[precision] * 10


def test_noalloc_rejects_oversize():
    big = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(stn.StnError) as err:
        stn.dense_svd_noalloc(1, 1024, 256, big.data_ptr(), big.data_ptr(), big.data_ptr())
    assert err.value.status == 7  # STN_EOVERFLOW: beyond the 1 MiB scratch, nothing launched
    with pytest.raises(stn.StnError) as err:
        stn.dense_svd_noalloc(1, 1, 10000, big.data_ptr(), big.data_ptr(), big.data_ptr())
    assert err.value.status == 1  # STN_EINVAL: n beyond 512, nothing launched
