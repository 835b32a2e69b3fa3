"""The tcgen05 tensor-core GEMM (stn_dense_gemm_tc) with the 3-term TF32
split against a float64 product: FP32-level accuracy, where a single TF32
product would be about 1e-3 off; tiles that are ragged in every dimension."""

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stn.build()


@pytest.mark.parametrize("m,n,k", [(128, 64, 8), (128, 64, 64), (100, 70, 37), (300, 150, 129), (1, 1, 1)])
def test_tensor_core_gemm_fp32_accuracy(m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a = rng.normal(size=(m, k)).astype(np.float32)
    b = rng.normal(size=(k, n)).astype(np.float32)
    da = torch.tensor(a, device="cuda")
    db = torch.tensor(b, device="cuda")
    dc = torch.full((m, n), np.nan, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stn.dense_gemm_tc(m, n, k, da.data_ptr(), db.data_ptr(), dc.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    c = dc.cpu().numpy().astype(np.float64)
    ref = a.astype(np.float64) @ b.astype(np.float64)
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64)
    err = np.abs(c - ref) / np.maximum(scale, 1e-30)
    assert np.all(np.isfinite(c))
    assert err.max() < 1e-5, err.max()


def _cmat(rng, r, c):
    return (rng.normal(size=(r, c)) + 1j * rng.normal(size=(r, c))).astype(np.complex64)


@pytest.mark.parametrize("units", [stn.GEMM_TENSOR, stn.GEMM_FMA])
@pytest.mark.parametrize("op_a,op_b", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(64, 32, 16), (128, 64, 32), (200, 96, 70), (256, 512, 256), (65, 33, 17),
                                   (10, 300, 40)])
def test_sweep_contraction_complex64(units, op_a, op_b, m, n, k):
    """The round kernel's complex contraction (stn_dense_cgemm, one CTA):
    C = alpha op(A) op(B) + beta C against a complex128 product, elementwise
    within 1e-5 of |op(A)| |op(B)| + |beta C|, for both contraction units,
    every op combination, tiles ragged in every dimension and a product
    below the tensor-core sizes (10 rows: CUDA cores either way)."""
    rng = np.random.default_rng(1000 * m + 10 * n + k + op_a * 7 + op_b * 3)
    a = _cmat(rng, *((k, m) if op_a else (m, k)))
    b = _cmat(rng, *((n, k) if op_b else (k, n)))
    c0 = _cmat(rng, m, n)
    alpha, beta = 0.7 - 0.2j, 0.3 + 0.5j
    da, db = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    dc = torch.tensor(c0, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stn.dense_cgemm(1, op_a, op_b, m, n, k, da.data_ptr(), a.shape[1], db.data_ptr(), b.shape[1],
                    dc.data_ptr(), n, st.data_ptr(), alpha=alpha, beta=beta, gemm_units=units)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    oa = a.astype(np.complex128).conj().T if op_a else a.astype(np.complex128)
    ob = b.astype(np.complex128).conj().T if op_b else b.astype(np.complex128)
    ref = alpha * (oa @ ob) + beta * c0.astype(np.complex128)
    scale = abs(alpha) * (np.abs(oa) @ np.abs(ob)) + abs(beta) * np.abs(c0)
    got = dc.cpu().numpy().astype(np.complex128)
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref) / scale
    assert err.max() < 1e-5, err.max()


@pytest.mark.parametrize("op_a,op_b", [(0, 0), (1, 1)])
def test_sweep_contraction_complex128(op_a, op_b):
    """The complex128 contraction (CUDA cores) to 1e-13."""
    m, n, k = 130, 70, 45
    rng = np.random.default_rng(17 + op_a)
    a = (rng.normal(size=(k, m) if op_a else (m, k)) + 1j * rng.normal(size=(k, m) if op_a else (m, k)))
    b = (rng.normal(size=(n, k) if op_b else (k, n)) + 1j * rng.normal(size=(n, k) if op_b else (k, n)))
    da, db = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    dc = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stn.dense_cgemm(0, op_a, op_b, m, n, k, da.data_ptr(), a.shape[1], db.data_ptr(), b.shape[1],
                    dc.data_ptr(), n, st.data_ptr())
    torch.cuda.synchronize()
    oa = a.conj().T if op_a else a
    ob = b.conj().T if op_b else b
    ref = oa @ ob
    err = np.abs(dc.cpu().numpy() - ref) / (np.abs(oa) @ np.abs(ob))
    assert err.max() < 1e-13, err.max()
