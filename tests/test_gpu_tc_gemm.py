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
