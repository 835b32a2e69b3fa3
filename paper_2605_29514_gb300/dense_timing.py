"""Single-CTA timings of the truncation sweep's dense routines through the C
ABI: the Householder R factor and the one-sided Jacobi SVD variants, at the
sizes the sweep meets, timed with CUDA events (mean of 5 runs after one
warm-up).  Prints one dict per case; with a path argument also writes them
as a JSON list.

    python -m paper_2605_29514_gb300.dense_timing [out.json]
"""

import json
import sys

import numpy as np

# (precision 0 = complex128 / 1 = complex64, stn_dense_svd mode, m, n)
SVD_CASES = [(0, 1, 32, 64), (0, 1, 64, 64), (0, 1, 60, 60), (1, 1, 64, 64), (1, 1, 100, 100),
             (1, 3, 128, 128), (1, 3, 256, 256), (1, 3, 512, 512), (0, 3, 128, 128), (1, 2, 128, 128)]
QR_CASES = [(1, 256, 128), (1, 1024, 512), (1, 512, 256), (0, 256, 128)]


def graded(m, n, decay=0.05, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    u, _, vh = np.linalg.svd(a, full_matrices=False)
    return (u * np.exp(-decay * np.arange(min(m, n)))) @ vh


def main():
    import torch

    import paper_2605_29514_gb300 as stn
    stn.build()
    cdt = {0: torch.complex128, 1: torch.complex64}
    rdt = {0: torch.float64, 1: torch.float32}

    def timeit(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = []
    for prec, mode, m, n in SVD_CASES:
        a = graded(m, n)
        src = torch.tensor(a if mode == 3 else a.T.copy(), dtype=cdt[prec], device="cuda")
        dc = src.clone()
        dv = torch.zeros((n, n), dtype=cdt[prec], device="cuda")
        ds = torch.zeros(n, dtype=rdt[prec], device="cuda")

        def svd():
            dc.copy_(src)
            stn.dense_svd(prec, m, n, dc.data_ptr(), dv.data_ptr(), ds.data_ptr(), mode)
        res.append({"what": "svd", "precision": prec, "mode": mode, "m": m, "n": n, "ms": timeit(svd)})
        print(res[-1], flush=True)
    for prec, m, n in QR_CASES:
        src = torch.tensor(graded(m, n), dtype=cdt[prec], device="cuda")
        d = src.clone()

        def qr():
            d.copy_(src)
            stn.dense_qr(prec, m, n, d.data_ptr())
        res.append({"what": "qr", "precision": prec, "m": m, "n": n, "ms": timeit(qr)})
        print(res[-1], flush=True)
    if len(sys.argv) > 1:
        json.dump(res, open(sys.argv[1], "w"), indent=1)


if __name__ == "__main__":
    main()
