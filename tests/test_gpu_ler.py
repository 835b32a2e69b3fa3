"""Logical error rate of the d=3 workload (3 rounds, theta = 0.05 ZZ on idle
adjacent pairs, no Pauli noise, chi cap 64, complex128, 1,000 shots, seed 0)
on the GPU against the oracle (tests/golden/oracle_d3_1000_records.txt,
written from oracle/ alone), both decoded by the lookup-table decoder built
from the Pauli-twirled error model (Sec. III C, Eq. 6; Sec. II, Eq. 1 reduces
to this sampled rate for Pauli errors).  The GPU's detectors and logical
parities come from the device; the two rates must lie in each other's 95%
Wilson intervals, and the records agree shot by shot except after a Born
draw within 1e-5 of its threshold."""

import os

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from paper_2605_29514_gb300.decoder import LookupDecoder, build_fault_model, logical_error_rate, wilson_interval
from workloads import D3_EXACT, theta_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name,basis", [("oracle_d3_1000_records.txt", "Z"), ("oracle_d3x_400_records.txt", "X")])
def test_d3_logical_error_rate_matches_oracle(name, basis):
    """Z-memory (the configuration: ZZ crosstalk makes only Z-type errors,
    which cannot flip Z_L, so its rate is zero on both sides) and the same
    circuit as an X-memory, where they flip X_L."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip("golden records not generated")
    stn.build()
    w = D3_EXACT.with_(memory_basis=basis)
    ref = {}
    for line in open(path):
        if line.startswith("#"):
            continue
        s, bits, near = line.split()
        ref[int(s)] = ([int(c) for c in bits], int(near))
    shots = len(ref)
    sim = stn.Simulator(w, max_shots=shots)
    theta = theta_table(w, sim.n_pairs)
    out = sim.sample_shots(shots, 0, theta)
    det, obs = sim.read_detectors()
    dec = LookupDecoder(build_fault_model(w, theta))
    ler_gpu, k_gpu = logical_error_rate(dec, det, obs)

    det_table, logical = stn.compile_detectors(w)
    recs = np.array([ref[s][0] for s in range(shots)], dtype=np.uint8)
    ext = np.concatenate([recs, np.zeros((shots, 1), dtype=np.uint8)], axis=1)
    det_ref = np.bitwise_xor.reduce(ext[:, det_table], axis=2)
    obs_ref = np.bitwise_xor.reduce(recs[:, logical], axis=1)
    ler_ref, k_ref = logical_error_rate(dec, det_ref, obs_ref)

    lo_g, hi_g = wilson_interval(k_gpu, shots)
    lo_r, hi_r = wilson_interval(k_ref, shots)
    assert lo_r <= ler_gpu <= hi_r and lo_g <= ler_ref <= hi_g, (ler_gpu, ler_ref)
    differ = [s for s in range(shots) if list(out["bits"][s]) != ref[s][0]]
    for s in differ:
        assert out["near_draws"][s] > 0 or ref[s][1] > 0, f"shot {s}: records differ"
    print(f"LER GPU {ler_gpu:.4f} ({k_gpu}/{shots}), oracle {ler_ref:.4f} ({k_ref}/{shots}); "
          f"{len(differ)} shots differ after near-threshold draws; unseen syndromes {dec.unseen}")
