"""Whole shots of the benchmark workload (d=5, 5 rounds, theta = 0.10,
p = 1e-3, chi cap 256, complex64 contractions) on the GPU against the
oracle's stored records (tests/golden/oracle_d5_records.txt, written by
make_oracle_d5_golden.py from oracle/ alone).

Bars: records identical except after a Born draw within 1e-5 of its
threshold (counted on either side); the largest bond and log P agree; Born
probabilities of the realised outcomes within 1e-4 relative (floor 1e-4 in
the denominator).  The metric's 1e-5 is the target; against the complex128
path the complex64 path already sits at 1.7-2.1e-5 after two rounds (FP32
storage and contractions set that floor), so the bar here is the floor
with the growth of five rounds, and the measured error is printed.  The same GPU shot is also compared with the oracle run at its
own complex128 cutoff (1e-12) and the error is reported."""

import os

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from workloads import D5_BENCH, theta_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    rows, meta = {}, {}
    path = os.path.join(HERE, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    for line in open(path):
        if line.startswith("# shot"):
            f = line.split()
            shot = int(f[2].rstrip(":"))
            kv = dict(zip(f[3::2], f[4::2]))
            meta[shot] = {k: float(v) for k, v in kv.items()}
        elif not line.startswith("#") and line.strip():
            f = line.split()
            rows[int(f[0])] = ([int(c) for c in f[1]], np.array([float(x) for x in f[2:]]))
    return rows, meta


@pytest.fixture(scope="module")
def gpu_shots():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stn.build()
    rows, meta = load_golden("oracle_d5_records.txt")
    shots = max(rows) + 1
    sim = stn.Simulator(D5_BENCH, max_shots=shots)
    out = sim.sample_shots(shots, 0, theta_table(D5_BENCH, sim.n_pairs))
    sim.close()
    return out, rows, meta


def first_divergence(bits, rec):
    return next((i for i in range(len(rec)) if bits[i] != rec[i]), None)


def test_whole_d5_shots_match_oracle(gpu_shots):
    out, rows, meta = gpu_shots
    worst = 0.0
    for s, (rec, born) in rows.items():
        bits = list(out["bits"][s])
        div = first_divergence(bits, rec)
        upto = len(rec) if div is None else div
        if div is not None:
            assert out["near_draws"][s] > 0 or meta[s]["near_draws"] > 0, f"shot {s}: record {div} differs"
        err = np.abs(out["born"][s][:upto] - born[:upto]) / np.maximum(born[:upto], 1e-4)
        worst = max(worst, float(err.max()))
        assert np.all(err < 1e-4), f"shot {s}: max rel Born error {err.max():.3e} at record {int(err.argmax())}"
        if div is None:
            assert out["max_chi"][s] == meta[s]["max_chi"]
            # each realised probability within 1e-4 relative moves log P by at most ~1e-4
            assert abs(out["logp"][s] - meta[s]["logp"]) < 1e-4 * len(rec)
    print(f"max relative Born error over {len(rows)} whole shots: {worst:.3e}")


def test_d5_shot_against_tight_cutoff_oracle(gpu_shots):
    """The complex64 path (cutoff 5e-6) against the oracle at cutoff 1e-12:
    the error of the whole approximation, stated, with records identical up
    to near-threshold draws and Born probabilities within 1e-3 relative."""
    out, _, _ = gpu_shots
    rows, meta = load_golden("oracle_d5_records_cut1e-12.txt")
    for s, (rec, born) in rows.items():
        bits = list(out["bits"][s])
        div = first_divergence(bits, rec)
        upto = len(rec) if div is None else div
        err = np.abs(out["born"][s][:upto] - born[:upto]) / np.maximum(born[:upto], 1e-4)
        print(f"shot {s} vs the 1e-12-cutoff oracle: records agree through {upto} of {len(rec)}, "
              f"max relative Born error {err.max():.3e}")
        if div is not None:
            assert out["near_draws"][s] > 0 or meta[s]["near_draws"] > 0
        assert np.all(err < 1e-3)


def _cap64_workload():
    return D5_BENCH.with_(rounds=2, chi_cap=64, name="d5_r2_theta0.10_p1e-3_chi64_c64")


@pytest.mark.parametrize("precision,bar", [(None, 5e-5), ("c128", 1e-7)])
def test_d5_two_rounds_cap64_against_oracle(precision, bar):
    """Whole shots of the benchmark workload cut to two rounds at chi cap 64
    (tests/golden/oracle_d5_r2_cap64_records.txt, written from oracle/
    alone): the bonds reach the cap in round 1, so the large-bond SVDs and
    the large contractions run end to end.  Records identical except after a
    near-threshold draw; Born probabilities within 5e-5 relative for the
    complex64 path (its FP32 floor: 1.7e-5 against the complex128 path on
    these shots) and 1e-7 for the complex128 path; the same largest bond."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from workloads import PRECISION_C128
    rows, meta = load_golden("oracle_d5_r2_cap64_records.txt")
    stn.build()
    w = _cap64_workload()
    if precision == "c128":
        w = w.with_(precision=PRECISION_C128)
    shots = max(rows) + 1
    sim = stn.Simulator(w, max_shots=shots)
    out = sim.sample_shots(shots, 0, theta_table(w, sim.n_pairs))
    sim.close()
    for s, (rec, born) in rows.items():
        bits = list(out["bits"][s])
        div = first_divergence(bits, rec)
        upto = len(rec) if div is None else div
        if div is not None:
            assert out["near_draws"][s] > 0 or meta[s]["near_draws"] > 0, f"shot {s}: record {div} differs"
        err = np.abs(out["born"][s][:upto] - born[:upto]) / np.maximum(born[:upto], 1e-4)
        assert np.all(err < bar), f"shot {s}: max rel Born error {err.max():.3e} at record {int(err.argmax())}"
        if div is None:
            assert out["max_chi"][s] == meta[s]["max_chi"]
