"""CPU pins of the threshold-sweep harness (paper_2605_29514_gb300.sweep):
Pauli-frame sampling from the fault model composes fault signatures by XOR
and fires each fault at its probability; below threshold the larger code
does better; the crossing interpolation is exact on straight lines; the
noiseless point has no failures."""

import dataclasses

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from paper_2605_29514_gb300.decoder import build_fault_model, wilson_interval
from paper_2605_29514_gb300.sweep import SweepPoint, crossing, frame_sample, sweep
from workloads import D3_EXACT, D5_BENCH


@pytest.fixture(scope="module", autouse=True)
def lib():
    stn.build()


@pytest.fixture(scope="module")
def model():
    w = D3_EXACT.with_(p=1e-3)
    k = stn.compile_program(w)[2].shape[0]
    return build_fault_model(w, np.full(k, w.theta))


def test_frame_sample_composes_signatures(model):
    """Two faults that always fire give every shot the XOR of their
    signatures; a third that never fires changes nothing."""
    rng = np.random.default_rng(0)
    f, g = 5, 400
    prob = np.zeros_like(model.prob)
    prob[[f, g]] = 1.0
    m = dataclasses.replace(model, prob=prob)
    det, obs = frame_sample(m, 50, rng)
    want = (model.det[f] ^ model.det[g]).astype(np.uint8)
    assert np.all(det == want) and np.all(obs == int(model.obs[f] ^ model.obs[g]))


def test_frame_sample_fires_at_the_fault_probability(model):
    """One fault at probability 0.25: the share of shots that show its
    signature lies in the 95% Wilson interval around 0.25 (4,000 shots)."""
    f = next(i for i in range(len(model.prob)) if model.det[i].any())
    prob = np.zeros_like(model.prob)
    prob[f] = 0.25
    det, _ = frame_sample(dataclasses.replace(model, prob=prob), 4000, np.random.default_rng(1))
    k = int(np.sum(np.all(det == model.det[f].astype(np.uint8), axis=1)))
    lo, hi = wilson_interval(k, 4000)
    assert lo <= 0.25 <= hi, k
    assert int(np.sum(det.any(axis=1))) == k  # every other shot is fault-free


def test_noiseless_point_has_no_failures():
    pts = sweep(D3_EXACT, [3], [0.0], 200, noise="pta", theta=0.0)
    assert pts[0].failures == 0 and pts[0].ler == 0.0


def test_larger_code_does_better_below_threshold():
    """Circuit-level Pauli noise of Table I at p = 2e-3 (below the ~0.6 %
    crossing these ratios give): d = 5 over 5 rounds fails significantly
    less often than d = 3 over 3 rounds under matching (disjoint 95%
    intervals, 10,000 shots each, fixed seed)."""
    pts = sweep(D5_BENCH, [3, 5], [2e-3], 10000, noise="pauli", theta=0.0, seed=3)
    d3, d5 = pts
    assert (d3.distance, d5.distance) == (3, 5)
    assert d5.hi < d3.lo, (d3, d5)


def test_crossing_interpolates_log_linearly():
    """Two straight lines in log p: d = 5 below d = 3 at p = 1e-3, above at
    1e-2, equal at sqrt(1e-3 * 1e-2) by construction."""
    def pt(d, p, ler):
        return SweepPoint(d, p, 0.0, "pauli", 1, 0, ler, 0.0, 1.0)
    pts = [pt(3, 1e-3, 0.02), pt(3, 1e-2, 0.2), pt(5, 1e-3, 0.01), pt(5, 1e-2, 0.21)]
    x = crossing(pts, 3, 5)
    # gaps -0.01 and +0.01: the zero is halfway in log p
    assert x == pytest.approx(np.sqrt(1e-3 * 1e-2), rel=1e-12)
    assert crossing(pts[:1] + pts[2:3], 3, 5) is None


def test_coherent_points_are_batched_through_the_simulator(monkeypatch, model):
    """The coherent sampler runs a point's shots through Simulator batches of
    at most max_shots, each at its own global shot offset, and concatenates
    the device's detector rows in order (a stand-in simulator that encodes
    the shot index in its detector row)."""
    import paper_2605_29514_gb300 as pkg
    from paper_2605_29514_gb300.sweep import coherent_sampler

    calls = []

    class FakeSim:
        def __init__(self, w, max_shots):
            self.max_shots = max_shots
            self.n_det = 8

        def sample_shots(self, n, offset, table, born=True, stats=True):
            calls.append((n, offset))
            self.cur = (n, offset)

        def read_detectors(self):
            n, off = self.cur
            idx = np.arange(off, off + n)
            det = ((idx[:, None] >> np.arange(8)) & 1).astype(np.uint8)
            return det, (idx & 1).astype(np.uint8)

        def close(self):
            pass

    monkeypatch.setattr(pkg, "Simulator", FakeSim)
    det, obs = coherent_sampler(max_shots=64, shot_offset=1000)(D3_EXACT, 150, np.zeros(3))
    assert calls == [(64, 1000), (64, 1064), (22, 1128)]
    idx = np.arange(1000, 1150)
    assert np.array_equal(det, ((idx[:, None] >> np.arange(8)) & 1).astype(np.uint8))
    assert np.array_equal(obs, (idx & 1).astype(np.uint8))
