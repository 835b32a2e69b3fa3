"""Logical-error-rate sweeps over distance and noise strength, the threshold
study of Sec. V (Fig. 4: Pauli noise alone, Pauli noise plus the
Pauli-twirled crosstalk of Eq. 6, and Pauli noise plus coherent crosstalk).

The Pauli and twirled points need no state simulation: every fault of those
models is a Pauli, a Pauli's effect on the detectors and the logical
observable does not depend on the other faults, and so a shot's syndrome is
the XOR of the signatures of the faults that fire (Pauli-frame sampling from
the fault model that decoder.build_fault_model derives).  The coherent points
run the GPU simulation (Simulator.sample_shots) and read the device's
detectors.  Every point is decoded by minimum-weight matching under the
twirled error model, as the paper decodes, and reported with its 95% Wilson
interval.  Host-side and off the timed path.
"""

from dataclasses import dataclass

import numpy as np

from . import compile_program
from .decoder import MatchingDecoder, build_fault_model, wilson_interval


@dataclass
class SweepPoint:
    distance: int
    p: float
    theta: float
    noise: str     # "pauli", "pta" or "coherent"
    shots: int
    failures: int
    ler: float
    lo: float      # 95% Wilson interval
    hi: float


def frame_sample(model, shots, rng, include=None):
    """Detector rows [shots, n_det] and logical flips [shots] of `shots`
    Pauli-frame samples of a FaultModel: fault f fires independently with
    probability model.prob[f] (only the faults where include is True, when
    given), and a shot's syndrome is the XOR of its faults' signatures."""
    prob = np.where(include, model.prob, 0.0) if include is not None else model.prob
    det = np.zeros((shots, model.det.shape[1]), dtype=np.uint8)
    obs = np.zeros(shots, dtype=np.uint8)
    chunk = max(1, 2_000_000 // max(1, len(prob)))
    # counts of firing faults per detector are small integers, exact in FP32
    d32, o32 = model.det.astype(np.float32), model.obs.astype(np.float32)
    for s0 in range(0, shots, chunk):
        n = min(chunk, shots - s0)
        fire = (rng.random((n, len(prob))) < prob).astype(np.float32)
        det[s0:s0 + n] = (fire @ d32).astype(np.int64) & 1
        obs[s0:s0 + n] = (fire @ o32).astype(np.int64) & 1
    return det, obs


def _pair_count(workload):
    return int(compile_program(workload)[2].shape[0])


def sweep(workload, distances, ps, shots, noise="pta", theta=None, seed=0, simulate=None, angles=None,
          rounds_equal_distance=True):
    """LER points over distances x physical error rates ps for one noise
    model.  workload (a Workload-like object with .with_()) supplies
    everything else (rounds, schedule, pair rule, Table I scales); theta
    defaults to the workload's, and angles(w, n_pairs) gives the per-pair
    table (default: theta on every pair); with rounds_equal_distance each
    distance d runs d rounds, as memory experiments are usually sized.
    noise:
      "pauli": the Table I Pauli noise alone (the crosstalk faults are off);
      "pta": Pauli noise plus each rotation's Pauli with probability
             sin^2 theta (Eq. 6), frame-sampled;
      "coherent": the full simulation; simulate(w, shots, theta_table) must
             return (det [shots, n_det], obs [shots]) from the device, e.g.
             coherent_sampler(max_shots).
    The decoder is always matching under the twirled model (Pauli noise plus
    the PTA crosstalk prior), as in the paper."""
    th = workload.theta if theta is None else float(theta)
    if angles is None:
        angles = lambda w, k: np.full(k, w.theta, dtype=np.float64)  # noqa: E731
    rng = np.random.default_rng(seed)
    out = []
    for d in distances:
        for p in ps:
            w = workload.with_(distance=int(d), p=float(p), theta=th)
            if rounds_equal_distance:
                w = w.with_(rounds=int(d))
            table = angles(w, _pair_count(w))
            model = build_fault_model(w, table)
            dec = MatchingDecoder(model)
            if noise == "pauli":
                det, obs = frame_sample(model, shots, rng, include=[k[0] != "rot" for k in model.kind])
            elif noise == "pta":
                det, obs = frame_sample(model, shots, rng)
            elif noise == "coherent":
                if simulate is None:
                    raise ValueError("coherent points need a simulate callable")
                det, obs = simulate(w, shots, table)
            else:
                raise ValueError(f"unknown noise model {noise!r}")
            k = int(np.sum(dec.predict(det) != np.asarray(obs, dtype=np.uint8)))
            lo, hi = wilson_interval(k, shots)
            out.append(SweepPoint(int(d), float(p), th, noise, int(shots), k, k / shots, lo, hi))
    return out


def coherent_sampler(max_shots, shot_offset=0):
    """simulate callable for sweep(noise="coherent"): runs the workload's
    shots on the GPU in batches of at most max_shots and returns the
    device's detector rows and logical parities."""
    from . import Simulator

    def run(w, shots, table):
        sim = Simulator(w, max_shots=min(max_shots, shots))
        dets, obss = [], []
        try:
            for s0 in range(0, shots, sim.max_shots):
                n = min(sim.max_shots, shots - s0)
                sim.sample_shots(n, shot_offset + s0, table, born=False, stats=False)
                det, obs = sim.read_detectors()
                dets.append(np.asarray(det)[:n])
                obss.append(np.asarray(obs)[:n])
        finally:
            sim.close()
        return np.concatenate(dets), np.concatenate(obss)

    return run


def crossing(points, d_small, d_large):
    """The physical error rate where the LER curves of two distances cross
    (log-linear interpolation between the last p where the larger distance
    does better and the first where it does worse), or None.  Points of one
    noise model and angle, sorted by p."""
    a = {pt.p: pt.ler for pt in points if pt.distance == d_small}
    b = {pt.p: pt.ler for pt in points if pt.distance == d_large}
    ps = sorted(set(a) & set(b))
    for p0, p1 in zip(ps, ps[1:]):
        g0, g1 = b[p0] - a[p0], b[p1] - a[p1]
        if g0 < 0 <= g1:
            t = -g0 / (g1 - g0)
            return float(np.exp(np.log(p0) + t * (np.log(p1) - np.log(p0))))
    return None
