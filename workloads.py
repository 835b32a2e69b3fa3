"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module only holds parameters and seeded random inputs (per-pair angles);
it contains none of the simulation's arithmetic.

The paper (Sec. III, Table I, Sec. V) simulates rotated surface codes of
distance 3-9 for d rounds with depolarising noise scaled by gate type and a
coherent ZZ crosstalk angle theta.  It uses no dataset: every input here is
synthetic by construction.
"""

from dataclasses import dataclass, replace

import numpy as np

PRECISION_C128 = 0  # complex128 contractions, FP64 SVD
PRECISION_C64 = 1  # complex64 contractions, FP64 scalars and small-bond SVDs
PRECISION_C64_SVD64 = 2  # complex64 contractions, every bond SVD in FP64


@dataclass(frozen=True)
class Workload:
    name: str
    distance: int
    rounds: int
    theta: float  # crosstalk angle in rad (uniform, or mean when quenched)
    p: float  # depolarising base rate; Table I scales it per gate type
    chi_cap: int
    precision: int
    shots: int
    seed: int = 0
    p1_scale: float = 0.1
    p2_scale: float = 1.0
    pR_scale: float = 2.0
    pM_scale: float = 5.0
    # Schmidt values at or below svd_cutoff * s_1 are dropped; at a chi cap,
    # kept values must exceed the first dropped one by degeneracy_tol * s_1.
    # A dropped value changes Born probabilities by up to its amplitude, so
    # both sit well below the Born tolerance and well above the rounding
    # level of the arithmetic.
    svd_cutoff: float = 1e-12
    degeneracy_tol: float = 1e-12
    pair_rule: str = "adjacent_idle"
    theta_sigma: float = 0.0
    theta_seed: int = 7
    # Eq. 9's random-sign crosstalk: "fixed" keeps every angle's sign;
    # "random_pair" draws one sign per pair from theta_seed (quenched).
    theta_sign: str = "fixed"
    # Z or X memory; optional caller CNOT schedule (one 4-tuple of data
    # qubits or -1 per ancilla, ancillas in ascending qubit order) and
    # explicit crosstalk pairs ((a, b, 'ZZ' | 'XX', layer mask or None), in
    # place of pair_rule).
    memory_basis: str = "Z"
    cnot_schedule: tuple = None
    pairs: tuple = None

    def with_(self, **kw):
        return replace(self, **kw)

    @property
    def n_qubits(self):
        return 2 * self.distance * self.distance - 1

    @property
    def n_meas(self):
        d = self.distance
        return self.rounds * (d * d - 1) + d * d


def theta_table(w, n_pairs):
    """Per-pair angles: uniform, or quenched N(theta, theta_sigma^2) from
    theta_seed (independent of the shot seed); with theta_sign =
    "random_pair", each pair's angle then takes a sign drawn from
    theta_seed + 1."""
    if w.theta_sigma == 0.0:
        table = np.full(n_pairs, w.theta, dtype=np.float64)
    else:
        rng = np.random.default_rng(w.theta_seed)
        table = rng.normal(w.theta, w.theta_sigma, size=n_pairs).astype(np.float64)
    if w.theta_sign == "random_pair":
        signs = np.random.default_rng(w.theta_seed + 1).integers(0, 2, size=n_pairs) * 2 - 1
        table = table * signs
    elif w.theta_sign != "fixed":
        raise ValueError(f"unknown theta_sign {w.theta_sign!r}")
    return table


# d=3, 3 rounds, theta = 0.05 ZZ on idle adjacent pairs, no Pauli noise,
# chi cap 64, complex128, 1000 shots, seed 0.
D3_EXACT = Workload(
    name="d3_r3_theta0.05_chi64_c128",
    distance=3,
    rounds=3,
    theta=0.05,
    p=0.0,
    chi_cap=64,
    precision=PRECISION_C128,
    shots=1000,
    seed=0,
)

# d=5, 5 rounds, theta = 0.10 ZZ on idle adjacent pairs, depolarising p = 1e-3
# with the Table I ratios, chi cap 256, complex64 contractions, 16384 shots.
D5_BENCH = Workload(
    name="d5_r5_theta0.10_p1e-3_chi256_c64",
    distance=5,
    rounds=5,
    theta=0.10,
    p=1e-3,
    chi_cap=256,
    precision=PRECISION_C64,
    shots=16384,
    seed=0,
    svd_cutoff=5e-6,
    degeneracy_tol=5e-6,
)
