"""CPU pins of the host decoder (paper_2605_29514_gb300.decoder): the PTA
fault signatures it derives by Pauli-frame propagation through the compiled
program equal what the oracle's full simulation records when that Pauli is
actually applied (a rotation by theta = pi/2 is exp(-i pi/2 P) = -i P, a
Pauli); the lookup table decodes the fault-free syndrome as no flip and most
single faults correctly at d = 3; the Wilson interval has its textbook
values."""

import math

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from paper_2605_29514_gb300.decoder import LookupDecoder, build_fault_model, wilson_interval
from oracle.circuit import detectors, logical_z
from oracle.shot import make_program, run_shot
from workloads import D3_EXACT, D5_BENCH, theta_table


@pytest.fixture(scope="module", autouse=True)
def lib():
    stn.build()


@pytest.mark.parametrize("rule,pair", [("adjacent_idle", 0), ("adjacent_idle", 7), ("adjacent_idle", 23),
                                       ("adjacent_idle+diag_xx", 30)])
def test_fault_signatures_match_oracle_with_applied_paulis(rule, pair):
    """theta = pi/2 on one pair and 0 elsewhere applies that pair's Pauli at
    each of its occurrences: the oracle's detectors and logical parity equal
    the XOR of the model's signatures of those occurrences."""
    w = D3_EXACT.with_(rounds=2, p=0.0, pair_rule=rule)
    prog = make_program(w)
    theta = np.zeros(len(prog.pairs))
    theta[pair] = math.pi / 2
    model = build_fault_model(w, theta)
    rows = [f for f, k in enumerate(model.kind) if k[0] == "rot" and k[2] == pair]
    assert len(rows) == 2 * bin(prog.pairs[pair].layer_mask).count("1")
    want_det = np.bitwise_xor.reduce(model.det[rows], axis=0)
    want_obs = int(np.bitwise_xor.reduce(model.obs[rows]))
    for shot in range(3):
        r = run_shot(w, shot, theta, prog)
        assert detectors(prog, r.record) == list(want_det.astype(int))
        assert logical_z(prog, r.record) == want_obs


def test_record_flip_faults_flip_their_detectors():
    """A flipped record (Table I, pM) flips exactly the detectors that read
    that record, and the logical parity when the record is one of its
    readouts."""
    w = D3_EXACT.with_(rounds=2, p=0.01, theta=0.0)
    model = build_fault_model(w, np.zeros(24))
    det_table, logical = stn.compile_detectors(w)
    recs = [k for k in model.kind if k[0] == "noise" and k[2] == "record"]
    assert len(recs) == w.n_meas
    for f, k in enumerate(model.kind):
        if k[0] == "noise" and k[2] == "record":
            ops = stn.compile_program(w)[1]
            rec = int(ops[k[1], 5])
            expect = np.any(det_table == rec, axis=1)
            assert np.array_equal(model.det[f], expect)
            assert bool(model.obs[f]) == bool(rec in set(logical.tolist()))


def test_lookup_decoder_on_single_faults():
    w = D3_EXACT
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    model = build_fault_model(w, theta)
    dec = LookupDecoder(model)
    assert dec.predict(np.zeros((1, model.det.shape[1]), dtype=np.uint8))[0] == 0
    pred = dec.predict(model.det.astype(np.uint8))
    ok = np.mean(pred == model.obs.astype(np.uint8))
    assert ok > 0.9, ok
    assert dec.unseen == 0


def test_wilson_interval():
    lo, hi = wilson_interval(0, 100)
    assert lo == 0.0 and abs(hi - 0.03699) < 1e-4
    lo, hi = wilson_interval(50, 100)
    assert abs(lo - 0.40383) < 1e-4 and abs(hi - 0.59617) < 1e-4


def test_eq1_estimate_reduces_to_failure_rate_for_pauli_errors():
    from paper_2605_29514_gb300.decoder import eq1_estimate
    e = np.array([1.0, -1.0, 1.0, -1.0])
    c = np.array([0, 1, 1, 0])
    assert eq1_estimate(e, c) == 0.5  # shots 2 and 3 fail
    assert abs(eq1_estimate([np.cos(0.4)], [0]) - np.sin(0.2)) < 1e-15


def _graphlike(model):
    return [f for f in range(len(model.prob)) if 1 <= int(model.det[f].sum()) <= 2]


@pytest.mark.parametrize("uniform", [True, False])
@pytest.mark.parametrize("w", [D3_EXACT.with_(p=1e-3), D5_BENCH], ids=["d3", "d5"])
def test_matching_corrects_every_single_fault(w, uniform):
    """Minimum-weight matching on the PTA-plus-Pauli detector graph decodes
    every single fault that flips one or two detectors to its own logical
    effect: at distance d >= 3 any other explanation with a different
    logical effect needs at least d - 1 >= 2 edges.  Also the empty syndrome
    decodes to no flip."""
    from paper_2605_29514_gb300.decoder import MatchingDecoder
    theta = theta_table(w, stn.compile_program(w)[2].shape[0])
    model = build_fault_model(w, theta)
    dec = MatchingDecoder(model, uniform=uniform)
    g = _graphlike(model)
    assert len(g) > 0.5 * len(model.prob)
    assert np.array_equal(dec.predict(model.det[g]), model.obs[g].astype(np.uint8))
    assert dec.predict(np.zeros((1, model.det.shape[1]), dtype=bool))[0] == 0
    assert dec.unmatched == 0


@pytest.mark.parametrize("dp_limit", [12, 0])
def test_matching_corrects_fault_pairs_at_distance_5(dp_limit):
    """At d = 5 every pair of graph-like faults is corrected with unit
    weights (another explanation with a different logical effect needs at
    least 5 - 2 = 3 edges), through the subset dynamic program and, with
    dp_limit = 0, through the blossom matching; 2,000 seeded pairs."""
    from paper_2605_29514_gb300.decoder import MatchingDecoder
    if dp_limit == 0:
        pytest.importorskip("networkx")
    w = D5_BENCH
    theta = theta_table(w, stn.compile_program(w)[2].shape[0])
    model = build_fault_model(w, theta)
    dec = MatchingDecoder(model, uniform=True, dp_limit=dp_limit)
    g = np.array(_graphlike(model))
    rng = np.random.default_rng(5)
    pairs = rng.choice(g, size=(2000, 2))
    det = model.det[pairs[:, 0]] ^ model.det[pairs[:, 1]]
    obs = model.obs[pairs[:, 0]] ^ model.obs[pairs[:, 1]]
    assert np.array_equal(dec.predict(det), obs.astype(np.uint8))


def test_matching_and_lookup_rates_agree_on_sampled_faults():
    """On 3,000 syndromes sampled from the d = 3 fault model itself (each
    fault fires independently with its probability), the matching decoder's
    failure rate and the lookup table's lie in each other's 95% Wilson
    intervals."""
    from paper_2605_29514_gb300.decoder import MatchingDecoder
    w = D3_EXACT.with_(p=1e-3)
    theta = theta_table(w, stn.compile_program(w)[2].shape[0])
    model = build_fault_model(w, theta)
    rng = np.random.default_rng(1)
    fire = (rng.random((3000, len(model.prob))) < model.prob).astype(np.uint8)
    det = (fire @ model.det.astype(np.uint8)) % 2
    obs = (fire @ model.obs.astype(np.uint8)) % 2
    n = len(obs)
    k_m = int(np.sum(MatchingDecoder(model).predict(det) != obs))
    k_l = int(np.sum(LookupDecoder(model).predict(det) != obs))
    lo_m, hi_m = wilson_interval(k_m, n)
    lo_l, hi_l = wilson_interval(k_l, n)
    assert lo_m <= k_l / n <= hi_m and lo_l <= k_m / n <= hi_l, (k_m, k_l)
