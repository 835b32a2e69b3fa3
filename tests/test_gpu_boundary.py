"""The boundary's problem statement and failure paths on the GPU, through the
C ABI: explicit crosstalk pairs equal to the default rule give the default
run bit for bit; X-memory and a caller's CNOT schedule match the oracle;
an arena too small for a sweep and a non-finite angle come back as statuses,
and the context stays usable."""

import numpy as np
import pytest

import paper_2605_29514_gb300 as stn
from oracle.circuit import build_layout, build_pairs, detectors, logical_z
from oracle.shot import make_program, run_shot
from test_gpu_parity import compare_shot, gpu_run
from test_oracle_shot import transposed_schedule
from workloads import D3_EXACT, theta_table

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stn.build()


def test_explicit_default_pairs_reproduce_records_bit_for_bit():
    rule = build_pairs(build_layout(3), "adjacent_idle")
    w = D3_EXACT.with_(p=0.02, rounds=2)
    shots = 8
    _, base, theta = gpu_run(w, shots)
    for masks in (True, False):
        we = w.with_(pairs=tuple((p.a, p.b, p.pauli, p.layer_mask if masks else None) for p in rule))
        _, out, _ = gpu_run(we, shots, theta=theta)
        assert np.array_equal(out["records"], base["records"])
        assert np.array_equal(out["born"], base["born"])


@pytest.mark.parametrize("variant", ["x_memory", "schedule_pairs_x_memory"])
def test_problem_statement_parity(variant):
    """X-memory (data prepared and read out in X), alone and with the
    transposed CNOT schedule and explicit pairs (a subset with the idle rule
    plus one XX pair on fixed layers): records, Born probabilities (1e-11),
    tableaux, and the device's detectors and X_L against the oracle."""
    w = D3_EXACT.with_(rounds=2, p=0.02, memory_basis="X")
    if variant == "schedule_pairs_x_memory":
        lay = build_layout(3)
        rule = build_pairs(lay, "adjacent_idle")
        pairs = tuple((p.a, p.b, p.pauli, None) for p in rule[::3]) + ((lay.data[0], lay.data[1], "XX", 0b0101),)
        w = w.with_(cnot_schedule=transposed_schedule(3), pairs=pairs)
    shots = 8
    sim, out, theta = gpu_run(w, shots)
    prog = make_program(w)
    det, obs = sim.read_detectors()
    for s in range(shots):
        ref = run_shot(w, s, theta, prog)
        assert compare_shot(sim, out, s, ref, 1e-11)
        rec = list(out["bits"][s])
        assert list(det[s]) == detectors(prog, rec)
        assert int(obs[s]) == logical_z(prog, rec)


def test_arena_cap_overflow_is_reported():
    """A per-shot span arena capped below what a sweep needs stops the shots
    with STN_EOVERFLOW through stn_sample_shots; the same context then runs a
    batch that fits (theta = 0 keeps every bond at 1)."""
    w = D3_EXACT.with_(rounds=1)
    sim = stn.Simulator(w, max_shots=4, arena_cap_bytes=8192)
    theta = theta_table(w, sim.n_pairs)
    with pytest.raises(stn.StnError) as e:
        sim.sample_shots(4, 0, theta)
    assert e.value.status == stn.STN_EOVERFLOW
    out = sim.sample_shots(4, 0, np.zeros_like(theta))
    assert np.all(out["max_chi"] == 1)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_theta_rejected(bad):
    w = D3_EXACT.with_(rounds=1)
    sim = stn.Simulator(w, max_shots=2)
    theta = theta_table(w, sim.n_pairs)
    theta[3] = bad
    with pytest.raises(stn.StnError) as e:
        sim.sample_shots(2, 0, theta)
    assert e.value.status == stn.STN_EINVAL
    theta[3] = 0.05
    out = sim.sample_shots(2, 0, theta)
    ref = run_shot(w, 1, theta)
    assert list(out["bits"][1]) == ref.record


def test_layer_steps_equal_rounds():
    """Running the 4 x rounds layer steps in order gives the same records,
    Born probabilities and statistics as running the round segments."""
    w = D3_EXACT.with_(p=0.02)
    shots = 6
    _, base, theta = gpu_run(w, shots)
    sim = stn.Simulator(w, max_shots=shots)
    assert sim.n_steps == 4 * w.rounds
    d_theta = torch.tensor(theta, dtype=torch.float64, device="cuda")
    sim.begin_batch(shots, 0)
    for s in range(sim.n_steps):
        sim.apply_step_device(s, d_theta.data_ptr())
    out = sim.read_records()
    for key in ("records", "born", "max_chi", "logp", "discarded"):
        assert np.array_equal(out[key], base[key]), key


def test_captured_batch_replays_equal_plain_batches():
    """A batch captured once as a CUDA graph and replayed for two shot
    offsets gives the records and Born probabilities of plain batches."""
    w = D3_EXACT.with_(p=0.02, rounds=2)
    shots = 5
    stream = torch.cuda.Stream()
    sim = stn.Simulator(w, max_shots=shots, stream=stream.cuda_stream)
    theta = theta_table(w, sim.n_pairs)
    d_theta = torch.tensor(theta, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    sim.capture_batch(shots, d_theta.data_ptr())
    for offset in (0, 1000):
        sim.launch_captured(offset)
        got = sim.read_records()
        _, ref, _ = gpu_run(w, shots, offset, theta)
        assert np.array_equal(got["records"], ref["records"])
        assert np.array_equal(got["born"], ref["born"])


def test_shot_queue_matches_small_batches():
    """A batch of more shots than the grid has CTAs (one per SM; the round
    kernel then takes the shots from a queue in the order CTAs finish) gives
    the records and Born probabilities of the same global shots run in small
    batches: each shot's randomness is keyed by its global index."""
    w = D3_EXACT.with_(p=0.02, rounds=1)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 2 * sms + 17
    sim = stn.Simulator(w, max_shots=n)
    theta = theta_table(w, sim.n_pairs)
    big = sim.sample_shots(n, 0, theta)
    sim.close()
    small = stn.Simulator(w, max_shots=64)
    recs, born = [], []
    for off in range(0, n, 64):
        k = min(64, n - off)
        out = small.sample_shots(k, off, theta)
        recs.append(out["records"][:k])
        born.append(out["born"][:k])
    small.close()
    assert np.array_equal(big["records"], np.concatenate(recs))
    assert np.array_equal(big["born"], np.concatenate(born))
