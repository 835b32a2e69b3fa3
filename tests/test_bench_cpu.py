"""CPU checks of bench.py's host logic: the reference arm (the oracle on the
host cores) prints one well-formed JSON line, and the textbook FLOP counts
used to convert its sample into shots/s are the standard ones."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_textbook_counts():
    assert bench._gemm(2, 3, 4) == 8 * 24
    assert bench._qr(6, 3) == 4 * (2 * 6 * 9 - 2 * 27 / 3)
    assert bench._qr(3, 6) == bench._qr(6, 3)
    assert bench._svd(4, 2) == 4 * (4 * 4 * 4 + 8 * 8)
    assert bench._svd(2, 4) == bench._svd(4, 2)
    # one doubled bond of 4 kept at 2
    got = bench._sweep_flops(0, [4], [2])
    want = bench._qr(8, 4) + bench._gemm(4, 8, 4) + bench._gemm(4, 4, 4) + bench._svd(4, 4) \
        + bench._gemm(4, 2, 4) + bench._gemm(8, 2, 4)
    assert got == want


def test_reference_arm_prints_one_line():
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "2"], capture_output=True, text=True, timeout=600,
                       env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "shots/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_timed_plan_counts_only_complete_batches():
    plan, complete = bench.timed_plan(20, 6)
    assert len(plan) == 20 and complete == 3
    assert plan[0] == (0, 0) and plan[5] == (0, 5) and plan[6] == (1, 0) and plan[19] == (3, 1)
    plan, complete = bench.timed_plan(4, 6)
    assert complete == 0 and [g for _, g in plan] == [0, 1, 2, 3]
    plan, complete = bench.timed_plan(12, 6)
    assert complete == 2 and plan[-1] == (1, 5)
