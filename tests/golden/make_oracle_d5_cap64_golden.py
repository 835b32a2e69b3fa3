"""Writes the whole-shot oracle records of the benchmark workload cut to two
rounds at chi cap 64 (tests/golden/oracle_d5_r2_cap64_records.txt): d = 5,
theta = 0.10, p = 1e-3, cutoff 5e-6, shots 0-3.  The bonds reach the cap in
round 1, so these shots exercise the large-bond SVD path and the large
contractions end to end.

Each line: shot, record bits, then per measurement the realised Born
probability; a trailing comment line per shot gives log P, max chi, the
discarded weight and the near-threshold draws.  Only oracle/ and the seeded
inputs of workloads.py are used; each shot runs in its own spawned process
with one BLAS thread.  Run from the repository root:
    python tests/golden/make_oracle_d5_cap64_golden.py
"""

import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
SHOTS = (0, 1, 2, 3)


def workload():
    sys.path.insert(0, ROOT)
    from workloads import D5_BENCH
    return D5_BENCH.with_(rounds=2, chi_cap=64, name="d5_r2_theta0.10_p1e-3_chi64_c64")


def _one(shot):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from oracle.shot import make_program, run_shot
    from workloads import theta_table

    w = workload()
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    t0 = time.time()
    res = run_shot(w, shot, theta, prog)
    dt = time.time() - t0
    line = f"{shot} {''.join(str(b) for b in res.record)} {' '.join(repr(p) for p in res.born)}\n"
    meta = (f"# shot {shot}: logp {res.logp!r} max_chi {res.max_chi} discarded {res.discarded!r} "
            f"near_draws {res.near_draws} oracle_seconds {dt:.0f}\n")
    return shot, line, meta


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(SHOTS)) as pool:
        rows = pool.map(_one, SHOTS)
    w = workload()
    with open(os.path.join(HERE, "oracle_d5_r2_cap64_records.txt"), "w") as f:
        f.write(f"# {w.name}: shot, record bits, then the realised Born probability of every measurement\n")
        f.write("# written by tests/golden/make_oracle_d5_cap64_golden.py from oracle/ only\n")
        for _, line, meta in sorted(rows):
            f.write(line)
            f.write(meta)


if __name__ == "__main__":
    main()
