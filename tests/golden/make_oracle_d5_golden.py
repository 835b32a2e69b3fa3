"""Writes the whole-shot oracle records of the d=5 benchmark workload.

  oracle_d5_records.txt        shots 0-3 of d5_r5_theta0.10_p1e-3_chi256_c64
                               (5 rounds, chi cap 256, the workload's cutoff)
  oracle_d5_records_cut1e-12.txt
                               shot 0 of the same workload with the oracle's
                               own complex128 cutoff and degeneracy tolerance
                               (1e-12), to state the total error of the
                               complex64 path against the untruncated-below-
                               1e-12 oracle

Each line: shot, record bits, then per measurement the realised Born
probability; a trailing comment line per shot gives log P, max chi, the
discarded weight and the near-threshold draws.  Only oracle/ and the seeded
inputs of workloads.py are used.  One shot is tens of minutes of one core, so
the shots run in parallel processes (spawned, one BLAS thread each).  Run from
the repository root:
    python tests/golden/make_oracle_d5_golden.py
"""

import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))

SHOTS = (0, 1, 2, 3)
TIGHT_SHOTS = (0,)
TIGHT_CUTOFF = 1e-12


def _one(args):
    shot, cutoff = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from oracle.shot import make_program, run_shot
    from workloads import D5_BENCH, theta_table

    w = D5_BENCH if cutoff is None else D5_BENCH.with_(svd_cutoff=cutoff, degeneracy_tol=cutoff)
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    t0 = time.time()
    res = run_shot(w, shot, theta, prog)
    dt = time.time() - t0
    print(f"shot {shot} cutoff {w.svd_cutoff:g}: {dt:.0f} s, max chi {res.max_chi}", file=sys.stderr, flush=True)
    line = f"{shot} {''.join(str(b) for b in res.record)} {' '.join(repr(p) for p in res.born)}\n"
    meta = (f"# shot {shot}: logp {res.logp!r} max_chi {res.max_chi} discarded {res.discarded!r} "
            f"near_draws {res.near_draws} oracle_seconds {dt:.0f}\n")
    return shot, cutoff, line, meta


def _write(path, title, rows):
    with open(path, "w") as f:
        f.write(f"# {title}: shot, record bits, then the realised Born probability of every measurement\n")
        f.write("# written by tests/golden/make_oracle_d5_golden.py from oracle/ only\n")
        for _, _, line, meta in sorted(rows, key=lambda r: r[0]):
            f.write(line)
            f.write(meta)


def main():
    jobs = [(s, None) for s in SHOTS] + [(s, TIGHT_CUTOFF) for s in TIGHT_SHOTS]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(jobs)) as pool:
        rows = pool.map(_one, jobs)
    sys.path.insert(0, ROOT)
    from workloads import D5_BENCH
    _write(os.path.join(HERE, "oracle_d5_records.txt"), D5_BENCH.name, [r for r in rows if r[1] is None])
    _write(os.path.join(HERE, "oracle_d5_records_cut1e-12.txt"),
           f"{D5_BENCH.name} at svd_cutoff = degeneracy_tol = {TIGHT_CUTOFF:g}",
           [r for r in rows if r[1] is not None])


if __name__ == "__main__":
    main()
