"""Writes oracle_d3_1000_records.txt: the records of shots 0-999 of the d=3,
3-round, theta = 0.05 workload (complex128, chi cap 64, no Pauli noise, seed
0), from the oracle alone, for the logical-error-rate comparison.  One line
per shot: shot index, the 33 record bits, the number of Born draws within
1e-5 of their threshold.  Run from the repository root:
    python tests/golden/make_oracle_d3_ler_golden.py
"""

import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
SHOTS = 1000


def _chunk(args):
    lo, hi = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from oracle.shot import make_program, run_shot
    from workloads import D3_EXACT, theta_table
    prog = make_program(D3_EXACT)
    theta = theta_table(D3_EXACT, len(prog.pairs))
    out = []
    for s in range(lo, hi):
        r = run_shot(D3_EXACT, s, theta, prog)
        out.append(f"{s} {''.join(str(b) for b in r.record)} {r.near_draws}\n")
    return out


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    step = (SHOTS + workers - 1) // workers
    jobs = [(lo, min(SHOTS, lo + step)) for lo in range(0, SHOTS, step)]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        parts = pool.map(_chunk, jobs)
    sys.path.insert(0, ROOT)
    from workloads import D3_EXACT
    with open(os.path.join(HERE, "oracle_d3_1000_records.txt"), "w") as f:
        f.write(f"# {D3_EXACT.name}: shot, record bits, near-threshold Born draws\n")
        f.write("# written by tests/golden/make_oracle_d3_ler_golden.py from oracle/ only\n")
        for part in parts:
            f.writelines(part)


if __name__ == "__main__":
    main()
