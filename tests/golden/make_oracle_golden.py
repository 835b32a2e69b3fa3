"""Writes oracle_d3_records.txt: records and realised Born probabilities of
shots 0-3 of the d=3, 3-round, theta = 0.05 workload (complex128, chi cap 64,
seed 0), from the oracle alone.  Run from the repository root:
    python tests/golden/make_oracle_golden.py
"""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.shot import make_program, run_shot  # noqa: E402
from workloads import D3_EXACT, theta_table  # noqa: E402

SHOTS = 4


def main():
    w = D3_EXACT
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_d3_records.txt")
    with open(path, "w") as f:
        f.write(f"# {w.name}: shot, record bits, then the realised Born probability of every measurement\n")
        f.write("# written by tests/golden/make_oracle_golden.py from oracle/ only\n")
        for s in range(SHOTS):
            res = run_shot(w, s, theta, prog)
            f.write(f"{s} {''.join(str(b) for b in res.record)} {' '.join(repr(p) for p in res.born)}\n")


if __name__ == "__main__":
    main()
