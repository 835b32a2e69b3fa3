"""Writes the oracle's records for the logical-error-rate comparison, from
the oracle alone:
  oracle_d3_1000_records.txt    shots 0-999 of the d=3, 3-round, theta = 0.05
                                workload (complex128, chi cap 64, no Pauli
                                noise, seed 0), a Z-memory;
  oracle_d3x_400_records.txt    shots 0-399 of the same workload as an
                                X-memory (the ZZ crosstalk's Z errors flip
                                X_L, so its logical error rate is not zero).
One line per shot: shot index, the 33 record bits, the number of Born draws
within 1e-5 of their threshold.  Run from the repository root:
    python tests/golden/make_oracle_d3_ler_golden.py [workers] [z|x]
"""

import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
SHOTS = 1000


def _workload(basis):
    from workloads import D3_EXACT
    return D3_EXACT if basis == "z" else D3_EXACT.with_(memory_basis="X", name=D3_EXACT.name + "_xmem")


def _chunk(args):
    lo, hi, basis = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from oracle.shot import make_program, run_shot
    from workloads import theta_table
    w = _workload(basis)
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    out = []
    for s in range(lo, hi):
        r = run_shot(w, s, theta, prog)
        out.append(f"{s} {''.join(str(b) for b in r.record)} {r.near_draws}\n")
    return out


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    basis = sys.argv[2] if len(sys.argv) > 2 else "z"
    shots = SHOTS if basis == "z" else 400
    step = (shots + workers - 1) // workers
    jobs = [(lo, min(shots, lo + step), basis) for lo in range(0, shots, step)]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        parts = pool.map(_chunk, jobs)
    sys.path.insert(0, ROOT)
    w = _workload(basis)
    name = "oracle_d3_1000_records.txt" if basis == "z" else "oracle_d3x_400_records.txt"
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {w.name}: shot, record bits, near-threshold Born draws\n")
        f.write("# written by tests/golden/make_oracle_d3_ler_golden.py from oracle/ only\n")
        for part in parts:
            f.writelines(part)


if __name__ == "__main__":
    main()
