"""Write tests/golden/oracle_iterations.txt: iteration counts and final true
relative residuals of the FP64 CPU oracle (oracle.solve, tol 1e-8) on the
full-size workloads.  Calls only the oracle and the seeded input generators.

Usage: python tests/golden/make_oracle_iterations.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main():
    rows = []
    cases = [("config0", W.config0()), ("config1", W.config1()), ("config2", W.config2())]
    s4, _ = W.config4()
    cases.append(("config4", s4))
    for name, s in cases:
        t = time.time()
        z, info = O.solve(s.faces, s.lam, s.f, tol=1e-8, maxit=1000)
        rows.append((name, info.iters, info.relres, time.time() - t))
        print(rows[-1], flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.txt")
    with open(out, "w") as fh:
        fh.write("# FP64 CPU oracle (oracle.solve, tol 1e-8, zero initial guess) on the full-size\n")
        fh.write("# workloads of workloads.config0/1/2/4; written by make_oracle_iterations.py.\n")
        fh.write("# Columns: workload iterations final_true_relres\n")
        for name, it, rr, _ in rows:
            fh.write(f"{name} {it} {rr:.6e}\n")


if __name__ == "__main__":
    main()
