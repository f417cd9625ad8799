"""Writes quartic_pop_n30_objective.txt: the optimal value of the
unconstrained quartic POP with n = 30 (Gram 496 x 496, m = 46376; the
precision form's workload) from the FP64 oracle, solved to a 1e-7 residual.
Only the oracle runs here; the GPU tests compare the mixed-precision form's
objective with this value.  Run: python tests/golden/make_quartic_pop_n30_objective.py
(a few minutes on a CPU)."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from instances import workloads as W  # noqa: E402
from oracle import admm, conic  # noqa: E402


def main():
    prog = W.quartic_pop(30, 0)
    res = admm.solve(conic.build(prog), 1e-7, 40000, k_check=10)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "quartic_pop_n30_objective.txt")
    with open(out, "w") as f:
        f.write("# quartic_pop(30, seed 0): FP64 oracle, tol 1e-7, k_check 10\n")
        f.write(f"status {res.status}\niters {res.iters}\npobj {res.res['pobj']:.17g}\ndobj {res.res['dobj']:.17g}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
