"""Write tests/golden/convdiff64.json from the CPU oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
The fixture records, for the 2D convection-diffusion system on a 64x64 grid
(Peclet 10, wind (1, 0.5), b = A*ones, x0 = 0, tol 1e-8, maxit 2000), the
status, iteration count and residual history (as float.hex) of Algorithm 1 and
Algorithm 2 in plain and exact dot modes, plus a digest of the final x.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2404_13216_gb300 import inputs  # noqa: E402


def main():
    A = inputs.convdiff2d(64, 10.0, (1.0, 0.5))
    b = inputs.rhs_ones(A)
    out = {"system": "convdiff2d N=64 Pe=10 wind=(1,0.5) b=A*ones x0=0 tol=1e-8 maxit=2000", "runs": {}}
    for alg, an in ((0, "bicgstab"), (1, "pbicgstab")):
        for mode, mn in ((0, "plain"), (1, "exact")):
            r = oracle.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-8, maxit=2000, alg=alg, mode=mode)
            out["runs"][f"{an}_{mn}"] = {
                "status": r.status, "iters": r.iters,
                "history": [float(h).hex() for h in r.history],
                "x_sha256": hashlib.sha256(r.x.tobytes()).hexdigest(),
            }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "convdiff64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path)


if __name__ == "__main__":
    main()
