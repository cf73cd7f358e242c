"""The oracle reproduces its committed fixture (written by tests/golden/make_golden.py)."""
import hashlib
import json
import os

import numpy as np

from paper_2404_13216_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "convdiff64.json")


def test_oracle_matches_fixture(orc):
    g = json.load(open(GOLDEN))
    A = inputs.convdiff2d(64, 10.0, (1.0, 0.5))
    b = inputs.rhs_ones(A)
    for alg, an in ((0, "bicgstab"), (1, "pbicgstab")):
        for mode, mn in ((0, "plain"), (1, "exact")):
            want = g["runs"][f"{an}_{mn}"]
            r = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-8, maxit=2000, alg=alg, mode=mode)
            assert r.status == want["status"] and r.iters == want["iters"]
            assert np.array_equal(r.history, np.array([float.fromhex(h) for h in want["history"]]))
            assert hashlib.sha256(r.x.tobytes()).hexdigest() == want["x_sha256"]
