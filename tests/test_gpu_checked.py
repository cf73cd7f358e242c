"""Memory-safety checks without compute-sanitizer.

1. pbcg_mat_check (every build) validates the uploaded layouts of the
   matrices the other tests use: clean.
2. The checked build (libpbcg_checked.so, device-side bounds checks in every
   kernel) runs small solves of every path -- passes (staged and streamed,
   both tile orders), the one-cluster loop, batched solves, a pool, a
   one-rank partition -- and its check word stays 0, with exact results
   bit-identical to the oracle.  Then one stored column is set out of range
   (still inside the vector's padded allocation, so even an unchecked read
   would stay in bounds): pbcg_mat_check names the entry, and a solve
   through the streamed passes records the bad column in the check word
   instead of reading it.

The checked library runs in a child process (PBCG_LIB selects it), so this
process keeps the ordinary build.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2404_13216_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_13216_gb300 import build
    build.build_library(checked=True)
    from paper_2404_13216_gb300 import pbcg
    c = pbcg.Context(0)
    yield c
    c.close()


def test_layouts_validate_clean(ctx):
    mats = [inputs.convdiff2d(64, 10.0), inputs.convdiff3d(24, 50.0),
            inputs.powerlaw(n=20000, mean_len=30, max_len=2000, seed=2), inputs.batched_convdiff(nsys=16, seed=4).A]
    for A in mats:
        M = ctx.upload_csr(A)
        assert ctx.mat_check(M) == 0
        M.free()
    enabled, word = ctx.check_word()
    assert not enabled and word == 0          # the ordinary build compiles no in-kernel checks


CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle
from paper_2404_13216_gb300 import comm as pcomm, inputs, pbcg
out = {}
ctx = pbcg.Context(0)
en, w = ctx.check_word(reset=True)
out["enabled"] = en

def same(a, b):
    return bool(np.array_equal(np.asarray(a).view(np.int64), np.asarray(b).view(np.int64)))

def exact_vs_oracle(A, alg, maxit, tol=1e-10):
    b = inputs.rhs_ones(A)
    ref = oracle.solve(A.row_ptr, A.col_idx, A.vals, b, tol=tol, maxit=maxit, alg=alg, mode=1, nthreads=8)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    r = ctx.solve(M, b, x, tol, maxit, alg, 1)
    ok = r.iters == ref.iters and same(ctx.history(), ref.history) and same(x, ref.x)
    return M, ok

oks = []
A3 = inputs.convdiff3d(24, 50.0)
ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 0)
for v in (pbcg.Variant(1, 0, 0, 0), pbcg.Variant(0, 0, 0, 0), pbcg.Variant(1, 2, 1, 0), pbcg.Variant(0, 1, 0, 0)):
    for alg in (0, 1):
        b = inputs.rhs_ones(A3)
        M = ctx.upload_csr(A3)
        ctx.set_variant(M, v)
        ref = oracle.solve(A3.row_ptr, A3.col_idx, A3.vals, b, tol=1e-10, maxit=300, alg=alg, mode=1, nthreads=8)
        x = np.zeros(A3.n)
        r = ctx.solve(M, b, x, 1e-10, 300, alg, 1)
        oks.append(r.iters == ref.iters and same(ctx.history(), ref.history) and same(x, ref.x))
        M.free()
ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 1)
M, ok = exact_vs_oracle(inputs.convdiff2d(40, 25.0), 1, 800)     # one cluster launch
oks.append(ok); M.free()
M, ok = exact_vs_oracle(inputs.powerlaw(n=6000, mean_len=20, max_len=300, seed=7), 1, 40)
oks.append(ok); M.free()
ctx.set_option(pbcg.OPT_RR_PERIOD, 20)
A2 = inputs.convdiff2d(48, 30.0)
b2 = inputs.rhs_ones(A2)
M = ctx.upload_csr(A2)
x = np.zeros(A2.n)
r = ctx.solve(M, b2, x, 1e-10, 600, pbcg.PIPELINED_RR, 1)
ref = oracle.solve(A2.row_ptr, A2.col_idx, A2.vals, b2, tol=1e-10, maxit=600, alg=1, mode=1, nthreads=8, rr_period=20)
oks.append(r.iters == ref.iters and same(x, ref.x)); M.free()
B = inputs.batched_convdiff(nsys=16, seed=4)
M = ctx.upload_csr(B.A)
x = np.zeros(B.A.n)
res = ctx.solve_batched(M, B.sys_row_ptr, inputs.rhs_ones(B.A), x, np.full(16, 1e-10), 400, 1, 1)
out["batched_iters"] = [q.iters for q in res]
M.free()
with pbcg.Pool(ctx, 1 << 16, 1 << 19, 8, 500, 1, 1) as P:
    slots = [P.admit(inputs.convdiff2d(s, 12.0), inputs.rhs_ones(inputs.convdiff2d(s, 12.0)), tol=1e-10, maxit=500)
             for s in (20, 33, 47)]
    done = set()
    while len(done) < 3:
        P.step(8)
        d, _ = P.poll(wait=True)
        done.update(d)
    for s in slots:
        P.result(s)
A = inputs.convdiff3d(16, 40.0)
part = pbcg.Partition(ctx, pcomm.LocalComm(), np.array([0, A.n], np.int32), A.row_ptr, A.col_idx, A.vals)
xp = np.zeros(A.n)
rp = part.solve(inputs.rhs_ones(A), xp, 1e-10, 300, 1, 1)
part.close()
ref = oracle.solve(A.row_ptr, A.col_idx, A.vals, inputs.rhs_ones(A), tol=1e-10, maxit=300, alg=1, mode=1, nthreads=8)
oks.append(rp.iters == ref.iters and same(xp, ref.x))
out["exact_ok"] = oks
en, w = ctx.check_word(reset=True)
out["word_clean"] = w
# a stored column set out of range (n + 7: still inside the padded vector)
A = inputs.convdiff2d(40, 25.0)                      # n = 1600, vectors padded to 1792 rows
M = ctx.upload_csr(A)
ctx.debug_set_col(M, 100, A.n + 7)
out["mat_check"] = ctx.mat_check(M)
ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 0)
ctx.set_variant(M, pbcg.Variant(0, 0, 0, 0))        # streamed entries: the pass reads the stored column
x = np.zeros(A.n)
ctx.solve(M, inputs.rhs_ones(A), x, 1e-300, 3, 1, 1)
en, w = ctx.check_word(reset=True)
out["word_bad"] = w
M.free()
ctx.close()
print("RESULT " + json.dumps(out))
'''


def test_checked_build_runs_clean_and_catches_a_bad_column(ctx):
    lib = os.path.join(ROOT, "paper_2404_13216_gb300", "_build", "libpbcg_checked.so")
    env = dict(os.environ, PBCG_LIB=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    line = [s for s in r.stdout.splitlines() if s.startswith("RESULT ")][-1]
    out = json.loads(line[7:])
    assert out["enabled"] is True
    assert all(out["exact_ok"]), out["exact_ok"]
    assert out["word_clean"] == 0, hex(out["word_clean"])
    assert out["mat_check"] >> 56 == 1                            # a column
    assert out["word_bad"] >> 56 == 1 and out["word_bad"] & ((1 << 56) - 1) == 1607, hex(out["word_bad"])
