"""Host logic of the serving loop, on the CPU: a fake pool with the admit /
step / poll / result contract of pbcg.Pool stands in for the GPU."""
import numpy as np

from paper_2404_13216_gb300 import inputs, serve


class FakeClock:
    def __init__(self, dt=2e-4):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakePool:
    """Slots and a row budget; a request needs ceil(n / 1000) iterations;
    poll reports what finished one step later (a step in flight)."""

    def __init__(self, slots, rows):
        self.slots, self.rows = slots, rows
        self.live = {}            # slot -> [n, need, done_iters, tol]
        self.used_rows = 0
        self.finished = []
        self.reported = set()
        self.in_flight = []       # per step: slots that finish in it
        self.steps = 0
        self.admitted = []

    def admit(self, A, b, x0=None, tol=1e-8, maxit=1000):
        n = A.n
        free = [s for s in range(self.slots) if s not in self.live]
        if not free or self.used_rows + n > self.rows:
            return None
        s = free[0]
        self.live[s] = [n, max(1, -(-n // 1000)), 0, tol]
        self.used_rows += n
        self.admitted.append(n)
        return s

    def step(self, K):
        assert len(self.in_flight) < 2, "more steps in flight than allowed"
        self.steps += 1
        fin = []
        for s, v in self.live.items():
            if v[2] < v[1] and s not in self.finished:
                v[2] = min(v[1], v[2] + K)
                if v[2] >= v[1]:
                    fin.append(s)
        self.in_flight.append(fin)

    def poll(self, wait=False):
        out = []
        if self.in_flight:
            fin = self.in_flight.pop(0)
            out = [s for s in fin if s in self.live]
            self.reported.update(out)
        return out, len(self.in_flight)

    def result(self, s):
        assert s in self.reported
        self.reported.discard(s)
        n, need, done, tol = self.live.pop(s)
        self.used_rows -= n
        return np.ones(n), type("R", (), dict(status=0, iters=done, relres_true=tol / 2))()


def test_serving_loop_finishes_every_request_in_order():
    reqs = inputs.serving_requests(count=60, rate=5000.0, n_lo=500, n_hi=8000, seed=3)
    templates = [serve.Template(inputs.CSR(r.n, None, None, None), None, r.n, 0, 0, r.dim, r.side, r.peclet)
                 for r in reqs[:10]]
    pools = {True: FakePool(4, 20000), False: FakePool(3, 15000)}
    out = serve.serve(reqs, templates, pools, K=4, clock=FakeClock())
    assert np.all(out["status"] == 0)
    assert np.all(out["latency"] > 0)
    for m, p in pools.items():
        # FIFO admission within a mode: admitted sizes follow arrival order
        want = [templates[i % len(templates)].n for i, r in enumerate(reqs) if r.exact == m]
        assert p.admitted == want
        assert p.live == {} and p.used_rows == 0
    s = serve.summarize(reqs, templates, out, 5000.0)
    assert s["finished"] == 60 and s["converged"] == 60 and s["p99_ms"] >= s["p50_ms"]


def test_serving_loop_waits_for_room():
    """A pool with room for one request at a time still serves them all."""
    reqs = inputs.serving_requests(count=12, rate=1e5, n_lo=900, n_hi=1000, seed=4)
    templates = [serve.Template(inputs.CSR(r.n, None, None, None), None, r.n, 0, 0, r.dim, r.side, r.peclet)
                 for r in reqs]
    pools = {True: FakePool(1, 1024), False: FakePool(1, 1024)}
    out = serve.serve(reqs, templates, pools, K=1, clock=FakeClock())
    assert np.all(out["status"] == 0)
    # one at a time: completion order equals arrival order within each mode
    for m in (True, False):
        idx = [i for i, r in enumerate(reqs) if r.exact == m]
        done_at = out["latency"][idx] + np.array([reqs[i].arrival for i in idx])
        assert np.all(np.diff(done_at) > 0)


def test_sell_entries_counts_slice_widths():
    from paper_2404_13216_gb300 import build
    build.build_library()
    from paper_2404_13216_gb300 import pbcg
    rp = np.array([0, 1, 4, 4] + [4] * 30 + [9], dtype=np.int64)    # 34 rows: slice 0 width 3, slice 1 width 5
    assert pbcg.sell_entries(rp) == 32 * 3 + 32 * 5


def test_serving_loop_rejects_what_can_never_fit():
    reqs = inputs.serving_requests(count=10, rate=1e5, n_lo=900, n_hi=1000, seed=4)
    templates = [serve.Template(inputs.CSR(r.n, None, None, None), None, r.n, 0, 0, r.dim, r.side, r.peclet)
                 for r in reqs]
    pools = {True: FakePool(2, 1000), False: FakePool(2, 1000)}
    out = serve.serve(reqs, templates, pools, K=2, clock=FakeClock())
    big = np.array([r.n > 1000 for r in reqs])
    assert big.any() and np.all(out["status"][big] == serve.REJECTED)
    assert np.all(out["status"][~big] == 0)
