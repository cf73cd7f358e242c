"""Serving loop over solver pools: an open-loop Poisson stream of independent
solves, admitted while earlier ones run, batched as they arrive (continuous
batching), each retired as soon as it stops.  Reports solves/s and latency
percentiles (arrival to result on the host, queueing included).

Requests carry their own tolerance and dot mode; exact and plain requests go
to two pools on two contexts, so their steps run on two streams side by side.
A pool is a fixed arena allocated once (rows, matrix entries, slots);
admission takes the first queued request of a mode when its pool has a free
slot and room for its rows and entries, in arrival order.

Every solve runs in the library's kernels through the C ABI (pbcg.Pool); this
module only schedules host calls.
"""
from __future__ import annotations

import argparse
import json
import time
from collections import deque
from dataclasses import dataclass

import numpy as np

from . import inputs

REJECTED = -5      # status of a request that no pool of its mode can hold


@dataclass
class Template:
    """A request's system: the CSR matrix and b = A * ones, in pinned host memory when torch is present."""
    A: object
    b: object
    n: int
    nnz: int
    entries: int
    dim: int
    side: int
    peclet: float


def _pin(a):
    try:
        import torch
        if torch.cuda.is_available():
            t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            return t
    except Exception:
        pass
    return np.ascontiguousarray(a)


def make_templates(reqs, count: int):
    """Systems of the first `count` requests of the stream; request i then
    uses system i mod count (the matrix set is a `count`-point sample of the
    stream's size and Peclet distribution)."""
    from .pbcg import sell_entries
    out = []
    for r in reqs[:count]:
        A = inputs.request_matrix(r)
        b = inputs.rhs_ones(A)
        P = inputs.CSR(A.n, _pin(A.row_ptr), _pin(A.col_idx), _pin(A.vals))
        out.append(Template(P, _pin(b), A.n, int(A.vals.size), sell_entries(A.row_ptr), r.dim, r.side, r.peclet))
    return out


def percentile(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else float("nan")


def serve(reqs, templates, pools: dict, K: int = 8, maxit: int = 2000, max_in_flight: int = 2,
          clock=time.perf_counter, time_limit: float = 600.0):
    """Run the request stream through `pools` ({True: exact pool, False: plain
    pool}).  Returns per-request arrays: latency (s), status, iterations,
    true relative residual, and the run's wall time."""
    nreq = len(reqs)
    lat = np.full(nreq, np.nan)
    status = np.full(nreq, -99, dtype=np.int64)
    iters = np.zeros(nreq, dtype=np.int64)
    relres = np.full(nreq, np.nan)
    queue = {m: deque() for m in pools}
    live = {m: {} for m in pools}
    steps = {m: 0 for m in pools}
    nxt = finished = 0
    t0 = clock()
    while finished < nreq:
        now = clock() - t0
        if now > time_limit:
            break
        while nxt < nreq and reqs[nxt].arrival <= now:
            queue[reqs[nxt].exact].append(nxt)
            nxt += 1
        busy = False
        for m, pool in pools.items():
            done, pending = pool.poll(wait=False)
            for s in done:
                i = live[m].pop(s)
                _, res = pool.result(s)
                lat[i] = clock() - t0 - reqs[i].arrival
                status[i], iters[i], relres[i] = res.status, res.iters, res.relres_true
                finished += 1
                busy = True
            q = queue[m]
            while q:
                i = q[0]
                T = templates[i % len(templates)]
                s = pool.admit(T.A, T.b, tol=reqs[i].tol, maxit=maxit)
                if s is None:
                    if not live[m]:                  # larger than the whole pool: reject it
                        q.popleft()
                        status[i], lat[i] = REJECTED, clock() - t0 - reqs[i].arrival
                        finished += 1
                        continue
                    break
                live[m][s] = i
                q.popleft()
                busy = True
            if live[m] and pending < max_in_flight:
                pool.step(K)
                steps[m] += 1
                busy = True
        if not busy:
            if any(live.values()):
                # wait for the pool whose newest step is oldest
                for m, pool in pools.items():
                    if live[m]:
                        d, _ = pool.poll(wait=True)
                        for s in d:
                            i = live[m].pop(s)
                            _, res = pool.result(s)
                            lat[i] = clock() - t0 - reqs[i].arrival
                            status[i], iters[i], relres[i] = res.status, res.iters, res.relres_true
                            finished += 1
                        break
            elif nxt < nreq:
                time.sleep(max(0.0, min(1e-3, reqs[nxt].arrival - (clock() - t0))))
    wall = clock() - t0
    return dict(latency=lat, status=status, iters=iters, relres=relres, wall=wall, steps=steps)


def summarize(reqs, templates, out, rate):
    lat = out["latency"]
    ok = ~np.isnan(lat)
    st = out["status"][ok]
    ns = np.array([templates[i % len(templates)].n for i in range(len(reqs))])
    return {
        "requests": len(reqs), "finished": int(ok.sum()), "rate_per_s": rate,
        "solves_per_s": float(ok.sum() / out["wall"]), "wall_s": out["wall"],
        "p50_ms": percentile(lat[ok] * 1e3, 50), "p99_ms": percentile(lat[ok] * 1e3, 99),
        "converged": int((st == 0).sum()), "maxit": int((st == 1).sum()), "breakdown": int((st == 2).sum()),
        "nonfinite": int((st == 3).sum()), "rejected": int((st == REJECTED).sum()),
        "failed": int(((st < 0) & (st != REJECTED)).sum()),
        "mean_iters": float(out["iters"][ok].mean()) if ok.any() else None,
        "mean_n": float(ns.mean()), "templates": len(templates),
        "exact_share": float(np.mean([r.exact for r in reqs])), "steps": out["steps"],
    }


def make_pools(ctx_exact, ctx_plain, templates, max_rows: int, max_entries: int, max_slots: int, maxit: int,
               alg: int):
    from . import pbcg
    big_n = max(t.n for t in templates)
    big_nnz = max(t.nnz for t in templates)
    mk = lambda c, mode: pbcg.Pool(c, max_rows=max_rows, max_entries=max_entries, max_slots=max_slots,
                                   maxit=maxit, alg=alg, mode=mode, max_request_rows=big_n,
                                   max_request_nnz=big_nnz)
    return {True: mk(ctx_exact, pbcg.EXACT), False: mk(ctx_plain, pbcg.PLAIN)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--templates", type=int, default=64)
    ap.add_argument("--k", type=int, default=8, help="iterations per step launch")
    ap.add_argument("--maxit", type=int, default=2000)
    ap.add_argument("--alg", type=int, default=1)
    ap.add_argument("--max-rows", type=int, default=48 << 20)
    ap.add_argument("--max-entries", type=int, default=384 << 20)
    ap.add_argument("--max-slots", type=int, default=512)
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args(argv)
    from . import pbcg
    reqs = inputs.serving_requests(count=a.requests, rate=a.rate, seed=a.seed)
    templates = make_templates(reqs, a.templates)
    ce, cp = pbcg.Context(0), pbcg.Context(0)
    pools = make_pools(ce, cp, templates, a.max_rows, a.max_entries, a.max_slots, a.maxit, a.alg)
    out = serve(reqs, templates, pools, K=a.k, maxit=a.maxit)
    print(json.dumps(summarize(reqs, templates, out, a.rate)))
    for p in pools.values():
        p.close()
    ce.close()
    cp.close()


if __name__ == "__main__":
    main()
