"""Seeded synthetic inputs: sparse unsymmetric systems A x = b in FP64 CSR.

The paper's experiments (Section 3) run on SuiteSparse matrices, which are not
available here; these generators stand in for them with the shapes, sparsity
patterns and value ranges of the workloads this library is measured on.  The
module holds no arithmetic of the solver: it builds matrices, right-hand sides
and request streams only, and is shared by the GPU path's tests and benchmark
and by the CPU oracle's tests.

CSR layout: ``row_ptr`` int32 (n+1), ``col_idx`` int32 (nnz, ascending within a
row), ``vals`` float64 (nnz).  The right-hand side is b = A * ones, each entry
the sequential sum of its row's values in stored order, so the solution of
every generated system is the ones vector.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def matrix_bytes(self) -> int:
        """Bytes of one full stream of the matrix: 8+4 per nonzero, 4 per row pointer."""
        return 12 * self.nnz + 4 * (self.n + 1)


def row_sums(row_ptr: np.ndarray, vals: np.ndarray) -> np.ndarray:
    """Per-row sum of values.  Rows of at most 64 entries are summed
    sequentially in stored order (bitwise reproducible on any machine);
    longer rows use numpy's segmented reduction."""
    n = row_ptr.size - 1
    lens = np.diff(row_ptr).astype(np.int64)
    maxlen = int(lens.max()) if n else 0
    if maxlen <= 64:
        out = np.zeros(n, dtype=np.float64)
        start = row_ptr[:-1].astype(np.int64)
        for k in range(maxlen):
            m = lens > k
            out[m] = out[m] + vals[start[m] + k]
        return out
    out = np.zeros(n, dtype=np.float64)
    nz = lens > 0
    out[nz] = np.add.reduceat(vals, row_ptr[:-1][nz].astype(np.int64))
    return out


def convdiff(N: int, dim: int, Pe: float, wind) -> CSR:
    """Upwind finite-difference convection-diffusion -Lap(u) + Pe (w . grad u)
    on the unit square (dim=2, 5-point) or cube (dim=3, 7-point), Dirichlet
    boundary, mesh width h = 1/(N+1), scaled by h^2, lexicographic order with x
    fastest.  Diagonal 2*dim + Pe*h*sum|w_k|; along axis k the upwind neighbour
    gets -1 - Pe*h*|w_k| and the downwind neighbour -1."""
    assert dim in (2, 3) and len(wind) == dim and N >= 1
    h = 1.0 / (N + 1)
    n = N ** dim
    idx = np.arange(n, dtype=np.int64)
    diag_val = float(2 * dim) + Pe * h * float(sum(abs(w) for w in wind))
    cols, vals, valid = [], [], []
    # ascending column order: -z, -y, -x, diag, +x, +y, +z
    for d in reversed(range(dim)):
        stride = N ** d
        c = (idx // stride) % N
        up = -1.0 - Pe * h * abs(wind[d]) if wind[d] > 0 else -1.0
        cols.append(idx - stride)
        vals.append(np.full(n, up))
        valid.append(c > 0)
    cols.append(idx)
    vals.append(np.full(n, diag_val))
    valid.append(np.ones(n, dtype=bool))
    for d in range(dim):
        stride = N ** d
        c = (idx // stride) % N
        up = -1.0 - Pe * h * abs(wind[d]) if wind[d] < 0 else -1.0
        cols.append(idx + stride)
        vals.append(np.full(n, up))
        valid.append(c < N - 1)
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    M = np.stack(valid, axis=1)
    counts = M.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr.astype(np.int32), C[M].astype(np.int32), V[M].astype(np.float64))


def convdiff2d(N: int = 64, Pe: float = 10.0, wind=(1.0, 0.5)) -> CSR:
    return convdiff(N, 2, Pe, wind)


def convdiff3d(N: int = 128, Pe: float = 50.0, wind=(1.0, 0.5, 0.25)) -> CSR:
    return convdiff(N, 3, Pe, wind)


def _pareto_shape(mean_off: float, kmax: int) -> float:
    """Exponent a of P(k) ~ k^-a on k = 1..kmax whose mean is mean_off (bisection)."""
    k = np.arange(1, kmax + 1, dtype=np.float64)

    def mean_of(a):
        w = k ** (-a)
        return float((k * w).sum() / w.sum())

    lo, hi = 1.0001, 4.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean_of(mid) > mean_off:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def powerlaw(n: int = 1 << 22, mean_len: float = 30.0, max_len: int = 2000, seed: int = 3) -> CSR:
    """Random unsymmetric sparse matrix with power-law row lengths.

    Row length L = 1 (diagonal) + k, k drawn from a discrete power law on
    1..max_len-1 whose exponent is fitted so that E[L] = mean_len.  Off-diagonal
    columns are uniform over j != i (duplicates dropped, so a few rows come out
    shorter), sorted ascending; values N(0,1) * 10^U(-4,4).  The diagonal is
    1.1 * (sum of |off-diagonal| in the row) with a random sign.
    """
    rng = np.random.default_rng(seed)
    kmax = max_len - 1
    a = _pareto_shape(mean_len - 1.0, kmax)
    kk = np.arange(1, kmax + 1, dtype=np.float64)
    pdf = kk ** (-a)
    cdf = np.cumsum(pdf / pdf.sum())
    cdf[-1] = 1.0
    k = (np.searchsorted(cdf, rng.random(n), side="right") + 1).astype(np.int64)
    k = np.minimum(k, kmax)
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    c = rng.integers(0, n - 1, size=rows.size, dtype=np.int64)
    c = c + (c >= rows)                      # skip the diagonal
    keys = np.concatenate([rows * n + c, np.arange(n, dtype=np.int64) * (n + 1)])
    del rows, c
    keys.sort()
    keep = np.ones(keys.size, dtype=bool)
    keep[1:] = keys[1:] != keys[:-1]
    keys = keys[keep]
    del keep
    r = keys // n
    col = (keys - r * n).astype(np.int32)
    del keys
    is_diag = col == r
    counts = np.bincount(r, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    del r
    nnz = int(row_ptr[-1])
    vals = rng.standard_normal(nnz) * 10.0 ** rng.uniform(-4.0, 4.0, nnz)
    vals[is_diag] = 0.0
    absum = np.add.reduceat(np.abs(vals), row_ptr[:-1])
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    vals[is_diag] = 1.1 * absum * sign
    return CSR(n, row_ptr.astype(np.int32), col, vals)


def rhs_ones(A: CSR) -> np.ndarray:
    """b = A * ones."""
    return row_sums(A.row_ptr, A.vals)


@dataclass
class BlockSystem:
    """Independent systems stacked as one block-diagonal CSR."""
    A: CSR
    sys_row_ptr: np.ndarray     # int32, nsys+1: rows of system k are [sys_row_ptr[k], sys_row_ptr[k+1])
    sides: np.ndarray
    peclet: np.ndarray

    @property
    def nsys(self) -> int:
        return int(self.sys_row_ptr.size - 1)


def block_diag(systems) -> tuple[CSR, np.ndarray]:
    """Stack CSR matrices into one block-diagonal CSR; returns (A, sys_row_ptr)."""
    ns = [s.n for s in systems]
    sys_row_ptr = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(ns, out=sys_row_ptr[1:])
    nnzs = [s.nnz for s in systems]
    nnz_off = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(nnzs, out=nnz_off[1:])
    n = int(sys_row_ptr[-1])
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(int(nnz_off[-1]), dtype=np.int32)
    vals = np.empty(int(nnz_off[-1]), dtype=np.float64)
    for k, s in enumerate(systems):
        r0, r1 = sys_row_ptr[k], sys_row_ptr[k + 1]
        row_ptr[r0:r1] = s.row_ptr[:-1].astype(np.int64) + nnz_off[k]
        col[nnz_off[k]:nnz_off[k + 1]] = s.col_idx + np.int32(r0)
        vals[nnz_off[k]:nnz_off[k + 1]] = s.vals
    row_ptr[n] = nnz_off[-1]
    return CSR(n, row_ptr.astype(np.int32), col, vals), sys_row_ptr.astype(np.int32)


def batched_convdiff(nsys: int = 512, side_lo: int = 32, side_hi: int = 256, pe_lo: float = 1.0,
                     pe_hi: float = 100.0, wind=(1.0, 0.5), seed: int = 4) -> BlockSystem:
    """nsys 2D convection-diffusion systems, grid side log-uniform in
    [side_lo, side_hi] (rounded), Peclet U(pe_lo, pe_hi), one block-diagonal CSR."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(math.log(side_lo), math.log(side_hi), nsys))).astype(np.int64)
    pes = rng.uniform(pe_lo, pe_hi, nsys)
    systems = [convdiff(int(s), 2, float(p), wind) for s, p in zip(sides, pes)]
    A, srp = block_diag(systems)
    return BlockSystem(A, srp, sides, pes)


@dataclass
class Request:
    arrival: float        # seconds from the start of the stream
    dim: int
    side: int
    peclet: float
    tol: float
    exact: bool

    @property
    def n(self) -> int:
        return self.side ** self.dim


def serving_requests(count: int = 4000, rate: float = 2000.0, n_lo: int = 4096, n_hi: int = 1 << 20,
                     seed: int = 5) -> list[Request]:
    """Open-loop Poisson request stream: 2D or 3D convection-diffusion solves
    (half each), n log-uniform in [n_lo, n_hi], side = round(n^(1/dim)),
    Peclet U(1,100), tolerance 1e-8 or 1e-10, plain or exact dots (half each)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    dims = np.where(rng.random(count) < 0.5, 2, 3)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))
    pes = rng.uniform(1.0, 100.0, count)
    tols = np.where(rng.random(count) < 0.5, 1e-8, 1e-10)
    exact = rng.random(count) < 0.5
    out = []
    for i in range(count):
        d = int(dims[i])
        side = max(2, int(round(ns[i] ** (1.0 / d))))
        out.append(Request(float(t[i]), d, side, float(pes[i]), float(tols[i]), bool(exact[i])))
    return out


def request_matrix(req: Request) -> CSR:
    wind = (1.0, 0.5) if req.dim == 2 else (1.0, 0.5, 0.25)
    return convdiff(req.side, req.dim, req.peclet, wind)
