"""CPU oracle for BiCGStab (Algorithm 1) and p-BiCGStab (Algorithm 2) of
arXiv 2404.13216, Section 2, with plain or exactly rounded dot products.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` / ``--cpu-table`` CPU-baseline code of
``bench.py`` may import this package.  It shares no code with the GPU library and never imports it.

The arithmetic lives in ``oracle.c`` (plain C, IEEE binary64, compiled with
``-O2 -ffp-contract=off`` so that every fma is explicit).  This module only
compiles it and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

CONVERGED, MAXIT, BREAKDOWN, NONFINITE = 0, 1, 2, 3
BICGSTAB, PIPELINED = 0, 1
PLAIN, EXACT = 0, 1
LIMBS = 136          # base-2^32 limbs of the exact accumulator
SCALE = 2148         # accumulator value = integer * 2^-SCALE

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, no fast-math, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
    P = ctypes.c_void_p
    lib.orc_dot_exact.restype = d
    lib.orc_dot_exact.argtypes = [i64, P, P, ctypes.c_int]
    lib.orc_dot_plain.restype = d
    lib.orc_dot_plain.argtypes = [i64, P, P]
    lib.orc_dot_exact_fixed.restype = ctypes.c_int
    lib.orc_dot_exact_fixed.argtypes = [i64, P, P, P, P]
    lib.orc_round_fixed.restype = d
    lib.orc_round_fixed.argtypes = [P, ctypes.c_int]
    lib.orc_spmv.restype = None
    lib.orc_spmv.argtypes = [i32, P, P, P, P, P]
    lib.orc_solve.restype = ctypes.c_int
    lib.orc_solve.argtypes = [i32, P, P, P, P, P, d, i32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              P, i32, P, P, i32, P, P, P]
    lib.orc_solve_jacobi.restype = ctypes.c_int
    lib.orc_solve_jacobi.argtypes = [i32, P, P, P, P, P, d, i32, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32,
                                     P, i32, P, P, i32, P, P, P]
    lib.orc_solve_rr.restype = ctypes.c_int
    lib.orc_solve_rr.argtypes = [i32, P, P, P, P, P, d, i32, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32,
                                 P, i32, P, P, i32, P, P, P]
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def dot_exact(a, b, nthreads: int = 1) -> float:
    """Correctly rounded sum_i a_i b_i (Section 2, ExBLAS accuracy)."""
    a, b = _f64(a), _f64(b)
    assert a.shape == b.shape and a.ndim == 1
    return _load().orc_dot_exact(a.size, _p(a), _p(b), int(nthreads))


def dot_plain(a, b) -> float:
    """Sequential fma dot: s = fma(a_i, b_i, s) in index order."""
    a, b = _f64(a), _f64(b)
    assert a.shape == b.shape and a.ndim == 1
    return _load().orc_dot_plain(a.size, _p(a), _p(b))


def dot_exact_fixed(a, b):
    """The exact sum as a Python int N with sum = N * 2^-SCALE (None if an operand is non-finite)."""
    a, b = _f64(a), _f64(b)
    limbs = np.zeros(LIMBS, dtype=np.uint32)
    sgn = ctypes.c_int(0)
    rc = _load().orc_dot_exact_fixed(a.size, _p(a), _p(b), _p(limbs), ctypes.byref(sgn))
    if rc < 0:
        return None
    mag = int.from_bytes(limbs.astype("<u4").tobytes(), "little")
    return -mag if sgn.value else mag


def round_fixed(N: int) -> float:
    """Round N * 2^-SCALE to the nearest double with the oracle's rounding routine."""
    mag = abs(N)
    limbs = np.frombuffer(mag.to_bytes(LIMBS * 4, "little"), dtype="<u4").astype(np.uint32)
    return _load().orc_round_fixed(_p(limbs), 1 if N < 0 else 0)


def spmv(row_ptr, col_idx, vals, x):
    """y = A x, each row an fma chain in stored column order."""
    rp, ci, v, x = _i32(row_ptr), _i32(col_idx), _f64(vals), _f64(x)
    n = rp.size - 1
    y = np.empty(n, dtype=np.float64)
    _load().orc_spmv(n, _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


@dataclass
class Result:
    status: int
    iters: int
    x: np.ndarray
    history: np.ndarray
    relres_recursive: float
    relres_true: float
    trace: np.ndarray = field(default=None)   # rows: alpha_i, omega_i, beta_i, res_{i+1}


def solve(row_ptr, col_idx, vals, b, x0=None, tol=1e-8, maxit=1000, alg=PIPELINED, mode=EXACT,
          nthreads: int = 1, trace: bool = False, rr_period: int = 0, jacobi: bool = False) -> Result:
    """Run Algorithm 1 (alg=BICGSTAB) or Algorithm 2 (alg=PIPELINED) from x0;
    rr_period > 0 adds residual replacement every rr_period iterations (Algorithm 2);
    jacobi=True solves with right Jacobi preconditioning (orc_solve_jacobi)."""
    rp, ci, v, b = _i32(row_ptr), _i32(col_idx), _f64(vals), _f64(b)
    n = rp.size - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    cap = int(maxit) + 1
    hist = np.full(cap, np.nan)
    tr = np.full((max(int(maxit), 1), 4), np.nan) if trace else None
    hl, it = ctypes.c_int32(0), ctypes.c_int32(0)
    rr, rt = ctypes.c_double(0), ctypes.c_double(0)
    fn = _load().orc_solve_jacobi if jacobi else _load().orc_solve_rr
    st = fn(n, _p(rp), _p(ci), _p(v), _p(b), _p(x), float(tol), int(maxit), int(alg),
                           int(mode), int(nthreads), int(rr_period), _p(hist), cap, ctypes.byref(hl),
                           _p(tr) if trace else None, tr.shape[0] if trace else 0,
                           ctypes.byref(it), ctypes.byref(rr), ctypes.byref(rt))
    if st < 0:
        raise ValueError("oracle: invalid input")
    return Result(st, it.value, x, hist[:hl.value].copy(), rr.value, rt.value,
                  tr[:it.value].copy() if trace else None)
