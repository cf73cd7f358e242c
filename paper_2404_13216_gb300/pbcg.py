"""ctypes binding of libpbcg.so (include/pbcg.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module moves
pointers and sizes across the C ABI.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA; their data_ptr is passed through).  Loading the
module raises if the library has not been built -- there is no fallback.
The environment variable PBCG_LIB, when set, names another build of the
library to load instead (for example _build/libpbcg_checked.so, the build
with device-side bounds checks); results do not change.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PBCG_LIB") or os.path.join(_HERE, "_build", "libpbcg.so")

OK, MAXIT, BREAKDOWN, NONFINITE = 0, 1, 2, 3
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_COMM = -1, -2, -3, -4, -5
BICGSTAB, PIPELINED, PIPELINED_RR = 0, 1, 2
OPT_RR_PERIOD, OPT_PRECOND, OPT_SMALL_CLUSTER, OPT_BATCH_GRAPH = 1, 3, 4, 5
PRECOND_NONE, PRECOND_JACOBI = 0, 1
PLAIN, EXACT = 0, 1

EXPORTS = ("pbcg_create", "pbcg_destroy", "pbcg_last_error", "pbcg_csr_upload", "pbcg_mat_free",
           "pbcg_solve", "pbcg_solve_batched", "pbcg_residual_history", "pbcg_dot", "pbcg_spmv",
           "pbcg_profile_solve", "pbcg_dot_noalloc", "pbcg_set_option", "pbcg_pool_create", "pbcg_pool_destroy",
           "pbcg_pool_admit", "pbcg_pool_step", "pbcg_pool_poll", "pbcg_pool_result", "pbcg_pool_history",
           "pbcg_pool_room", "pbcg_check_wait", "pbcg_part_plan", "pbcg_part_create", "pbcg_part_solve",
           "pbcg_part_destroy", "pbcg_set_variant", "pbcg_get_variant", "pbcg_tune", "pbcg_mat_check",
           "pbcg_check_word", "pbcg_debug_set_col")


class PbcgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pbcg error {code}: {msg}")
        self.code = code


class _PoolConfig(ctypes.Structure):
    _fields_ = [("max_rows", ctypes.c_int64), ("max_entries", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("maxit", ctypes.c_int32), ("alg", ctypes.c_int32), ("dot_mode", ctypes.c_int32),
                ("max_request_rows", ctypes.c_int64), ("max_request_nnz", ctypes.c_int64),
                ("precond", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("relres_recursive", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("seconds", ctypes.c_double), ("launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_ALLREDUCE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64)
_ALLTOALLV = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int64))


class _Variant(ctypes.Structure):
    _fields_ = [("staged", ctypes.c_int32), ("order", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("batched_ctas_per_sm", ctypes.c_int32), ("us_per_iter", ctypes.c_double)]


class _Comm(ctypes.Structure):
    _fields_ = [("user", ctypes.c_void_p), ("allreduce_sum_i64", _ALLREDUCE), ("alltoallv", _ALLTOALLV)]


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2404_13216_gb300.build.build_library()")
    lib = ctypes.CDLL(path)
    P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.pbcg_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P]
    lib.pbcg_create.restype = ctypes.c_int
    lib.pbcg_destroy.argtypes = [P]
    lib.pbcg_destroy.restype = None
    lib.pbcg_last_error.argtypes = [P]
    lib.pbcg_last_error.restype = ctypes.c_char_p
    lib.pbcg_csr_upload.argtypes = [P, i32, i64, P, P, P, ctypes.c_int, ctypes.POINTER(P)]
    lib.pbcg_csr_upload.restype = ctypes.c_int
    lib.pbcg_mat_free.argtypes = [P, P]
    lib.pbcg_mat_free.restype = ctypes.c_int
    lib.pbcg_solve.argtypes = [P, P, P, P, d, i32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Result)]
    lib.pbcg_solve.restype = ctypes.c_int
    lib.pbcg_solve_batched.argtypes = [P, P, i32, P, P, P, P, i32, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(_Result)]
    lib.pbcg_solve_batched.restype = ctypes.c_int
    lib.pbcg_residual_history.argtypes = [P, i32, P, i32, ctypes.POINTER(i32)]
    lib.pbcg_residual_history.restype = ctypes.c_int
    lib.pbcg_dot.argtypes = [P, i64, P, P, ctypes.c_int, ctypes.POINTER(d)]
    lib.pbcg_dot.restype = ctypes.c_int
    lib.pbcg_spmv.argtypes = [P, P, P, P]
    lib.pbcg_spmv.restype = ctypes.c_int
    lib.pbcg_check_wait.argtypes = [P, i32, ctypes.POINTER(i32), ctypes.POINTER(d)]
    lib.pbcg_check_wait.restype = ctypes.c_int
    lib.pbcg_profile_solve.argtypes = [P, P, P, P, d, i32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Result),
                                       P, P, P, i32, ctypes.POINTER(i32)]
    lib.pbcg_profile_solve.restype = ctypes.c_int
    lib.pbcg_dot_noalloc.argtypes = [i64, P, P, ctypes.c_int, P, P]
    lib.pbcg_set_option.argtypes = [P, ctypes.c_int, i64]
    lib.pbcg_set_option.restype = ctypes.c_int
    lib.pbcg_dot_noalloc.restype = ctypes.c_int
    lib.pbcg_pool_create.argtypes = [P, ctypes.POINTER(_PoolConfig), ctypes.POINTER(P)]
    lib.pbcg_pool_create.restype = ctypes.c_int
    lib.pbcg_pool_destroy.argtypes = [P]
    lib.pbcg_pool_destroy.restype = None
    lib.pbcg_pool_admit.argtypes = [P, i32, i64, P, P, P, P, P, d, i32, ctypes.POINTER(i32)]
    lib.pbcg_pool_admit.restype = ctypes.c_int
    lib.pbcg_pool_step.argtypes = [P, i32]
    lib.pbcg_pool_step.restype = ctypes.c_int
    lib.pbcg_pool_poll.argtypes = [P, ctypes.c_int, P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.pbcg_pool_poll.restype = ctypes.c_int
    lib.pbcg_pool_result.argtypes = [P, i32, P, ctypes.POINTER(_Result)]
    lib.pbcg_pool_result.restype = ctypes.c_int
    lib.pbcg_pool_history.argtypes = [P, i32, P, i32, ctypes.POINTER(i32)]
    lib.pbcg_pool_history.restype = ctypes.c_int
    lib.pbcg_pool_room.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.pbcg_pool_room.restype = ctypes.c_int
    lib.pbcg_part_plan.argtypes = [i32, i32, P, i64, P, P, ctypes.POINTER(i32), P, i32, P, P]
    lib.pbcg_part_plan.restype = ctypes.c_int
    lib.pbcg_part_create.argtypes = [P, ctypes.POINTER(_Comm), i32, i32, P, i64, P, P, P, ctypes.POINTER(P)]
    lib.pbcg_part_create.restype = ctypes.c_int
    lib.pbcg_part_solve.argtypes = [P, P, P, d, i32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Result)]
    lib.pbcg_part_solve.restype = ctypes.c_int
    lib.pbcg_part_destroy.argtypes = [P]
    lib.pbcg_part_destroy.restype = None
    lib.pbcg_set_variant.argtypes = [P, P, ctypes.POINTER(_Variant)]
    lib.pbcg_set_variant.restype = ctypes.c_int
    lib.pbcg_get_variant.argtypes = [P, P, ctypes.POINTER(_Variant)]
    lib.pbcg_get_variant.restype = ctypes.c_int
    lib.pbcg_tune.argtypes = [P, P, ctypes.c_int, ctypes.c_int, i32, P, i32, ctypes.c_char_p,
                              ctypes.POINTER(_Variant), P, i32, ctypes.POINTER(i32)]
    lib.pbcg_tune.restype = ctypes.c_int
    lib.pbcg_mat_check.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint64)]
    lib.pbcg_mat_check.restype = ctypes.c_int
    lib.pbcg_check_word.argtypes = [P, ctypes.c_int, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint64)]
    lib.pbcg_check_word.restype = ctypes.c_int
    lib.pbcg_debug_set_col.argtypes = [P, P, i64, i32]
    lib.pbcg_debug_set_col.restype = ctypes.c_int
    return lib


_lib = load_library()


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _host(a, dtype):
    """A numpy input converted to a C-contiguous `dtype` array, or a torch
    tensor (host or device), which must already be contiguous `dtype`."""
    if hasattr(a, "data_ptr"):
        want = np.dtype(dtype).name
        if str(a.dtype) != "torch." + want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor, got {a.dtype}"
                            + ("" if a.is_contiguous() else " (not contiguous)"))
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _count(a) -> int:
    return a.numel() if hasattr(a, "numel") else a.size


def _vec_in(a, n: int, name: str, dtype=np.float64):
    """An input vector of exactly n entries."""
    a = _host(a, dtype)
    if _count(a) != n:
        raise ValueError(f"{name} has {_count(a)} entries, expected {n}")
    return a


def _vec_out(a, n: int, name: str):
    """A float64 vector of n entries that the library writes in place, so it
    is checked, never converted."""
    if hasattr(a, "data_ptr"):
        _host(a, np.float64)
    elif not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.flags.writeable):
        raise TypeError(f"{name} must be a writable C-contiguous float64 array or tensor (written in place)")
    if _count(a) != n:
        raise ValueError(f"{name} has {_count(a)} entries, expected {n}")
    return a


def _csr(row_ptr, col_idx, vals):
    rp, ci, va = _host(row_ptr, np.int32), _host(col_idx, np.int32), _host(vals, np.float64)
    n, nnz = _count(rp) - 1, _count(va)
    if n < 0 or _count(ci) != nnz:
        raise ValueError(f"CSR arrays disagree: {_count(rp)} row pointers, {_count(ci)} column indices, "
                         f"{nnz} values")
    return rp, ci, va, n, nnz


def _cuda_f64(t, name: str):
    """A contiguous float64 CUDA tensor on the current device (pbcg_dot_noalloc
    takes device memory only and reads or writes it without a copy)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (device memory)")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 tensor, got {t.dtype}"
                        + ("" if t.is_contiguous() else " (not contiguous)"))
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, the current device is cuda:{torch.cuda.current_device()}")
    return t


def dot_noalloc(a, b, out, mode: int = EXACT, stream=None) -> int:
    """pbcg_dot_noalloc: (a, b) into out[0]; a, b, out are contiguous float64
    CUDA tensors on the current device, b as long as a.  Asynchronous on
    `stream` (a raw cudaStream_t or None).  Returns the library's status code
    (0 or negative)."""
    a, b, out = _cuda_f64(a, "a"), _cuda_f64(b, "b"), _cuda_f64(out, "out")
    n = a.numel()
    if b.numel() != n:
        raise ValueError(f"b has {b.numel()} entries, expected {n}")
    if out.numel() < 1:
        raise ValueError("out needs at least one entry")
    s = ctypes.c_void_p(stream) if stream else None
    return _lib.pbcg_dot_noalloc(n, _ptr(a), _ptr(b), int(mode), _ptr(out), s)


@dataclass
class Variant:
    """A launch variant of the passes (pbcg_variant): none changes exact results."""
    staged: int = 1
    order: int = 0
    ctas_per_sm: int = 0
    batched_ctas_per_sm: int = 0
    us_per_iter: float = 0.0

    def _c(self):
        return _Variant(int(self.staged), int(self.order), int(self.ctas_per_sm), int(self.batched_ctas_per_sm),
                        float(self.us_per_iter))

    @staticmethod
    def _of(v):
        return Variant(v.staged, v.order, v.ctas_per_sm, v.batched_ctas_per_sm, v.us_per_iter)


@dataclass
class Result:
    status: int
    iters: int
    relres_recursive: float
    relres_true: float
    seconds: float
    launches: int = 0


class Matrix:
    def __init__(self, ctx: "Context", handle, n: int, nnz: int):
        self.ctx, self.handle, self.n, self.nnz = ctx, handle, n, nnz

    def free(self):
        if self.handle:
            self.ctx._check(_lib.pbcg_mat_free(self.ctx.handle, self.handle))
            self.handle = None


class Context:
    """One libpbcg context: a device, a stream, its matrices and workspace."""

    def __init__(self, device: int = 0, stream=None):
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream else None
        rc = _lib.pbcg_create(ctypes.byref(h), int(device), s)
        if rc != 0:
            raise PbcgError(rc, "pbcg_create failed")
        self.handle = h

    def close(self):
        if self.handle:
            _lib.pbcg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        self._check(_lib.pbcg_set_option(self.handle, int(option), int(value)))

    def last_error(self) -> str:
        return _lib.pbcg_last_error(self.handle).decode()

    def _check(self, rc: int) -> int:
        if rc < 0:
            raise PbcgError(rc, self.last_error())
        return rc

    def upload(self, row_ptr, col_idx, vals) -> Matrix:
        rp, ci, va, n, nnz = _csr(row_ptr, col_idx, vals)
        m = ctypes.c_void_p()
        dev = int(hasattr(rp, "is_cuda") and rp.is_cuda)
        self._check(_lib.pbcg_csr_upload(self.handle, n, nnz, _ptr(rp), _ptr(ci), _ptr(va), dev, ctypes.byref(m)))
        return Matrix(self, m, n, nnz)

    def upload_csr(self, A) -> Matrix:
        return self.upload(A.row_ptr, A.col_idx, A.vals)

    def solve(self, mat: Matrix, b, x, tol: float, maxit: int, alg: int = PIPELINED, mode: int = EXACT) -> Result:
        """Solve in place: x holds x0 on entry and the last iterate on return."""
        b, x = _vec_in(b, mat.n, "b"), _vec_out(x, mat.n, "x")
        r = _Result()
        self._check(_lib.pbcg_solve(self.handle, mat.handle, _ptr(b), _ptr(x), float(tol), int(maxit), int(alg),
                                    int(mode), ctypes.byref(r)))
        return Result(r.status, r.iters, r.relres_recursive, r.relres_true, r.seconds, r.launches)

    def solve_batched(self, mat: Matrix, sys_row_ptr, b, x, tol, maxit: int, alg: int = PIPELINED,
                      mode: int = EXACT):
        srp = _host(sys_row_ptr, np.int32)
        nsys = _count(srp) - 1
        if nsys < 1:
            raise ValueError("sys_row_ptr needs at least two entries")
        tl = _vec_in(tol, nsys, "tol")
        b, x = _vec_in(b, mat.n, "b"), _vec_out(x, mat.n, "x")
        res = (_Result * nsys)()
        self._check(_lib.pbcg_solve_batched(self.handle, mat.handle, nsys, _ptr(srp), _ptr(b), _ptr(x), _ptr(tl),
                                            int(maxit), int(alg), int(mode), res))
        return [Result(r.status, r.iters, r.relres_recursive, r.relres_true, r.seconds, r.launches) for r in res]

    def history(self, sys: int = 0) -> np.ndarray:
        ln = ctypes.c_int32(0)
        self._check(_lib.pbcg_residual_history(self.handle, int(sys), None, 0, ctypes.byref(ln)))
        out = np.empty(ln.value, dtype=np.float64)
        self._check(_lib.pbcg_residual_history(self.handle, int(sys), _ptr(out), ln.value, ctypes.byref(ln)))
        return out

    def dot(self, a, b, mode: int = EXACT) -> float:
        a = _host(a, np.float64)
        n = _count(a)
        b = _vec_in(b, n, "b")
        out = ctypes.c_double(0.0)
        self._check(_lib.pbcg_dot(self.handle, n, _ptr(a), _ptr(b), int(mode), ctypes.byref(out)))
        return out.value

    def set_variant(self, mat: Matrix, v: "Variant" = None):
        """Set mat's launch variant (None: the default)."""
        c = v._c() if v is not None else None
        self._check(_lib.pbcg_set_variant(self.handle, mat.handle, ctypes.byref(c) if c is not None else None))

    def get_variant(self, mat: Matrix) -> "Variant":
        v = _Variant()
        self._check(_lib.pbcg_get_variant(self.handle, mat.handle, ctypes.byref(v)))
        return Variant._of(v)

    def tune(self, mat: Matrix, alg: int = PIPELINED, mode: int = EXACT, iters: int = 30, sys_row_ptr=None,
             cache_path: str = None):
        """pbcg_tune: time the launch variants on a trial solve and keep the
        fastest for mat.  Returns (chosen Variant, [tried Variants])."""
        srp = None if sys_row_ptr is None else _host(sys_row_ptr, np.int32)
        nsys = 0 if srp is None else _count(srp) - 1
        cap = 16
        tried = (_Variant * cap)()
        ch, nt = _Variant(), ctypes.c_int32(0)
        self._check(_lib.pbcg_tune(self.handle, mat.handle, int(alg), int(mode), nsys, _ptr(srp), int(iters),
                                   cache_path.encode() if cache_path else None, ctypes.byref(ch),
                                   ctypes.cast(tried, ctypes.c_void_p), cap, ctypes.byref(nt)))
        return Variant._of(ch), [Variant._of(tried[i]) for i in range(min(nt.value, cap))]

    def mat_check(self, mat: Matrix) -> int:
        """pbcg_mat_check: 0, or the first layout failure (kind << 56 | position)."""
        w = ctypes.c_uint64(0)
        self._check(_lib.pbcg_mat_check(self.handle, mat.handle, ctypes.byref(w)))
        return w.value

    def check_word(self, reset: bool = False):
        """pbcg_check_word: (checks compiled in, first failed in-kernel check or 0)."""
        en, w = ctypes.c_int32(0), ctypes.c_uint64(0)
        self._check(_lib.pbcg_check_word(self.handle, int(bool(reset)), ctypes.byref(en), ctypes.byref(w)))
        return bool(en.value), w.value

    def debug_set_col(self, mat: Matrix, entry: int, col: int):
        """pbcg_debug_set_col (checked build): overwrite one stored column of mat's device layout."""
        self._check(_lib.pbcg_debug_set_col(self.handle, mat.handle, int(entry), int(col)))

    def check_wait(self, probes: int):
        """Run the bounded device wait on a phase nothing completes; returns (expired, seconds)."""
        exp, sec = ctypes.c_int32(0), ctypes.c_double(0.0)
        self._check(_lib.pbcg_check_wait(self.handle, int(probes), ctypes.byref(exp), ctypes.byref(sec)))
        return bool(exp.value), sec.value

    def spmv(self, mat: Matrix, x, y=None):
        x = _vec_in(x, mat.n, "x")
        y = np.empty(mat.n, dtype=np.float64) if y is None else _vec_out(y, mat.n, "y")
        self._check(_lib.pbcg_spmv(self.handle, mat.handle, _ptr(x), _ptr(y)))
        return y

    def profile_solve(self, mat: Matrix, b, x, tol: float, maxit: int, alg: int = PIPELINED, mode: int = EXACT):
        """Solve with a host-driven loop and CUDA events around every kernel.
        Returns (Result, {kernel: (total_ms, launches)})."""
        b, x = _vec_in(b, mat.n, "b"), _vec_out(x, mat.n, "x")
        cap = 32
        names = (ctypes.c_char * 32 * cap)()
        ms = np.zeros(cap, dtype=np.float64)
        cnt = np.zeros(cap, dtype=np.int32)
        k = ctypes.c_int32(0)
        r = _Result()
        self._check(_lib.pbcg_profile_solve(self.handle, mat.handle, _ptr(b), _ptr(x), float(tol), int(maxit),
                                            int(alg), int(mode), ctypes.byref(r), ctypes.cast(names, ctypes.c_void_p),
                                            _ptr(ms), _ptr(cnt), cap, ctypes.byref(k)))
        prof = {}
        for i in range(min(k.value, cap)):
            prof[bytes(names[i]).split(b"\0")[0].decode()] = (float(ms[i]), int(cnt[i]))
        return Result(r.status, r.iters, r.relres_recursive, r.relres_true, r.seconds, r.launches), prof


def sell_entries(row_ptr) -> int:
    """SELL-32 entries a system takes in a pool: 32 x the longest row of each 32-row slice."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    ln = np.zeros(((n + 31) // 32) * 32, dtype=np.int64)
    ln[:n] = np.diff(rp)
    return int(32 * ln.reshape(-1, 32).max(axis=1).sum())


class Pool:
    """A pbcg_pool: continuous batching of independent solves on one context.

    admit() returns a slot or None when the pool has no room now; step()
    enqueues K iterations of every live system; poll() returns the slots that
    finished (each once); result() retires a slot and returns (x, Result)."""

    def __init__(self, ctx: Context, max_rows: int, max_entries: int, max_slots: int, maxit: int,
                 alg: int = PIPELINED, mode: int = EXACT, max_request_rows: int = None,
                 max_request_nnz: int = None, precond: int = 0):
        cfg = _PoolConfig(int(max_rows), int(max_entries), int(max_slots), int(maxit), int(alg), int(mode),
                          int(max_request_rows or max_rows), int(max_request_nnz or max_entries), int(precond), 0)
        h = ctypes.c_void_p()
        ctx._check(_lib.pbcg_pool_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.ctx, self.handle, self.max_slots = ctx, h, int(max_slots)
        self.sizes = {}
        self._buf = np.zeros(self.max_slots, dtype=np.int32)

    def close(self):
        if self.handle:
            _lib.pbcg_pool_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def admit(self, A, b, x0=None, tol: float = 1e-8, maxit: int = 1000):
        rp, ci, va, n, nnz = _csr(A.row_ptr, A.col_idx, A.vals)
        b = _vec_in(b, n, "b")
        x0 = None if x0 is None else _vec_in(x0, n, "x0")
        slot = ctypes.c_int32(-1)
        rc = self.ctx._check(_lib.pbcg_pool_admit(self.handle, n, nnz, _ptr(rp), _ptr(ci), _ptr(va), _ptr(b),
                                                  _ptr(x0), float(tol), int(maxit), ctypes.byref(slot)))
        if rc == 1:
            return None
        self.sizes[slot.value] = n
        return slot.value

    def step(self, iters: int):
        self.ctx._check(_lib.pbcg_pool_step(self.handle, int(iters)))

    def poll(self, wait: bool = False):
        """(finished slots, steps still in flight)."""
        cnt, pend = ctypes.c_int32(0), ctypes.c_int32(0)
        self.ctx._check(_lib.pbcg_pool_poll(self.handle, int(bool(wait)), _ptr(self._buf), self.max_slots,
                                            ctypes.byref(cnt), ctypes.byref(pend)))
        return [int(v) for v in self._buf[:min(cnt.value, self.max_slots)]], pend.value

    def history(self, slot: int) -> np.ndarray:
        ln = ctypes.c_int32(0)
        self.ctx._check(_lib.pbcg_pool_history(self.handle, int(slot), None, 0, ctypes.byref(ln)))
        out = np.empty(ln.value, dtype=np.float64)
        self.ctx._check(_lib.pbcg_pool_history(self.handle, int(slot), _ptr(out), ln.value, ctypes.byref(ln)))
        return out

    def result(self, slot: int, x=None):
        """Retire `slot`: (x, Result).  A request that failed (bad column
        index, device wait expired) gives a Result with its negative code."""
        n = self.sizes.get(slot)
        if x is None:
            x = None if n is None else np.empty(n, dtype=np.float64)
        elif n is not None:
            x = _vec_out(x, n, "x")
        r = _Result()
        rc = _lib.pbcg_pool_result(self.handle, int(slot), _ptr(x), ctypes.byref(r))
        if rc < 0 and r.status >= 0:
            raise PbcgError(rc, self.ctx.last_error())
        self.sizes.pop(slot, None)
        return x, Result(r.status, r.iters, r.relres_recursive, r.relres_true, r.seconds, r.launches)

    def room(self):
        """(free slots, largest free row range, largest free entry range)."""
        fs, fr, fe = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
        self.ctx._check(_lib.pbcg_pool_room(self.handle, ctypes.byref(fs), ctypes.byref(fr), ctypes.byref(fe)))
        return fs.value, fr.value, fe.value


def part_plan(nranks: int, rank: int, row_starts, row_ptr, col_idx):
    """pbcg_part_plan (host only): (halo columns, per-rank counts, local column
    of every entry) of rank `rank`'s block with global column indices."""
    rs = np.ascontiguousarray(row_starts, dtype=np.int32)
    if rs.size != nranks + 1:
        raise ValueError(f"row_starts has {rs.size} entries, expected {nranks + 1}")
    rp, ci = np.ascontiguousarray(row_ptr, dtype=np.int32), np.ascontiguousarray(col_idx, dtype=np.int32)
    nh = ctypes.c_int32(0)
    cnt = np.zeros(max(nranks, 1), dtype=np.int32)
    loc = np.zeros(ci.size, dtype=np.int32)
    rc = _lib.pbcg_part_plan(nranks, rank, _ptr(rs), ci.size, _ptr(rp), _ptr(ci), ctypes.byref(nh), None, 0,
                             _ptr(cnt), _ptr(loc))
    if rc != 0:
        raise PbcgError(rc, "pbcg_part_plan refused the block")
    halo = np.zeros(max(nh.value, 1), dtype=np.int32)
    rc = _lib.pbcg_part_plan(nranks, rank, _ptr(rs), ci.size, _ptr(rp), _ptr(ci), ctypes.byref(nh), _ptr(halo),
                             nh.value, None, None)
    if rc != 0:
        raise PbcgError(rc, "pbcg_part_plan refused the block")
    return halo[:nh.value], cnt[:nranks], loc


def _c_comm(comm):
    """C callbacks calling comm.allreduce_sum_i64(int64 array) and
    comm.alltoallv(send, send_bytes, send_displs, recv, recv_bytes,
    recv_displs) on numpy views of the library's host buffers; an exception
    becomes a nonzero return (PBCG_ERR_COMM)."""
    size = int(comm.size)

    def _view(addr, nbytes):
        if nbytes <= 0 or not addr:
            return np.zeros(0, np.uint8)
        return np.ctypeslib.as_array((ctypes.c_uint8 * nbytes).from_address(addr))

    def allreduce(user, buf, count):
        try:
            if count > 0:
                comm.allreduce_sum_i64(np.ctypeslib.as_array(buf, shape=(count,)))
            return 0
        except Exception:
            return 1

    def alltoallv(user, send, sb, sd, recv, rb, rd):
        try:
            sbn, sdn = np.ctypeslib.as_array(sb, shape=(size,)), np.ctypeslib.as_array(sd, shape=(size,))
            rbn, rdn = np.ctypeslib.as_array(rb, shape=(size,)), np.ctypeslib.as_array(rd, shape=(size,))
            comm.alltoallv(_view(send, int((sbn + sdn).max(initial=0))), sbn, sdn,
                           _view(recv, int((rbn + rdn).max(initial=0))), rbn, rdn)
            return 0
        except Exception:
            return 1

    f1, f2 = _ALLREDUCE(allreduce), _ALLTOALLV(alltoallv)
    return _Comm(None, f1, f2), (f1, f2)


class Partition:
    """pbcg_part_*: this rank's block of a row-partitioned system.

    comm has .size and the two collectives (paper_2404_13216_gb300.comm);
    row_ptr, col_idx (global columns) and vals hold the block's rows
    row_starts[rank] .. row_starts[rank+1] - 1.  Creation and solve are
    collective: every rank calls them in the same order."""

    def __init__(self, ctx: "Context", comm, row_starts, row_ptr, col_idx, vals):
        rs = np.ascontiguousarray(row_starts, dtype=np.int32)
        nranks, rank = int(comm.size), int(comm.rank)
        if rs.size != nranks + 1:
            raise ValueError(f"row_starts has {rs.size} entries, expected {nranks + 1}")
        rp, ci, va, n, nnz = _csr(row_ptr, col_idx, vals)
        if n != int(rs[rank + 1] - rs[rank]):
            raise ValueError(f"the block has {n} rows, row_starts gives {int(rs[rank + 1] - rs[rank])}")
        self._ccomm, self._keep = _c_comm(comm)
        h = ctypes.c_void_p()
        ctx._check(_lib.pbcg_part_create(ctx.handle, ctypes.byref(self._ccomm), nranks, rank, _ptr(rs), nnz,
                                         _ptr(rp), _ptr(ci), _ptr(va), ctypes.byref(h)))
        self.ctx, self.handle, self.n, self.rank, self.nranks = ctx, h, n, rank, nranks

    def solve(self, b, x, tol: float, maxit: int, alg: int = PIPELINED, mode: int = EXACT) -> Result:
        """Solve in place over all ranks: x holds this rank's block of x0 on entry
        and of the last iterate on return."""
        b, x = _vec_in(b, self.n, "b"), _vec_out(x, self.n, "x")
        r = _Result()
        self.ctx._check(_lib.pbcg_part_solve(self.handle, _ptr(b), _ptr(x), float(tol), int(maxit), int(alg),
                                             int(mode), ctypes.byref(r)))
        return Result(r.status, r.iters, r.relres_recursive, r.relres_true, r.seconds, r.launches)

    def close(self):
        if self.handle:
            _lib.pbcg_part_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
