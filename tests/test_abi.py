"""The C-ABI library builds, loads and exports every entry point include/pbcg.h declares.
No compute calls here: these run without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pbcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pbcg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_13216_gb300 import build
    path = build.build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("pbcg_create", "pbcg_csr_upload", "pbcg_solve", "pbcg_solve_batched", "pbcg_residual_history",
              "pbcg_destroy", "pbcg_last_error"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_lists_every_symbol():
    from paper_2404_13216_gb300 import pbcg
    assert sorted(pbcg.EXPORTS) == declared_symbols()


def test_null_handling_without_gpu(lib):
    lib.pbcg_destroy.argtypes = [ctypes.c_void_p]
    lib.pbcg_destroy(None)                       # no-op
    lib.pbcg_last_error.restype = ctypes.c_char_p
    lib.pbcg_last_error.argtypes = [ctypes.c_void_p]
    assert lib.pbcg_last_error(None) == b"no context"
    lib.pbcg_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.pbcg_create(None, 0, None) == -1  # INVALID: out == NULL
    lib.pbcg_solve.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_double, ctypes.c_int32, ctypes.c_int,
                                                       ctypes.c_int, ctypes.c_void_p]
    assert lib.pbcg_solve(None, None, None, None, 1e-8, 10, 1, 1, None) == -1


def test_create_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.pbcg_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
    assert lib.pbcg_create(ctypes.byref(h), 0, None) < 0
    assert not h.value


def test_null_handles_rejected_before_cuda(lib):
    """Every entry point answers a NULL handle (or, for pbcg_dot_noalloc,
    bad arguments) with PBCG_ERR_INVALID before any CUDA call; the destroy
    calls take NULL as a no-op; pbcg_last_error(NULL) names the problem."""
    P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    INVALID = -1
    lib.pbcg_last_error.restype = ctypes.c_char_p
    lib.pbcg_last_error.argtypes = [P]
    assert lib.pbcg_last_error(None) == b"no context"
    lib.pbcg_destroy.argtypes = [P]
    lib.pbcg_destroy(None)
    lib.pbcg_pool_destroy.argtypes = [P]
    lib.pbcg_pool_destroy(None)
    calls = [
        ("pbcg_create", [P, ctypes.c_int, P], (None, 0, None)),
        ("pbcg_csr_upload", [P, i32, i64, P, P, P, ctypes.c_int, P], (None, 1, 0, None, None, None, 0, None)),
        ("pbcg_mat_free", [P, P], (None, None)),
        ("pbcg_solve", [P, P, P, P, d, i32, ctypes.c_int, ctypes.c_int, P],
         (None, None, None, None, 1e-8, 10, 1, 1, None)),
        ("pbcg_solve_batched", [P, P, i32, P, P, P, P, i32, ctypes.c_int, ctypes.c_int, P],
         (None, None, 1, None, None, None, None, 10, 1, 1, None)),
        ("pbcg_residual_history", [P, i32, P, i32, P], (None, 0, None, 0, None)),
        ("pbcg_set_option", [P, ctypes.c_int, i64], (None, 1, 5)),
        ("pbcg_dot", [P, i64, P, P, ctypes.c_int, P], (None, 0, None, None, 1, None)),
        ("pbcg_spmv", [P, P, P, P], (None, None, None, None)),
        ("pbcg_check_wait", [P, i32, P, P], (None, 16, None, None)),
        ("pbcg_pool_create", [P, P, P], (None, None, None)),
        ("pbcg_pool_admit", [P, i32, i64, P, P, P, P, P, d, i32, P],
         (None, 1, 0, None, None, None, None, None, 1e-8, 10, None)),
        ("pbcg_pool_step", [P, i32], (None, 1)),
        ("pbcg_pool_poll", [P, ctypes.c_int, P, i32, P, P], (None, 0, None, 0, None, None)),
        ("pbcg_pool_result", [P, i32, P, P], (None, 0, None, None)),
        ("pbcg_pool_history", [P, i32, P, i32, P], (None, 0, None, 0, None)),
        ("pbcg_pool_room", [P, P, P, P], (None, None, None, None)),
    ]
    for name, argtypes, args in calls:
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = argtypes, ctypes.c_int
        assert fn(*args) == INVALID, name
    noalloc = lib.pbcg_dot_noalloc
    noalloc.argtypes, noalloc.restype = [i64, P, P, ctypes.c_int, P, P], ctypes.c_int
    out = ctypes.c_double(0.0)
    assert noalloc(-1, None, None, 1, ctypes.byref(out), None) == INVALID          # n < 0
    assert noalloc(1 << 31, None, None, 1, ctypes.byref(out), None) == INVALID     # n beyond 2^31 - 1
    assert noalloc(4, None, None, 1, ctypes.byref(out), None) == INVALID           # NULL operands
    assert noalloc(0, None, None, 7, ctypes.byref(out), None) == INVALID           # unknown dot mode


def test_create_without_a_device_fails_cleanly(lib):
    """On a machine with no GPU, pbcg_create returns an error and leaves *out NULL."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is visible")
    except ImportError:
        pass
    lib.pbcg_create.argtypes, lib.pbcg_create.restype = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int
    out = ctypes.c_void_p(1234)
    assert lib.pbcg_create(ctypes.byref(out), 0, None) < 0
    assert out.value is None
