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
