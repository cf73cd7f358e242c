"""The oracle and the CUDA path stay apart, read from the sources (CPU only).

- No module of the package imports the oracle, and the oracle imports nothing
  of the package: the CUDA path cannot fall back to it, and the oracle shares
  no arithmetic with what it checks.  The seeded input generators
  (`inputs.py`) are the one module both sides use, and they import neither.
- No CUDA source includes a file of the oracle, and the oracle's C includes
  only system headers.
- In `bench.py` only the CPU-baseline code (the `cpu_baseline` sample, the
  reference arm and the `--cpu-table` mode) imports the oracle.
- The binding fails loudly, not silently, when the library is missing.
"""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2404_13216_gb300")


def imported_modules(path):
    """Top-level names of every module a Python file imports (anywhere in it)."""
    tree = ast.parse(open(path).read(), path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            if node.level:
                out.add("." + (node.module or ""))
            elif node.module:
                out.add(node.module.split(".")[0])
    return out


def package_files():
    return sorted(os.path.join(PKG, f) for f in os.listdir(PKG) if f.endswith(".py"))


def test_package_never_imports_the_oracle():
    for f in package_files():
        assert "oracle" not in imported_modules(f), f


def test_oracle_imports_nothing_of_the_package():
    mods = imported_modules(os.path.join(ROOT, "oracle", "__init__.py"))
    assert not any(m.startswith("paper_2404_13216_gb300") or m.startswith(".") for m in mods), mods


def test_input_generators_import_neither_side():
    mods = imported_modules(os.path.join(PKG, "inputs.py"))
    assert not mods & {"oracle", "ctypes", "torch"} and not any(m.startswith(".") for m in mods), mods


def test_sources_include_nothing_across_the_line():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        for inc in re.findall(r'#include\s+"([^"]+)"', open(os.path.join(csrc, f)).read()):
            assert "oracle" not in inc, (f, inc)
    quoted = re.findall(r'#include\s+"([^"]+)"', open(os.path.join(ROOT, "oracle", "oracle.c")).read())
    assert quoted == [], quoted


def test_bench_imports_the_oracle_only_for_cpu_baselines():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"oracle_sample", "run_reference", "run_cpu_table"}
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    users.add(fn.name)
    assert users and users <= allowed, users
    top = {a.name for n in tree.body if isinstance(n, ast.Import) for a in n.names}
    assert "oracle" not in top


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2404_13216_gb300 import build
    build.build_library()
    from paper_2404_13216_gb300 import pbcg
    with pytest.raises(RuntimeError, match="missing"):
        pbcg.load_library(str(tmp_path / "libpbcg.so"))
