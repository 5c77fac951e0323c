"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sdcheat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdc_[a-z0-9_]+)\s*\(", src)) - {"sdc_alloc_fn", "sdc_free_fn"})


def test_library_exports_every_declared_symbol():
    from paper_1707_03581_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_1707_03581_gb300 import binding

    assert sorted(binding._SIGS) == _declared()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1707_03581_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "oracle/" not in text, f


def test_solver_refuses_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1707_03581_gb300 import Solver

    with pytest.raises(RuntimeError):
        Solver(0)
