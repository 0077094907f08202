"""The C-ABI library loads and exports every entry point include/fpic.h
declares (no compute calls; runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:\w+\s+)+\**\s*(fpic_\w+)\s*\(", src, re.M))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = _declared()
    for required in ["fpic_init_metric", "fpic_push", "fpic_hamiltonian", "fpic_set_grid"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2602_07452_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_header_symbol():
    from paper_2602_07452_gb300 import fpic
    assert set(_declared()) == set(fpic.declared_symbols())
