"""The C ABI library builds for sm_103a and exports every function include/qbx.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?(?:int|void|const char\s*\*)\s*\*?\s*(qbx_\w+)\s*\(", src, re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("qbx_build_tree", "qbx_build_lists", "qbx_eval", "qbx_tree_query", "qbx_tree_free",
              "qbx_lists_free", "qbx_lists_cost", "qbx_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1805_06106_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path, mode=os.RTLD_NOW)  # every symbol the library needs resolves at load
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
