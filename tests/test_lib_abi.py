"""The C ABI library builds for sm_103a, exports every function include/qbx.h declares, and rejects bad
arguments on the host with the documented codes (no GPU)."""
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


def test_host_side_argument_checks_without_a_gpu():
    """Calls that fail their argument checks return the documented error code and message before any
    device work, so they run on a machine without a GPU."""
    if not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1805_06106_gb300 import binding as B

    lib = B.lib()
    err = lambda: lib.qbx_last_error().decode()  # noqa: E731
    buf = (ctypes.c_double * 3)()
    h = ctypes.c_void_p()

    def tree(flags=0, max_depth=40, n_max=32):
        opts = B._TreeOpts(n_max, 0.9, max_depth, flags)
        return lib.qbx_build_tree(buf, 1, None, None, 0, None, 0, ctypes.byref(opts), ctypes.byref(h), None)

    assert tree(flags=4) == -1 and "tree options" in err()           # unknown tree flag
    assert tree(n_max=0) == -1 and "tree options" in err()
    assert tree(max_depth=51) == -4                                   # QBX_ERR_DEPTH
    assert lib.qbx_build_tree(None, 1, None, None, 0, None, 0, ctypes.byref(B._TreeOpts(32, 0.9, 40, 0)),
                              ctypes.byref(h), None) == -1 and "NULL" in err()
    # element marks: NULL tree
    assert lib.qbx_refine_marks(None, 0, None, None, 0, 0.025, None, None) == -1 and "bad argument" in err()
    # evaluation: NULL handles
    opts = B._EvalOpts(5, 10, None, None, B.QBX_M2L_3XTF32 | B.QBX_MIXED_M2L_ONLY)
    assert lib.qbx_eval(None, None, None, None, None, None, None, ctypes.byref(opts), None, None) == -1
