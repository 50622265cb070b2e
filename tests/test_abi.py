"""The C-ABI library builds, loads and exports every entry point include/gdc.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gdc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gdc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2106_00449_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_lists_the_binding_exports():
    import paper_2106_00449_gb300 as g
    assert _declared() == sorted(g.EXPORTS)


def test_library_exports_every_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_workspace_rejects_bad_input_without_gpu(libpath):
    import numpy as np
    import paper_2106_00449_gb300 as g
    lib = g.load_library()
    p = g.Params()._c()
    n = np.array([3], dtype=np.int32)
    off = np.array([0, 2], dtype=np.int64)
    bt = np.array([0, 0], dtype=np.int32)
    ok = lib.gdc_workspace_bytes(ctypes.byref(p), 1, g._np_ptr(n), 1, g._np_ptr(off), g._np_ptr(bt))
    assert ok > 0
    bad_bt = np.array([0, 5], dtype=np.int32)
    assert lib.gdc_workspace_bytes(ctypes.byref(p), 1, g._np_ptr(n), 1, g._np_ptr(off), g._np_ptr(bad_bt)) == 0
    p2 = g.Params(gmres_restart=1)._c()
    assert lib.gdc_workspace_bytes(ctypes.byref(p2), 1, g._np_ptr(n), 1, g._np_ptr(off), g._np_ptr(bt)) == 0
    empty = np.array([0, 0], dtype=np.int64)
    assert lib.gdc_workspace_bytes(ctypes.byref(p), 1, g._np_ptr(n), 1, g._np_ptr(empty), g._np_ptr(bt)) == 0
