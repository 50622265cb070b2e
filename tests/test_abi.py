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


def test_workspace_checks_the_mobility_and_force_options_without_gpu(libpath):
    import numpy as np
    import paper_2106_00449_gb300 as g
    lib = g.load_library()
    n = np.array([3], dtype=np.int32)
    off1, bt1 = np.array([0, 2], dtype=np.int64), np.array([0, 0], dtype=np.int32)
    off2, bt2 = np.array([0, 1, 2], dtype=np.int64), np.array([0, 0], dtype=np.int32)

    def ws(params, off=off1, bt=bt1):
        c = params._c()
        return lib.gdc_workspace_bytes(ctypes.byref(c), 1, g._np_ptr(n), len(off) - 1, g._np_ptr(off), g._np_ptr(bt))

    fcm = dict(mobility=g.MOB_FCM, box_L=20.0, fcm_N=64)
    assert ws(g.Params(**fcm)) > ws(g.Params())                     # the FCM grids live in the workspace
    assert ws(g.Params(**fcm), off2, bt2) == 0                      # one suspension only
    # pair forces in the periodic cube need a side of 3 cutoffs (soft sphere 2a + 36 b = 5.6a here)
    assert ws(g.Params(rep_A=4.0, **fcm)) > 0
    assert ws(g.Params(rep_A=4.0, **dict(fcm, box_L=15.0))) == 0
    assert ws(g.Params(potential=1, well_A=5.0, **fcm)) > 0          # wells: 3a + 6 lambda = 6a
    assert ws(g.Params(shear_rate=1.0, **fcm)) == 0                 # linear shear is not periodic
    assert ws(g.Params(**dict(fcm, fcm_N=48))) == 0                 # not a power of two
    assert ws(g.Params(**dict(fcm, box_L=5.0))) == 0                # 3a truncation reaches the image
    assert ws(g.Params(mobility=2)) == 0
    # pair potentials and the pair search
    assert ws(g.Params(potential=2, well_A=5.0, well_lambda=0.5, force_method=2)) > 0
    assert ws(g.Params(potential=3)) == 0
    assert ws(g.Params(potential=1, well_A=5.0, well_lambda=0.0)) == 0
    assert ws(g.Params(force_method=3)) == 0
    assert ws(g.Params(well_A=-1.0)) == 0
    # blobs above a wall: per-body blocks enlarge the workspace; RPY only, no shear
    wall = dict(wall=1, wall_V0=23.0, wall_b=0.5, body_weight=0.18)
    assert ws(g.Params(**wall)) > ws(g.Params())
    assert ws(g.Params(**dict(wall, wall_b=0.0))) == 0
    assert ws(g.Params(**dict(wall, wall_V0=-1.0))) == 0
    assert ws(g.Params(**dict(wall, shear_rate=1.0))) == 0
    assert ws(g.Params(**dict(wall, **fcm))) == 0
    assert ws(g.Params(wall_V0=23.0)) == 0                        # wall forces without the wall
    assert ws(g.Params(lanczos_precond=2)) == 0
    # the double-float residual kernel: ordered (1) or symmetric at 3 or 4 blocks per SM
    for k in (0, 1, 3, 4):
        assert ws(g.Params(df_kernel=k)) > 0
    assert ws(g.Params(df_kernel=2)) == 0


def test_fcm_workspace_checks_the_grid_without_gpu(libpath):
    import paper_2106_00449_gb300 as g
    lib = g.load_library()

    def ws(*a):
        p = g._FcmParams(*a)
        return lib.gdc_fcm_workspace_bytes(ctypes.byref(p))

    good = ws(64, 20.0, 0.5642, 3.0, 1.0, 100)
    assert good > 13 * 64 ** 3 * 8                   # nine complex and two packed grids
    assert ws(63, 20.0, 0.5642, 3.0, 1.0, 100) == 0
    assert ws(1024, 20.0, 0.5642, 3.0, 1.0, 100) == 0
    assert ws(64, 20.0, 0.5642, 10.0, 1.0, 100) == 0    # R_t >= L/2
    assert ws(512, 20.0, 0.5642, 3.0, 1.0, 100) == 0    # R_t beyond 15 grid spacings (h = L/512)
    assert ws(64, 20.0, 0.5642, 3.0, 0.0, 100) == 0
    assert ws(64, 20.0, 0.5642, 3.0, 1.0, 0) == 0
