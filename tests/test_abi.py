"""The C-ABI library loads, exports every symbol include/flashnav.h declares,
and rejects bad arguments before touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(nav_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def fn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import flashnav
    return flashnav


def test_every_declared_symbol_is_exported(fn):
    lib = fn.load()
    declared = _declared("flashnav.h")
    assert declared, "no declarations parsed"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(fn.EXPORTS)


def test_default_params_are_table7(fn):
    p = fn.params_struct(None)
    assert p.dt == pytest.approx(0.1) and p.goal_tol == pytest.approx(0.2)
    assert p.c_progress == 2.0 and p.r_goal == 10.0 and p.r_coll == 10.0
    assert p.horizon == 200 and p.fov_deg == 360.0


def _maps(occ):
    m = (fn_mod().nav_map * 1)()
    m[0] = fn_mod().nav_map(occ.shape[1], occ.shape[0], 0.05, occ.ctypes.data)
    return m


def fn_mod():
    from paper_2606_15846_b300 import flashnav
    return flashnav


def _robot(shape=0, radius=0.18, length=0.0, width=0.0):
    return fn_mod().nav_robot(shape, radius, length, width, 0.0, 0.5, -1.0, 1.0)


def test_bad_arguments_are_rejected_on_the_host(fn):
    lib = fn.load()
    occ = np.zeros((32, 32), np.uint8)
    maps = _maps(occ)
    h = C.c_void_p()
    r = _robot()
    assert lib.nav_create(maps, 1, 0, 8, 2.0, C.byref(r), None, C.byref(h)) == -1
    assert lib.nav_create(maps, 1, 4, 0, 2.0, C.byref(r), None, C.byref(h)) == -1
    assert lib.nav_create(maps, 1, 4, 8, -1.0, C.byref(r), None, C.byref(h)) == -1
    assert lib.nav_create(None, 1, 4, 8, 2.0, C.byref(r), None, C.byref(h)) == -1
    bad = _robot(radius=-0.1)
    assert lib.nav_create(maps, 1, 4, 8, 2.0, C.byref(bad), None, C.byref(h)) == -1
    p = fn.params_struct(None)
    p.n_dyn = 99
    assert lib.nav_create(maps, 1, 4, 8, 2.0, C.byref(r), C.byref(p), C.byref(h)) == -1
    assert not h.value
    assert lib.nav_step(None, None, None, None, None, None) == -1
    assert lib.nav_reset(None, 0, None) == -1


def test_map_without_free_cell_reports_nospawn(fn):
    lib = fn.load()
    occ = np.ones((16, 16), np.uint8)
    maps = _maps(occ)
    h = C.c_void_p()
    r = _robot()
    assert lib.nav_create(maps, 1, 4, 8, 2.0, C.byref(r), None, C.byref(h)) == -4
    assert not h.value
