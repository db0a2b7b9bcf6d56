"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every function include/dss.h declares; host-only entry points and
argument validation work with no device present."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nat():
    from paper_2108_01013_gb300 import _native
    _native.build()
    _native.load()
    return _native


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dss_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dss_create", "dss_set_state", "dss_neighbour_build", "dss_force_eval",
                 "dss_step", "dss_stress", "dss_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(nat):
    lib = ctypes.CDLL(nat.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(nat.SIGNATURES) == declared_functions()


def test_capacity_estimate_from_shell_volume(nat):
    lib = nat.load()
    # ((a_max + 2 a0)^3 - a_max^3) / a_min^3, rounded up
    assert lib.dss_capacity_estimate(1.0, 1.4, 1.0) == 37
    assert lib.dss_capacity_estimate(1.0, 10.0, 1.0) == 728
    assert lib.dss_capacity_estimate(1.0, 3.0, 1.0) == 98
    assert lib.dss_capacity_estimate(1.0, 1.0, 1.0) == 26
    assert lib.dss_capacity_estimate(0.0, 1.0, 1.0) == -1
    assert lib.dss_capacity_estimate(2.0, 1.0, 1.0) == -1


def test_create_rejects_bad_arguments_before_touching_cuda(nat):
    from paper_2108_01013_gb300 import default_params
    lib = nat.load()
    h = ctypes.c_void_p()
    box = (ctypes.c_double * 3)(20.0, 20.0, 20.0)
    p = default_params()
    assert lib.dss_create(None, ctypes.byref(p), 100, box, None) == -1
    assert lib.dss_create(ctypes.byref(h), ctypes.byref(p), 1, box, None) == -1
    bad = (ctypes.c_double * 3)(20.0, -1.0, 20.0)
    assert lib.dss_create(ctypes.byref(h), ctypes.byref(p), 100, bad, None) == -1
    q = default_params(dt=-1.0)
    assert lib.dss_create(ctypes.byref(h), ctypes.byref(q), 100, box, None) == -1
    q = default_params(precision=7)
    assert lib.dss_create(ctypes.byref(h), ctypes.byref(q), 100, box, None) == -1
    assert lib.dss_step(None, 1) == -1
    assert lib.dss_strerror(-3) == b"neighbour-list capacity exceeded"
