"""The C ABI: libdgw.so builds for sm_103a, loads, and exports every symbol include/dgw.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dgw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_08813_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["dgw_mesh_create", "dgw_apply_laplace", "dgw_apply_divergence", "dgw_apply_convective",
              "dgw_apply_viscous", "dgw_pressure_solve", "dgw_update_eddy_viscosity", "dgw_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1705_08813_gb300 import dgw
    assert sorted(set(dgw.EXPORTS)) == _declared()


def test_invalid_arguments_fail_without_a_device(lib):
    from paper_1705_08813_gb300 import dgw
    dgw.load()
    p = dgw.MeshParams(4, 4, 4, 9, 1, 8, 0, 0, 1, 6.28, 2.0, 3.14, 1.8, 1e-3, 1e-2, 3)
    h = ctypes.c_void_p()
    st = dgw._lib.dgw_mesh_create(ctypes.byref(p), None, ctypes.byref(h))
    assert st == -1 and not h.value
    assert b"degree" in dgw._lib.dgw_last_error()
