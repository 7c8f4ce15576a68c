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


def test_null_handles_and_bad_options_are_rejected_without_a_device(lib):
    """Every entry point checks its arguments before it touches the device: null handles and invalid
    options return DGW_EINVAL with a message naming the call."""
    from paper_1705_08813_gb300 import dgw
    L = dgw.load()
    vp = ctypes.c_void_p
    calls = {
        "dgw_apply_mass": lambda: L.dgw_apply_mass(None, 0, None, None, None),
        "dgw_apply_gradient": lambda: L.dgw_apply_gradient(None, None, None, None),
        "dgw_apply_divdiv": lambda: L.dgw_apply_divdiv(None, None, None, None, None),
        "dgw_tau_divdiv": lambda: L.dgw_tau_divdiv(None, None, ctypes.c_double(1e-3), ctypes.c_double(0.14), None, None),
        "dgw_apply_curl": lambda: L.dgw_apply_curl(None, None, None, None),
        "dgw_apply_inverse_mass": lambda: L.dgw_apply_inverse_mass(None, None, None, None),
        "dgw_wall_shear_stress": lambda: L.dgw_wall_shear_stress(None, None, None, None),
        "dgw_set_wall_shear_stress": lambda: L.dgw_set_wall_shear_stress(None, None, None),
        "dgw_project_velocity": lambda: L.dgw_project_velocity(None, None, None, None, None),
        "dgw_set_enrichment_switch": lambda: L.dgw_set_enrichment_switch(None, ctypes.c_double(30.0), None),
        "dgw_enrichment_active": lambda: L.dgw_enrichment_active(None, None, None, None),
        "dgw_add_pressure_neumann": lambda: L.dgw_add_pressure_neumann(None, None, None, ctypes.c_double(1.0), None,
                                                                       None, ctypes.c_double(0.0), None, None, None),
        "dgw_ns_step": lambda: L.dgw_ns_step(None, None, None),
        "dgw_ns_state": lambda: L.dgw_ns_state(None, None, None, None),
        "dgw_ns_copy_state": lambda: L.dgw_ns_copy_state(None, None, None, None),
        "dgw_ns_create": lambda: L.dgw_ns_create(None, None, None, None, ctypes.byref(vp())),
        "dgw_helmholtz_solve": lambda: L.dgw_helmholtz_solve(None, ctypes.c_double(1.0), None, None, None, None, None),
        "dgw_mesh_destroy": lambda: L.dgw_mesh_destroy(None),
        "dgw_mesh_info": lambda: L.dgw_mesh_info(None, None, None, None, None),
        "dgw_mesh_node_coords": lambda: L.dgw_mesh_node_coords(None, None),
        "dgw_update_eddy_viscosity": lambda: L.dgw_update_eddy_viscosity(None, None, None),
        "dgw_apply_laplace": lambda: L.dgw_apply_laplace(None, 0, None, None, None),
        "dgw_apply_divergence": lambda: L.dgw_apply_divergence(None, None, None, None),
        "dgw_apply_divergence_prec": lambda: L.dgw_apply_divergence_prec(None, 0, None, None, None),
        "dgw_apply_convective": lambda: L.dgw_apply_convective(None, 0, None, None, None),
        "dgw_apply_viscous": lambda: L.dgw_apply_viscous(None, 0, None, None, None),
        "dgw_cfl_rate": lambda: L.dgw_cfl_rate(None, None, None, None),
        "dgw_pressure_solve": lambda: L.dgw_pressure_solve(None, None, None, None, None, None),
        "dgw_pressure_solve_batch": lambda: L.dgw_pressure_solve_batch(None, 1, None, None, None, None, None),
        "dgw_pressure_solve_jacobi_noalloc": lambda: L.dgw_pressure_solve_jacobi_noalloc(
            None, None, None, ctypes.c_double(1e-10), 10, None, None),
        "dgw_solver_describe": lambda: L.dgw_solver_describe(None, 1, None, None, None, 0, None),
        "dgw_server_create": lambda: L.dgw_server_create(ctypes.c_size_t(1 << 30), 0, ctypes.byref(vp())),
        "dgw_submit": lambda: L.dgw_submit(None, None, None),
        "dgw_poll": lambda: L.dgw_poll(None, ctypes.c_long(1), None, None, None),
        "dgw_server_stats": lambda: L.dgw_server_stats(None, None, None, None, None),
        "dgw_server_destroy": lambda: L.dgw_server_destroy(None, 0),
    }
    for name, call in calls.items():
        assert call() == -1, name
        assert name.encode() in L.dgw_last_error(), (name, L.dgw_last_error())


def test_mesh_options_are_validated_without_a_device(lib):
    """enrich_l outside {0, 1}, full_quadrature outside {0, 1} and q_wall outside 1..10 are rejected
    by dgw_mesh_create before any device work."""
    from paper_1705_08813_gb300 import dgw
    L = dgw.load()
    bad = [
        (dgw.MeshParams(4, 4, 4, 2, 2, 8, 0, 0, 1, 6.28, 2.0, 3.14, 1.8, 1e-3, 1e-2, 3, 0), b"enrich_l"),
        (dgw.MeshParams(4, 4, 4, 2, 1, 8, 0, 0, 1, 6.28, 2.0, 3.14, 1.8, 1e-3, 1e-2, 3, 2), b"full_quadrature"),
        (dgw.MeshParams(4, 4, 4, 2, 1, 11, 1, 0, 1, 9.0, 3.036, 4.5, 1.8, 1e-3, 1e-2, 3, 1), b"q_wall"),
    ]
    for p, word in bad:
        h = ctypes.c_void_p()
        assert L.dgw_mesh_create(ctypes.byref(p), None, ctypes.byref(h)) == -1 and not h.value
        assert word in L.dgw_last_error(), L.dgw_last_error()
