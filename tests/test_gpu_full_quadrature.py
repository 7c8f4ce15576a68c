"""GPU parity under the paper-literal enriched quadrature (Sec. 4.4: q_w Gauss points in every
direction of the enriched cells, q_w per tangential direction on faces touching them): every
velocity operator, the wall shear stress, the L2 projection and dual-splitting steps against the
oracle built with the same rule, on channel meshes and on curved bump meshes (whose metric is then
also tabulated at the q_w^2 in-plane points of the enriched cells)."""
import numpy as np
import pytest

import oracle as O
from paper_1705_08813_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def dgw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_08813_gb300 import dgw as d
    assert torch.cuda.is_available()
    return d


def _cmp(y, ref, tol, what):
    y = np.asarray(y, dtype=np.float64)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    ele = np.abs(y - ref).max() / np.abs(ref).max()
    assert rel <= tol and ele <= tol, f"{what}: rel {rel:.3e} elem {ele:.3e}"


KEYS = ("n_layers", "q_wall", "wall_law", "enrich_l")


def _meshes(dgw, w, **kw):
    om = O.Mesh(**w.mesh_kwargs(), full_quadrature=True, **{k: v for k, v in kw.items() if k in KEYS})
    gm = dgw.mesh_for(w, full_quadrature=True, **kw)
    assert (gm.n_p, gm.n_u, gm.n_e) == (om.n_p, om.n_u, om.n_e)
    return om, gm


def _velocity(om, w, kw):
    nef = 1 if kw.get("enrich_l", 1) == 0 else 8
    u = I.workload_velocity(om.node_coords(), om.n_e, w, n_layers=kw.get("n_layers", 1), nef=nef)
    u[3 * om.n_p:] += 0.2 * w.u_tau * I.uniform(w.seed, u.size - 3 * om.n_p, -1.0, 1.0, stream=91)
    return u


CASES = [
    ("c1_q2_8x8x8", I.WORKLOADS["channel_q2_8x8x8"], {}),
    ("ragged_q3_5x3x2_qwall_10", I.Workload("f3", 5, 3, 2, 3, 395.0, 1.0 / 6000.0, seed=92), {"q_wall": 10}),
    ("q4_two_layers_l0_vandriest", I.Workload("f4", 3, 4, 3, 4, 590.0, 1.0 / 12000.0, seed=93),
     {"n_layers": 2, "enrich_l": 0, "wall_law": 1}),
    ("bump_q3_6x4x3", I.bump_workload("fb3", 6, 4, 3, 3, seed=102), {}),
    ("bump_q2_5x4x2_qwall_10_l0", I.bump_workload("fb2", 5, 4, 2, 2, seed=103), {"q_wall": 10, "enrich_l": 0}),
    ("bump_q4_4x4x2_two_layers_vandriest", I.bump_workload("fb4", 4, 4, 2, 4, seed=104),
     {"n_layers": 2, "wall_law": 1}),
]


@pytest.mark.parametrize("name,w,kw", CASES, ids=[c[0] for c in CASES])
def test_operators_match_oracle(dgw, name, w, kw):
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, kw)
    ud = torch.tensor(u, device=dev)
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    _cmp(gm.divergence(ud, b).cpu().numpy(), om.divergence(u), TOL64, "divergence")
    y = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    refc = om.convective(u)
    _cmp(gm.convective(ud, y).cpu().numpy(), refc, TOL64, "convective")
    # a random field: the normal velocity changes sign on every face, so the Lax-Friedrichs flux is not
    # polynomial there and each face's point rule matters (the faces above the enriched layer)
    ur = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=101)
    _cmp(gm.convective(torch.tensor(ur, device=dev), y).cpu().numpy(), om.convective(ur), TOL64, "convective (random)")
    y32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.convective(ud.float(), y32).cpu().numpy(), refc, 2e-5, "convective fp32")
    gm.update_eddy_viscosity(ud)
    v = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=94)
    vd = torch.tensor(v, device=dev)
    _cmp(gm.viscous(vd, y).cpu().numpy(), om.viscous(u, v), TOL64, "viscous")
    _cmp(gm.mass(vd, y).cpu().numpy(), om.vmass(v), TOL64, "mass")
    p = I.uniform(w.seed, om.n_p, -1.0, 1.0, stream=95)
    _cmp(gm.gradient(torch.tensor(p, device=dev), y).cpu().numpy(), om.gradient(p), TOL64, "gradient")
    tau = om.tau_divdiv(u, 2e-3, 0.14)
    td = torch.empty(gm.nc, dtype=torch.float64, device=dev)
    _cmp(gm.tau_divdiv(ud, 2e-3, 0.14, td).cpu().numpy(), tau, TOL64, "tau_D")
    _cmp(gm.divdiv(torch.tensor(tau, device=dev), vd, y).cpu().numpy(), om.divdiv(tau, v), TOL64, "div-div")
    _cmp(gm.curl(ud, y).cpu().numpy(), om.curl(u), TOL64, "curl")
    tn = torch.empty(gm.n_wall_nodes, dtype=torch.float64, device=dev)
    _cmp(gm.wall_shear_stress(ud, tn).cpu().numpy(), om.wall_shear(u), TOL64, "tau_w,B")
    # a varying nodal tau_w makes grad psi vary over the wall faces, which the wall-face rule must follow
    tv = w.tau_w * (1.0 + 0.5 * I.uniform(w.seed, om.n_wall_nodes, -1.0, 1.0, stream=99))
    om.set_tau_nodes(tv)
    gm.set_wall_shear_stress(torch.tensor(tv, device=dev))
    _cmp(gm.wall_shear_stress(ud, tn).cpu().numpy(), om.wall_shear(u), TOL64, "tau_w,B (varying tau_w)")
    w0 = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=100)
    base = np.zeros(om.n_p)
    ref = om.pressure_neumann(u, w0, 1.5, f=(0.1, 0.0, 0.0))
    b = torch.tensor(base, device=dev)
    gm.add_pressure_neumann(b, ud, torch.tensor(w0, device=dev), 1.5, force=(0.1, 0.0, 0.0))
    _cmp(b.cpu().numpy(), ref, TOL64, "pressure Neumann data (varying tau_w)")
    gm.update_eddy_viscosity(ud)
    _cmp(gm.viscous(vd, y).cpu().numpy(), om.viscous(u, v), TOL64, "viscous (varying tau_w)")


def _l2(om, d, ref):
    return float(np.sqrt(abs(d @ om.vmass(d)) / (ref @ om.vmass(ref))))


STEP_CASES = [
    ("channel_q2_4x4x2", I.Workload("fs", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=96)),
    ("bump_q2_6x4x2", I.bump_workload("fsb", 6, 4, 2, 2, seed=105)),
]


@pytest.mark.parametrize("name,w", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_projection_and_time_steps_match_oracle(dgw, name, w):
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, {})
    tn = w.tau_w * (1.0 + 0.4 * I.uniform(w.seed, om.n_wall_nodes, -1.0, 1.0, stream=97))
    ref = om.project(tn, u)
    un = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    gm.project_velocity(torch.tensor(tn, device=dev), torch.tensor(u, device=dev), un)
    got = un.cpu().numpy()
    assert _l2(om, got - ref, ref) < 1e-9
    om2, gm2 = _meshes(dgw, w)
    u0 = I.workload_velocity(om2.node_coords(), om2.n_e, w)
    force = (w.tau_w / (0.5 * w.ly), 0.0, 0.0)
    ds = O.DualSplitting(om2, u0, dt=2e-3, force=force, rtol=1e-13, high_order_pressure_bc=True)
    ns = dgw.DualSplitting(gm2, torch.tensor(u0, device=dev), dt=2e-3, force=force, rtol_pressure=1e-12,
                           rtol_projection=1e-12, rtol_viscous=1e-12, pressure_mode=0, high_order_pressure_bc=True)
    for _ in range(2):
        ns.step()
        ur, _ = ds.step()
        assert _l2(om2, ns.velocity().cpu().numpy() - ur, ur) < 1e-8

