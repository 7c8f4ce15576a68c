"""GPU parity for the viscous step of the dual-splitting scheme: the velocity mass operator
element by element against the FP64 oracle (standard and enriched DoFs, channel and bump), and the
Helmholtz solve gamma M u - F^nu(u) = rhs (eq. helmholtzspat) whose returned u is checked with the
oracle's own mass and viscous operators to the requested relative residual."""
import numpy as np
import pytest

import oracle as O
from paper_1705_08813_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


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


def _meshes(dgw, w, **kw):
    om = O.Mesh(**w.mesh_kwargs(), **{k: v for k, v in kw.items() if k in ("n_layers", "q_wall", "wall_law")})
    gm = dgw.mesh_for(w, **kw)
    assert (gm.n_p, gm.n_u, gm.n_e) == (om.n_p, om.n_u, om.n_e)
    return om, gm


MASS_CASES = [
    ("c1_q2_8x8x8", I.WORKLOADS["channel_q2_8x8x8"], {}),
    ("ragged_q3_5x3x2", I.Workload("r3", 5, 3, 2, 3, 395.0, 1.0 / 6000.0, seed=12), {}),
    ("q4_qwall_5_vandriest", I.Workload("r8", 3, 4, 3, 4, 590.0, 1.0 / 12000.0, seed=17), {"q_wall": 5, "wall_law": 1}),
    ("q3_no_enrichment", I.Workload("r7", 4, 3, 3, 3, 180.0, 1.0 / 3250.0, seed=16), {"n_layers": 0}),
    ("bump_q3_6x4x3", I.bump_workload("b2", 6, 4, 3, 3, seed=22), {}),
]


@pytest.mark.parametrize("name,w,kw", MASS_CASES, ids=[c[0] for c in MASS_CASES])
def test_mass_matches_oracle(dgw, name, w, kw):
    om, gm = _meshes(dgw, w, **kw)
    u = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=41)
    ref = om.vmass(u)
    ud = torch.tensor(u, device="cuda")
    y = torch.empty_like(ud)
    _cmp(gm.mass(ud, y).cpu().numpy(), ref, TOL64, "mass fp64")
    y32 = torch.empty(gm.n_u, dtype=torch.float32, device="cuda")
    _cmp(gm.mass(ud.float(), y32).cpu().numpy(), ref, TOL32, "mass fp32")


HELM_CASES = [
    ("channel_q2_dt1e-3", I.WORKLOADS["channel_q2_8x8x8"], 1.5e3),
    ("channel_q2_small_gamma", I.WORKLOADS["channel_q2_8x8x8"], 20.0),
    ("channel_q4_4x6x3", I.Workload("h4", 4, 6, 3, 4, 590.0, 1.0 / 12000.0, seed=13), 3.0e2),
    ("bump_q2_8x4x2", I.bump_workload("hb", 8, 4, 2, 2, seed=21), 5.0e2),
]


@pytest.mark.parametrize("name,w,gamma", HELM_CASES, ids=[c[0] for c in HELM_CASES])
def test_helmholtz_solve_residual_checked_by_oracle(dgw, name, w, gamma):
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u_hat = I.workload_velocity(om.node_coords(), om.n_e, w)
    gm.update_eddy_viscosity(torch.tensor(u_hat, device=dev))
    rhs = gamma * om.vmass(u_hat)
    u = torch.tensor(u_hat, device=dev)   # initial guess: the projected velocity
    info = gm.helmholtz_solve(gamma, torch.tensor(rhs, device=dev), u, rtol=1e-10, max_iter=2000, restart=30)
    uh = u.cpu().numpy()
    res = rhs - (gamma * om.vmass(uh) + om.viscous(u_hat, uh))
    rel = np.linalg.norm(res) / np.linalg.norm(rhs)
    assert info["rel_residual"] <= 1e-10 and rel <= 1.5e-10, (info, rel)
    assert info["iterations"] > 0


def test_helmholtz_reports_nonconvergence(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u_hat = I.workload_velocity(om.node_coords(), om.n_e, w)
    gm.update_eddy_viscosity(torch.tensor(u_hat, device=dev))
    rhs = torch.tensor(20.0 * om.vmass(u_hat), device=dev)
    u = torch.zeros_like(rhs)
    info = gm.helmholtz_solve(20.0, rhs, u, rtol=1e-14, max_iter=3, restart=30, check=False)
    assert info["status"] == -3 and info["iterations"] == 3
    with pytest.raises(dgw.DGWError):
        gm.helmholtz_solve(-1.0, rhs, u)
