"""GPU parity with constant enrichment weights (l = 0, one coefficient per component and wall cell,
the setting of the paper's simulations, Sec. 5.1): every velocity operator and nu_t element by
element against the FP64 oracle built with l = 0, on channel and bump meshes, and the Helmholtz
solve checked with the oracle's own l = 0 operators."""
import numpy as np
import pytest

import oracle as O
from paper_1705_08813_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


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
    om = O.Mesh(**w.mesh_kwargs(), enrich_l=0,
                **{k: v for k, v in kw.items() if k in ("n_layers", "q_wall", "wall_law")})
    gm = dgw.mesh_for(w, enrich_l=0, **kw)
    assert (gm.n_p, gm.n_u, gm.n_e) == (om.n_p, om.n_u, om.n_e)
    assert gm.n_u == 3 * gm.n_p + 3 * gm.n_e
    return om, gm


def _velocity(om, w, n_layers=1):
    u = I.workload_velocity(om.node_coords(), om.n_e, w, n_layers=n_layers, nef=1)
    # perturb all three enrichment components so that every coefficient reaches the outputs
    u[3 * om.n_p:] += 0.2 * w.u_tau * I.uniform(w.seed, 3 * om.n_e, -1.0, 1.0, stream=61)
    return u


CASES = [
    ("c1_q2_8x8x8", I.WORKLOADS["channel_q2_8x8x8"], {}),
    ("ragged_q3_5x3x2_vandriest", I.Workload("r3", 5, 3, 2, 3, 395.0, 1.0 / 6000.0, seed=12), {"wall_law": 1}),
    ("q4_two_layers_qwall_5", I.Workload("r8", 3, 4, 3, 4, 590.0, 1.0 / 12000.0, seed=17), {"q_wall": 5, "n_layers": 2}),
    ("q2_single_cells_1x2x1", I.Workload("r6", 1, 2, 1, 2, 180.0, 1.0 / 3250.0, seed=15), {}),
    ("bump_q3_6x4x3", I.bump_workload("b2", 6, 4, 3, 3, seed=22), {}),
    ("bump_q2_5x4x2_ragged", I.bump_workload("b5", 5, 4, 2, 2, seed=25), {}),
]


@pytest.mark.parametrize("name,w,kw", CASES, ids=[c[0] for c in CASES])
def test_l0_operators_match_oracle(dgw, name, w, kw):
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, kw.get("n_layers", 1))
    ud = torch.tensor(u, device=dev)
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    _cmp(gm.divergence(ud, b).cpu().numpy(), om.divergence(u), TOL64, "divergence")
    refc = om.convective(u)
    yc = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    _cmp(gm.convective(ud, yc).cpu().numpy(), refc, TOL64, "convective fp64")
    yc32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.convective(ud.float(), yc32).cpu().numpy(), refc, TOL32, "convective fp32")
    # viscous with nu_t frozen from u, applied to a different vector
    gm.update_eddy_viscosity(ud)
    v = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=62)
    vd = torch.tensor(v, device=dev)
    refv = om.viscous(u, v)
    yv = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    _cmp(gm.viscous(vd, yv).cpu().numpy(), refv, TOL64, "viscous fp64")
    yv32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.viscous(vd.float(), yv32).cpu().numpy(), refv, TOL32, "viscous fp32")
    refm = om.vmass(v)
    ym = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    _cmp(gm.mass(vd, ym).cpu().numpy(), refm, TOL64, "mass fp64")


HELM_CASES = [
    ("channel_q2", I.WORKLOADS["channel_q2_8x8x8"], 1.5e3),
    ("channel_q4_4x6x3", I.Workload("h4", 4, 6, 3, 4, 590.0, 1.0 / 12000.0, seed=13), 3.0e2),
    ("bump_q2_8x4x2", I.bump_workload("hb", 8, 4, 2, 2, seed=21), 5.0e2),
]


@pytest.mark.parametrize("name,w,gamma", HELM_CASES, ids=[c[0] for c in HELM_CASES])
def test_l0_helmholtz_solve_residual_checked_by_oracle(dgw, name, w, gamma):
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u_hat = _velocity(om, w)
    gm.update_eddy_viscosity(torch.tensor(u_hat, device=dev))
    rhs = gamma * om.vmass(u_hat)
    u = torch.tensor(u_hat, device=dev)
    info = gm.helmholtz_solve(gamma, torch.tensor(rhs, device=dev), u, rtol=1e-10, max_iter=2000, restart=30)
    uh = u.cpu().numpy()
    res = rhs - (gamma * om.vmass(uh) + om.viscous(u_hat, uh))
    rel = np.linalg.norm(res) / np.linalg.norm(rhs)
    assert info["rel_residual"] <= 1e-10 and rel <= 1.5e-10, (info, rel)


def test_enrich_l_outside_range_rejected(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    with pytest.raises(dgw.DGWError):
        dgw.mesh_for(w, enrich_l=2)
