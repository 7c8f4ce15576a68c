"""GPU parity on the curved bump channel (isoparametric Q_k cells, per-point metric tables): every
operator against the FP64 CPU oracle on the same seeded inputs, element by element, and the
pressure solves in all three modes against the oracle's residual. Bar as for the channel:
relative 2-norm and max elementwise error <= 1e-12 (FP64), 1e-5 (FP32, 2e-5 for the nonlinear
vector operators), solves to 1e-10 relative residual."""
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
    return rel


def _meshes(dgw, w, **kw):
    om = O.Mesh(**w.mesh_kwargs(), **{k: v for k, v in kw.items() if k in ("n_layers", "q_wall", "wall_law")})
    gm = dgw.mesh_for(w, **kw)
    assert (gm.n_p, gm.n_u, gm.n_e) == (om.n_p, om.n_u, om.n_e)
    return om, gm


CASES = [
    ("bump_q2_8x4x2", I.bump_workload("b1", 8, 4, 2, 2, seed=21), {}),
    ("bump_q3_6x4x3_ragged", I.bump_workload("b2", 6, 4, 3, 3, seed=22), {}),
    ("bump_q4_8x4x2", I.bump_workload("b3", 8, 4, 2, 4, seed=23), {}),
    ("bump_q1_5x3x2_vandriest", I.bump_workload("b4", 5, 3, 2, 1, seed=24), {"wall_law": 1}),
    ("bump_q2_single_cells_1x2x1", I.bump_workload("b5", 1, 2, 1, 2, seed=25), {}),
    ("bump_q3_no_enrichment", I.bump_workload("b6", 6, 3, 2, 3, seed=26), {"n_layers": 0}),
    ("bump_q2_qwall_5_two_layers", I.bump_workload("b7", 6, 5, 2, 2, seed=27), {"q_wall": 5, "n_layers": 2}),
]


@pytest.mark.parametrize("name,w,kw", CASES, ids=[c[0] for c in CASES])
def test_bump_operators_match_oracle(dgw, name, w, kw):
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    u = I.workload_velocity(om.node_coords(), om.n_e, w, n_layers=kw.get("n_layers", 1))
    p = I.pressure_field(om.n_p, w.seed)
    ud, pd = torch.tensor(u, device=dev), torch.tensor(p, device=dev)
    y = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    ref = om.laplace(p)
    _cmp(gm.laplace(pd, y).cpu().numpy(), ref, TOL64, "laplace fp64")
    y32 = torch.empty(gm.n_p, dtype=torch.float32, device=dev)
    _cmp(gm.laplace(pd.float(), y32).cpu().numpy(), ref, TOL32, "laplace fp32")
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    _cmp(gm.divergence(ud, b).cpu().numpy(), om.divergence(u), TOL64, "divergence")
    yc = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    refc = om.convective(u)
    _cmp(gm.convective(ud, yc).cpu().numpy(), refc, TOL64, "convective fp64")
    yc32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.convective(ud.float(), yc32).cpu().numpy(), refc, 2 * TOL32, "convective fp32")
    gm.update_eddy_viscosity(ud)
    yv = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    refv = om.viscous(u, u)
    _cmp(gm.viscous(ud, yv).cpu().numpy(), refv, TOL64, "viscous fp64")
    yv32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.viscous(ud.float(), yv32).cpu().numpy(), refv, 2 * TOL32, "viscous fp32")


def test_bump_node_coordinates_match_oracle(dgw):
    w = I.bump_workload("b8", 6, 4, 3, 3, seed=28)
    om, gm = _meshes(dgw, w)
    assert np.abs(gm.node_coords() - om.node_coords()).max() < 1e-13


@pytest.mark.parametrize("mode,w", [
    (2, I.bump_workload("s1", 8, 4, 2, 2, seed=31)),
    (0, I.bump_workload("s2", 16, 8, 8, 2, seed=32)),   # h-levels, dense coarse at degree k
    (1, I.bump_workload("s3", 16, 8, 8, 3, seed=33)),   # h-levels then Q1, dense
    (0, I.bump_workload("s4", 6, 4, 3, 3, seed=34)),    # odd counts: semi-coarsening
])
def test_bump_pressure_solve(dgw, mode, w):
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    b = I.pressure_rhs(om.n_p, w.seed)
    bd = torch.tensor(b, device=dev)
    p = torch.zeros_like(bd)
    info = gm.pressure_solve(bd, p, rtol=1e-10, max_iter=5000 if mode == 2 else 200, mode=mode)
    ph = p.cpu().numpy()
    res = np.linalg.norm(b - om.laplace(ph)) / np.linalg.norm(b)
    assert info["rel_residual"] <= 1e-10 and res <= 1.5e-10, (info, res)
    assert abs(ph.mean()) < 1e-13
