"""GPU parity: every operator of the CUDA library against the FP64 CPU oracle on the same seeded
inputs, element by element. Bar: relative 2-norm error <= 1e-12 and max elementwise error
<= 1e-12 * max |y| for FP64; 1e-5 for FP32 applies."""
import math

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
    nref = np.linalg.norm(ref)
    rel = np.linalg.norm(y - ref) / nref
    ele = np.abs(y - ref).max() / np.abs(ref).max()
    assert rel <= tol and ele <= tol, f"{what}: rel {rel:.3e} elem {ele:.3e}"
    return rel


def _meshes(dgw, w, **kw):
    om = O.Mesh(**w.mesh_kwargs(), **{k: v for k, v in kw.items() if k in ("n_layers", "q_wall", "wall_law")})
    gm = dgw.mesh_for(w, **kw)
    assert (gm.n_p, gm.n_u, gm.n_e) == (om.n_p, om.n_u, om.n_e)
    return om, gm


CASES = [
    # name, workload, mesh kwargs
    ("c1_q2_8x8x8", I.WORKLOADS["channel_q2_8x8x8"], {}),
    ("ragged_q1_3x4x5", I.Workload("r1", 3, 4, 5, 1, 180.0, 1.0 / 3250.0, seed=11), {}),
    ("ragged_q3_5x3x2", I.Workload("r3", 5, 3, 2, 3, 395.0, 1.0 / 6000.0, seed=12), {}),
    ("q4_4x6x3_vandriest", I.Workload("r4", 4, 6, 3, 4, 590.0, 1.0 / 12000.0, seed=13), {"wall_law": 1}),
    ("q5_3x4x2_two_layers", I.Workload("r5", 3, 4, 2, 5, 180.0, 1.0 / 3250.0, seed=14), {"n_layers": 2}),
    ("q2_single_cells_1x2x1", I.Workload("r6", 1, 2, 1, 2, 180.0, 1.0 / 3250.0, seed=15), {}),
    ("q3_no_enrichment", I.Workload("r7", 4, 3, 3, 3, 180.0, 1.0 / 3250.0, seed=16), {"n_layers": 0}),
    ("q4_qwall_5", I.Workload("r8", 3, 4, 3, 4, 590.0, 1.0 / 12000.0, seed=17), {"q_wall": 5}),
]


@pytest.mark.parametrize("name,w,kw", CASES, ids=[c[0] for c in CASES])
def test_operators_match_oracle(dgw, name, w, kw):
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    u = I.velocity_field(om.node_coords(), om.n_e, w, n_layers=kw.get("n_layers", 1))
    p = I.pressure_field(om.n_p, w.seed)
    ud, pd = torch.tensor(u, device=dev), torch.tensor(p, device=dev)
    # Laplace (FP64, FP32)
    y = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    ref = om.laplace(p)
    _cmp(gm.laplace(pd, y).cpu().numpy(), ref, TOL64, "laplace fp64")
    y32 = torch.empty(gm.n_p, dtype=torch.float32, device=dev)
    _cmp(gm.laplace(pd.float(), y32).cpu().numpy(), ref, TOL32, "laplace fp32")
    # divergence
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    _cmp(gm.divergence(ud, b).cpu().numpy(), om.divergence(u), TOL64, "divergence")
    # convective
    yc = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    refc = om.convective(u)
    _cmp(gm.convective(ud, yc).cpu().numpy(), refc, TOL64, "convective fp64")
    yc32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.convective(ud.float(), yc32).cpu().numpy(), refc, 2 * TOL32, "convective fp32")
    # viscous with nu_t frozen from u
    gm.update_eddy_viscosity(ud)
    yv = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    refv = om.viscous(u, u)
    _cmp(gm.viscous(ud, yv).cpu().numpy(), refv, TOL64, "viscous fp64")
    yv32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.viscous(ud.float(), yv32).cpu().numpy(), refv, 2 * TOL32, "viscous fp32")


def test_viscous_frozen_field_differs_from_input(dgw):
    """nu_t comes from the field of the last update, not from the applied vector (frozen)."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u = I.velocity_field(om.node_coords(), om.n_e, w)
    v = I.uniform(99, om.n_u, -1, 1)
    gm.update_eddy_viscosity(torch.tensor(u, device=dev))
    y = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    _cmp(gm.viscous(torch.tensor(v, device=dev), y).cpu().numpy(), om.viscous(u, v), TOL64, "viscous frozen")


def test_pressure_solve_jacobi_reaches_tolerance(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u = I.velocity_field(om.node_coords(), om.n_e, w)
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    gm.divergence(torch.tensor(u, device=dev), b)
    p = torch.zeros_like(b)
    info = gm.pressure_solve(b, p, rtol=1e-10, max_iter=5000, mode=2)
    bh = b.cpu().numpy()
    bh = bh - bh.mean()
    res = np.linalg.norm(bh - om.laplace(p.cpu().numpy())) / np.linalg.norm(bh)
    assert info["rel_residual"] <= 1e-10 and res <= 1.5e-10, (info, res)
    assert abs(p.cpu().numpy().mean()) < 1e-14
    # agrees with the oracle's own solve to the conditioning-limited accuracy
    pref, it, rr = om.solve(bh, rtol=1e-13)
    assert np.linalg.norm(p.cpu().numpy() - pref) / np.linalg.norm(pref) < 1e-6


def test_empty_input_rejected(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    gm = dgw.mesh_for(w)
    with pytest.raises(ValueError):
        gm.laplace(torch.zeros(0, dtype=torch.float64, device="cuda"), torch.zeros(0, dtype=torch.float64, device="cuda"))
    with pytest.raises(dgw.DGWError):
        dgw.Mesh(0, 4, 4, 2, lx=1.0, lz=1.0, nu=1e-3, tau_w=1e-2)


@pytest.mark.parametrize("mode", [0, 1])
def test_pressure_solve_multigrid_modes(dgw, mode):
    """FP64 CG with the FP64 (mode 0) or FP32 (mode 1) multigrid V-cycle reaches 1e-10; the residual
    is re-evaluated with the oracle's own operator."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u = I.velocity_field(om.node_coords(), om.n_e, w)
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    gm.divergence(torch.tensor(u, device=dev), b)
    p = torch.zeros_like(b)
    info = gm.pressure_solve(b, p, rtol=1e-10, max_iter=200, mode=mode)
    bh = b.cpu().numpy()
    bh = bh - bh.mean()
    res = np.linalg.norm(bh - om.laplace(p.cpu().numpy())) / np.linalg.norm(bh)
    assert info["rel_residual"] <= 1e-10 and res <= 1.5e-10, (info, res)
    assert info["iterations"] < 60, info
    assert abs(p.cpu().numpy().mean()) < 1e-14


@pytest.mark.parametrize("dims,k", [((6, 4, 4), 3), ((5, 6, 3), 2), ((4, 2, 4), 4)])
def test_pressure_solve_multigrid_odd_and_semi_coarsening(dgw, dims, k):
    """Odd cell counts stop the coarsening of that direction (semi-coarsening) or the hierarchy."""
    w = I.Workload("mg", *dims, k, 180.0, 1.0 / 3250.0, seed=21)
    gm = dgw.mesh_for(w)
    om = O.Mesh(**w.mesh_kwargs())
    b = torch.tensor(I.pressure_rhs(gm.n_p, 5), device="cuda")
    p = torch.zeros_like(b)
    info = gm.pressure_solve(b, p, rtol=1e-10, max_iter=300, mode=1)
    bh = b.cpu().numpy()
    res = np.linalg.norm(bh - om.laplace(p.cpu().numpy())) / np.linalg.norm(bh)
    assert res <= 1.5e-10, (info, res)
