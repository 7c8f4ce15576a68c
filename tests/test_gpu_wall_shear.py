"""GPU parity for the wall-shear-stress update (Sec. 3.2): the nodal tau_w,B computed from a velocity
field against the FP64 oracle, every operator after a spatially varying nodal tau_w has been set
(this exercises the grad tau_w,h terms of grad y+), and one full update cycle (tau_w from u, new
wall tables, new nu_t, viscous apply) on channel and bump meshes."""
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
    om = O.Mesh(**w.mesh_kwargs(), **{k: v for k, v in kw.items() if k in KEYS})
    gm = dgw.mesh_for(w, **kw)
    assert (gm.n_p, gm.n_u, gm.n_e) == (om.n_p, om.n_u, om.n_e)
    assert gm.n_wall_nodes == om.n_wall_nodes
    return om, gm


def _velocity(om, w, kw):
    nef = 1 if kw.get("enrich_l", 1) == 0 else 8
    u = I.workload_velocity(om.node_coords(), om.n_e, w, n_layers=kw.get("n_layers", 1), nef=nef)
    u[3 * om.n_p:] += 0.2 * w.u_tau * I.uniform(w.seed, u.size - 3 * om.n_p, -1.0, 1.0, stream=71)
    return u


CASES = [
    ("c1_q2_8x8x8", I.WORKLOADS["channel_q2_8x8x8"], {}),
    ("ragged_q3_5x3x2_vandriest", I.Workload("r3", 5, 3, 2, 3, 395.0, 1.0 / 6000.0, seed=12), {"wall_law": 1}),
    ("q4_two_layers_l0", I.Workload("r8", 3, 4, 3, 4, 590.0, 1.0 / 12000.0, seed=17), {"n_layers": 2, "enrich_l": 0}),
    ("q2_single_cells_1x2x1", I.Workload("r6", 1, 2, 1, 2, 180.0, 1.0 / 3250.0, seed=15), {}),
    ("q3_no_enrichment", I.Workload("r7", 4, 3, 3, 3, 180.0, 1.0 / 3250.0, seed=16), {"n_layers": 0}),
    ("bump_q3_6x4x3", I.bump_workload("b2", 6, 4, 3, 3, seed=22), {}),
    ("bump_q2_5x4x2_l0", I.bump_workload("b5", 5, 4, 2, 2, seed=25), {"enrich_l": 0}),
]


@pytest.mark.parametrize("name,w,kw", CASES, ids=[c[0] for c in CASES])
def test_nodal_wall_shear_matches_oracle(dgw, name, w, kw):
    om, gm = _meshes(dgw, w, **kw)
    u = _velocity(om, w, kw)
    ref = om.wall_shear(u)
    tau = torch.empty(gm.n_wall_nodes, dtype=torch.float64, device="cuda")
    _cmp(gm.wall_shear_stress(torch.tensor(u, device="cuda"), tau).cpu().numpy(), ref, TOL64, "tau_w,B")


@pytest.mark.parametrize("name,w,kw", [c for c in CASES if c[2].get("n_layers", 1) > 0],
                         ids=[c[0] for c in CASES if c[2].get("n_layers", 1) > 0])
def test_operators_after_varying_nodal_tau(dgw, name, w, kw):
    """A seeded nodal tau_w in [0.5, 1.5] tau_w: the enrichment space, y+ and nu_t all vary along the
    wall; every operator must still match the oracle given the same nodal values."""
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    tn = w.tau_w * (1.0 + 0.5 * I.uniform(w.seed, om.n_wall_nodes, -1.0, 1.0, stream=72))
    om.set_tau_nodes(tn)
    gm.set_wall_shear_stress(torch.tensor(tn, device=dev))
    u = _velocity(om, w, kw)
    ud = torch.tensor(u, device=dev)
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    _cmp(gm.divergence(ud, b).cpu().numpy(), om.divergence(u), TOL64, "divergence")
    y = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    _cmp(gm.convective(ud, y).cpu().numpy(), om.convective(u), TOL64, "convective")
    _cmp(gm.mass(ud, y).cpu().numpy(), om.vmass(u), TOL64, "mass")
    gm.update_eddy_viscosity(ud)
    v = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=73)
    _cmp(gm.viscous(torch.tensor(v, device=dev), y).cpu().numpy(), om.viscous(u, v), TOL64, "viscous")
    y32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.viscous(torch.tensor(v, device=dev).float(), y32).cpu().numpy(), om.viscous(u, v), 2e-5, "viscous fp32")


@pytest.mark.parametrize("wname", ["channel_q2_8x8x8", "bump_q3"])
def test_update_cycle_matches_oracle(dgw, wname):
    """tau_w,B from u, set as the new nodal tau_w, nu_t from u in the new space, then the wall shear
    of the same u in the new space and a viscous apply - both sides run the same cycle."""
    w = I.WORKLOADS["channel_q2_8x8x8"] if wname.startswith("channel") else I.bump_workload("b3", 6, 4, 2, 3, seed=26)
    om, gm = _meshes(dgw, w)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, {})
    ud = torch.tensor(u, device=dev)
    tau = torch.empty(gm.n_wall_nodes, dtype=torch.float64, device=dev)
    gm.wall_shear_stress(ud, tau)
    om.set_tau_nodes(om.wall_shear(u))
    gm.set_wall_shear_stress(tau)
    gm.update_eddy_viscosity(ud)
    _cmp(gm.wall_shear_stress(ud, tau).cpu().numpy(), om.wall_shear(u), TOL64, "tau after update")
    y = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    _cmp(gm.viscous(ud, y).cpu().numpy(), om.viscous(u, u), TOL64, "viscous after update")


def test_set_wall_shear_rejects_non_positive(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    gm = dgw.mesh_for(w)
    tn = torch.full((gm.n_wall_nodes,), w.tau_w, dtype=torch.float64, device="cuda")
    tn[3] = 0.0
    with pytest.raises(dgw.DGWError):
        gm.set_wall_shear_stress(tn)
    tn[3] = float("nan")
    with pytest.raises(dgw.DGWError):
        gm.set_wall_shear_stress(tn)


def _l2(om, d, ref):
    """relative L2 norm of d against ref in the mesh's current (new) space"""
    return float(np.sqrt(abs(d @ om.vmass(d)) / (ref @ om.vmass(ref))))


PROJ_CASES = [
    ("c1_q2_8x8x8", I.WORKLOADS["channel_q2_8x8x8"], {}),
    ("q4_two_layers_l0", I.Workload("r8", 3, 4, 3, 4, 590.0, 1.0 / 12000.0, seed=17), {"n_layers": 2, "enrich_l": 0}),
    ("ragged_q3_vandriest_qwall6", I.Workload("r3", 5, 3, 2, 3, 395.0, 1.0 / 6000.0, seed=12),
     {"wall_law": 1, "q_wall": 6}),
    ("bump_q3_6x4x3", I.bump_workload("b2", 6, 4, 3, 3, seed=22), {}),
]


@pytest.mark.parametrize("name,w,kw", PROJ_CASES, ids=[c[0] for c in PROJ_CASES])
def test_projection_matches_oracle(dgw, name, w, kw):
    """Cell-wise L2 projection onto a varying new nodal tau_w (eq. l2): the cells off the wall are
    copied bit for bit; in the wall cells the projected functions agree in the L2 norm (the cell
    systems are ill-conditioned, so coefficients are not compared), and so do their Galerkin
    moments M_new u_new."""
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, kw)
    tn = w.tau_w * (1.0 + 0.5 * I.uniform(w.seed, om.n_wall_nodes, -1.0, 1.0, stream=74))
    ref = om.project(tn, u)
    un = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    gm.project_velocity(torch.tensor(tn, device=dev), torch.tensor(u, device=dev), un)
    got = un.cpu().numpy()
    wall = np.zeros(om.nc, dtype=bool)
    L = kw.get("n_layers", 1)
    for c in range(om.nc):
        j = (c // w.nx) % w.ny
        wall[c] = j < L or j >= w.ny - L
    std = lambda v: v[: 3 * om.n_p].reshape(om.nc, -1)
    assert np.array_equal(std(got)[~wall], std(u)[~wall])
    # two backward-stable FP64 solves (Cholesky here, pivoted LU in the oracle) of a cell system with
    # condition number kappa differ by about N eps sqrt(kappa) in the energy norm; the wall cells of
    # these meshes reach kappa ~ 1e10 (N <= 133 unknowns), hence 1e-9 for the functions
    l2 = _l2(om, got - ref, ref)
    mg, mr = om.vmass(got), om.vmass(ref)
    mom = np.linalg.norm(mg - mr) / np.linalg.norm(mr)
    assert l2 < 1e-9 and mom < 1e-10, (l2, mom)
    # the GPU mesh now holds the new space: the mass operators of both sides agree on the result
    y = torch.empty_like(un)
    _cmp(gm.mass(un, y).cpu().numpy(), mg, 1e-12, "mass in the new space")


def test_projection_in_place_equals_out_of_place(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    dev = torch.device("cuda:0")
    g1, g2 = dgw.mesh_for(w), dgw.mesh_for(w)
    om = O.Mesh(**w.mesh_kwargs())
    u = torch.tensor(_velocity(om, w, {}), device=dev)
    tn = torch.tensor(w.tau_w * (1.0 + 0.3 * I.uniform(9, g1.n_wall_nodes, -1.0, 1.0)), device=dev)
    out = torch.empty_like(u)
    g1.project_velocity(tn, u, out)
    v = u.clone()
    g2.project_velocity(tn, v, v)
    assert torch.equal(out, v)


def test_projection_rejects_non_positive_tau_and_singular_cell_spaces(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    gm = dgw.mesh_for(w)
    u = torch.zeros(gm.n_u, dtype=torch.float64, device="cuda")
    tn = torch.full((gm.n_wall_nodes,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(dgw.DGWError):
        gm.project_velocity(tn, u, u)
    # k = 3 with l = 1 has 6 wall-normal functions: 5 points cannot separate them
    w3 = I.Workload("r3", 5, 3, 2, 3, 395.0, 1.0 / 6000.0, seed=12)
    g3 = dgw.mesh_for(w3, q_wall=5)
    u3 = torch.zeros(g3.n_u, dtype=torch.float64, device="cuda")
    t3 = torch.full((g3.n_wall_nodes,), w3.tau_w, dtype=torch.float64, device="cuda")
    with pytest.raises(dgw.DGWError):
        g3.project_velocity(t3, u3, u3)


SWITCH_CASES = [
    ("c1_q2_8x8x8", I.WORKLOADS["channel_q2_8x8x8"], {}),
    ("q3_two_layers_l0", I.Workload("s3", 4, 6, 2, 3, 395.0, 1.0 / 6000.0, seed=35), {"n_layers": 2, "enrich_l": 0}),
    ("bump_q3_6x4x3", I.bump_workload("b2", 6, 4, 3, 3, seed=22), {}),
]


def _switched(dgw, w, kw, thr=None):
    """Seeded nodal tau_w over two decades; the threshold (if not given) is the first of a ladder that
    leaves part of the wall columns on and part off in the oracle."""
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    tn = w.tau_w * 10.0 ** I.uniform(w.seed, om.n_wall_nodes, -1.0, 1.0, stream=75)
    om.set_tau_nodes(tn)
    for t in ([thr] if thr is not None else list(10.0 * 1.25 ** np.arange(25))):
        om.set_switch(t)
        if 0 < om.active().sum() < om.n_e:
            thr = float(t)
            break
    assert thr is not None
    gm.set_wall_shear_stress(torch.tensor(tn, device=dev))
    gm.set_enrichment_switch(thr)
    return om, gm, tn


@pytest.mark.parametrize("name,w,kw", SWITCH_CASES, ids=[c[0] for c in SWITCH_CASES])
def test_switch_off_operators_match_oracle(dgw, name, w, kw):
    """Part of the wall columns switched off (y+ threshold between the smallest and largest column
    maxima): the same columns on both sides, and every operator equal to the oracle's; outputs of the
    switched-off enrichment slots are written as zeros (buffers start as NaN)."""
    om, gm, _ = _switched(dgw, w, kw)
    on = om.active()
    assert 0 < on.sum() < om.n_e, on.sum()
    assert np.array_equal(gm.enrichment_active(), on)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, kw)
    ud = torch.tensor(u, device=dev)
    y = torch.full((gm.n_u,), float("nan"), dtype=torch.float64, device=dev)
    _cmp(gm.convective(ud, y).cpu().numpy(), om.convective(u), TOL64, "convective")
    # random field: sign-changing normal velocity makes each face's point rule matter (faces of a
    # switched-off cell next to a switched-on one take q_w along y, the others the standard rule)
    ur = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=102)
    _cmp(gm.convective(torch.tensor(ur, device=dev), y).cpu().numpy(), om.convective(ur), TOL64, "convective (random)")
    y.fill_(float("nan"))
    _cmp(gm.mass(ud, y).cpu().numpy(), om.vmass(u), TOL64, "mass")
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    _cmp(gm.divergence(ud, b).cpu().numpy(), om.divergence(u), TOL64, "divergence")
    gm.update_eddy_viscosity(ud)
    v = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=76)
    y.fill_(float("nan"))
    _cmp(gm.viscous(torch.tensor(v, device=dev), y).cpu().numpy(), om.viscous(u, v), TOL64, "viscous")
    tau = torch.empty(gm.n_wall_nodes, dtype=torch.float64, device=dev)
    _cmp(gm.wall_shear_stress(ud, tau).cpu().numpy(), om.wall_shear(u), TOL64, "tau_w,B")


def test_switch_off_everywhere_equals_mesh_without_enrichment(dgw):
    w = I.WORKLOADS["channel_q2_8x8x8"]
    dev = torch.device("cuda:0")
    gm, g0 = dgw.mesh_for(w), dgw.mesh_for(w, n_layers=0)
    gm.set_enrichment_switch(1e30)
    assert gm.enrichment_active().sum() == 0
    om = O.Mesh(**w.mesh_kwargs())
    u = torch.tensor(_velocity(om, w, {}), device=dev)
    np3 = 3 * gm.n_p
    for op in ("convective", "mass"):
        y = torch.full((gm.n_u,), float("nan"), dtype=torch.float64, device=dev)
        y0 = torch.empty(g0.n_u, dtype=torch.float64, device=dev)
        getattr(gm, op)(u, y)
        getattr(g0, op)(u[:np3].contiguous(), y0)
        # the (switched-off) wall-layer rows take the general kernel on gm and the degree-specialised
        # one on g0: equal to rounding; the enrichment slots are exactly zero
        diff = (y[:np3] - y0).abs().max().item()
        assert diff <= 1e-13 * y0.abs().max().item() and not torch.any(y[np3:] != 0), (op, diff)
    gm.set_enrichment_switch(0.0)
    assert gm.enrichment_active().sum() == gm.n_e


def test_switch_off_helmholtz_and_projection(dgw):
    """Helmholtz solve and L2 projection with part of the wall columns switched off, checked with the
    oracle's operators (residual) and projection (L2 norm and Galerkin moments)."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    om, gm, tn = _switched(dgw, w, {}, 25.0)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, {})
    ud = torch.tensor(u, device=dev)
    # projection onto a new space with a different switched-off pattern
    tn2 = w.tau_w * 10.0 ** I.uniform(w.seed, om.n_wall_nodes, -1.0, 1.0, stream=77)
    ref = om.project(tn2, u)
    un = torch.empty_like(ud)
    gm.project_velocity(torch.tensor(tn2, device=dev), ud, un)
    assert np.array_equal(gm.enrichment_active(), om.active())
    got = un.cpu().numpy()
    l2 = _l2(om, got - ref, ref)
    mom = np.linalg.norm(om.vmass(got) - om.vmass(ref)) / np.linalg.norm(om.vmass(ref))
    assert l2 < 1e-9 and mom < 1e-10, (l2, mom)
    # Helmholtz in the new space
    gamma = 1.5e3
    gm.update_eddy_viscosity(un)
    rhs = gamma * om.vmass(ref)
    x = un.clone()
    info = gm.helmholtz_solve(gamma, torch.tensor(rhs, device=dev), x, rtol=1e-10, max_iter=2000, restart=30)
    xh = x.cpu().numpy()
    res = rhs - (gamma * om.vmass(xh) + om.viscous(got, xh))
    assert info["rel_residual"] <= 1e-10 and np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(rhs)
    off = np.repeat(om.active() == 0, 24)
    assert not np.any(xh[3 * om.n_p:][off])
