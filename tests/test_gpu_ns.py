"""GPU parity for the operators of the projection step (Sec. 4.2, eq. projectionspat) and the exact
inverse mass of the explicit convective step: pressure gradient P(v, p), tau_D, div-div penalty
D(v, u) and M^-1, element by element (or as functions, where the wall-cell systems are
ill-conditioned) against the FP64 oracle on channel and bump meshes."""
import math

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
    return om, gm


def _velocity(om, w, kw):
    nef = 1 if kw.get("enrich_l", 1) == 0 else 8
    u = I.workload_velocity(om.node_coords(), om.n_e, w, n_layers=kw.get("n_layers", 1), nef=nef)
    u[3 * om.n_p:] += 0.2 * w.u_tau * I.uniform(w.seed, u.size - 3 * om.n_p, -1.0, 1.0, stream=81)
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
def test_projection_step_operators_match_oracle(dgw, name, w, kw):
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    p = I.uniform(w.seed, om.n_p, -1.0, 1.0, stream=82)
    y = torch.full((gm.n_u,), float("nan"), dtype=torch.float64, device=dev)
    _cmp(gm.gradient(torch.tensor(p, device=dev), y).cpu().numpy(), om.gradient(p), TOL64, "gradient")
    u = _velocity(om, w, kw)
    ud = torch.tensor(u, device=dev)
    dt, cr = 2e-3, 0.14
    tau_ref = om.tau_divdiv(u, dt, cr)
    tau = torch.empty(gm.nc, dtype=torch.float64, device=dev)
    _cmp(gm.tau_divdiv(ud, dt, cr, tau).cpu().numpy(), tau_ref, TOL64, "tau_D")
    v = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=83)
    y.fill_(float("nan"))
    _cmp(gm.divdiv(torch.tensor(tau_ref, device=dev), torch.tensor(v, device=dev), y).cpu().numpy(),
         om.divdiv(tau_ref, v), TOL64, "div-div")


@pytest.mark.parametrize("name,w,kw", CASES, ids=[c[0] for c in CASES])
def test_curl_and_pressure_neumann_match_oracle(dgw, name, w, kw):
    """(v, curl u) element by element; the wall integrals of the high-order pressure Neumann data
    (eq. bc_d_pres) with two history levels, given the same vorticities, element by element."""
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, kw)
    u1 = u + 0.05 * I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=84)
    y = torch.full((gm.n_u,), float("nan"), dtype=torch.float64, device=dev)
    _cmp(gm.curl(torch.tensor(u, device=dev), y).cpu().numpy(), om.curl(u), TOL64, "curl")
    w0 = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=85)
    w1 = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=86)
    force = (0.3, -0.2, 0.1)
    base = I.uniform(w.seed, om.n_p, -1.0, 1.0, stream=87)
    ref = base + om.pressure_neumann(u, w0, 2.0, u1, w1, -1.0, force)
    b = torch.tensor(base, device=dev)
    t = lambda a: torch.tensor(a, device=dev)
    gm.add_pressure_neumann(b, t(u), t(w0), 2.0, t(u1), t(w1), -1.0, force)
    _cmp(b.cpu().numpy(), ref, TOL64, "pressure Neumann data")


def _l2(om, d, ref):
    return float(np.sqrt(abs(d @ om.vmass(d)) / (ref @ om.vmass(ref))))


@pytest.mark.parametrize("name,w,kw", CASES, ids=[c[0] for c in CASES])
def test_inverse_mass_matches_oracle(dgw, name, w, kw):
    """x = M^-1 (M u): cells without enrichment coefficient by coefficient (collocation, well
    conditioned); the whole field as a function in the L2 norm (two backward-stable solves of the
    ill-conditioned wall-cell systems differ by about N eps sqrt(kappa))."""
    om, gm = _meshes(dgw, w, **kw)
    dev = torch.device("cuda:0")
    u = _velocity(om, w, kw)
    r = om.vmass(u)
    ref = om.inverse_mass(r)
    x = torch.full((gm.n_u,), float("nan"), dtype=torch.float64, device=dev)
    got = gm.inverse_mass(torch.tensor(r, device=dev), x).cpu().numpy()
    assert _l2(om, got - ref, ref) < 1e-9 and _l2(om, got - u, u) < 1e-9
    L = kw.get("n_layers", 1)
    wall = np.array([((c // w.nx) % w.ny) < L or ((c // w.nx) % w.ny) >= w.ny - L for c in range(om.nc)])
    std = lambda v: v[: 3 * om.n_p].reshape(om.nc, -1)
    if (~wall).any():
        _cmp(std(got)[~wall], std(ref)[~wall], TOL64, "inverse mass off the wall")
    # the factor is reused: a second call gives the same bits
    x2 = torch.empty_like(x)
    gm.inverse_mass(torch.tensor(r, device=dev), x2)
    assert torch.equal(x, x2)


def _std_field(om, fx, fy, fz):
    X = om.node_coords()
    n3 = (om.k + 1) ** 3
    u = np.zeros(om.n_u)
    std = u[: 3 * om.n_p].reshape(om.nc, 3, n3)
    for a, f in enumerate((fx, fy, fz)):
        std[:, a, :] = f(X[:, 0], X[:, 1], X[:, 2]).reshape(om.nc, n3)
    return u


def test_dual_splitting_keeps_poiseuille_flow_steady(dgw):
    nu, U = 1e-2, 1.0
    w = I.Workload("pois", 4, 4, 2, 2, 180.0, nu, seed=42)
    om = O.Mesh(**w.mesh_kwargs(), n_layers=0)
    gm = dgw.mesh_for(w, n_layers=0)
    u0 = _std_field(om, lambda x, y, z: U * (1 - y ** 2), lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    for hobc in (False, True):
        ns = dgw.DualSplitting(gm, torch.tensor(u0, device="cuda"), dt=5e-3, force=(2 * nu * U, 0.0, 0.0),
                               rtol_pressure=1e-12, rtol_projection=1e-12, rtol_viscous=1e-12, pressure_mode=0,
                               high_order_pressure_bc=hobc)
        for _ in range(3):
            ns.step()
        u = ns.velocity().cpu().numpy()
        assert _l2(om, u - u0, u0) < 1e-10
        assert ns.pressure().abs().max().item() < 1e-9


NS_CASES = [
    ("channel_q2_4x4x2", I.Workload("ns", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=41), {}, False, 3, False),
    ("channel_q3_l0", I.Workload("ns3", 3, 4, 2, 3, 395.0, 1.0 / 6000.0, seed=43), {"enrich_l": 0}, False, 3, False),
    ("bump_q2_6x4x2", I.bump_workload("nsb", 6, 4, 2, 2, seed=44), {}, False, 2, False),
    ("channel_q2_wall_update", I.Workload("nsw", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=45), {}, True, 2, False),
    ("channel_q2_high_order_bc", I.Workload("nsh", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=47), {}, False, 3, True),
    ("bump_q2_high_order_bc_wall_update", I.bump_workload("nsbh", 6, 4, 2, 2, seed=48), {}, True, 2, True),
]


@pytest.mark.parametrize("name,w,kw,update,nsteps,hobc", NS_CASES, ids=[c[0] for c in NS_CASES])
def test_dual_splitting_matches_oracle(dgw, name, w, kw, update, nsteps, hobc):
    """Time steps of the GPU integrator against the oracle's, step by step. The GPU solves stop at
    1e-12 and the oracle's at 1e-13 relative residual; with condition numbers up to ~1e4 for these
    meshes the velocities agree to ~1e-8 as functions. The pressure solves for the divergence of a
    nearly divergence-free u^, a small difference of large terms, so its error is measured against the
    pressure scale of the first step (where u0 is far from divergence-free)."""
    om, gm = _meshes(dgw, w, **kw)
    nef = 1 if kw.get("enrich_l", 1) == 0 else 8
    u0 = I.workload_velocity(om.node_coords(), om.n_e, w, nef=nef)
    dt, force = 2e-3, (w.tau_w / (0.5 * w.ly), 0.0, 0.0)
    ref = O.DualSplitting(om, u0, dt=dt, force=force, rtol=1e-13, update_wall_model=update,
                          high_order_pressure_bc=hobc)
    ns = dgw.DualSplitting(gm, torch.tensor(u0, device="cuda"), dt=dt, force=force, rtol_pressure=1e-12,
                           rtol_projection=1e-12, rtol_viscous=1e-12, pressure_mode=0, update_wall_model=update,
                           high_order_pressure_bc=hobc)
    pscale = None
    for step in range(nsteps):
        info = ns.step()
        ur, pr = ref.step()
        u = ns.velocity().cpu().numpy()
        p = ns.pressure().cpu().numpy()
        pscale = pscale or np.linalg.norm(pr)
        du = _l2(om, u - ur, ur)
        dp = np.linalg.norm(p - pr) / pscale
        assert du < 1e-8 and dp < 1e-6, (step, du, dp, info)


RATE_CASES = [
    ("channel_q2_4x4x2", I.Workload("cr", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=61), {}),
    ("channel_q3_two_layers_l0", I.Workload("cr3", 3, 6, 2, 3, 395.0, 1.0 / 6000.0, seed=62), {"n_layers": 2, "enrich_l": 0}),
    ("bump_q3_6x4x2", I.bump_workload("crb", 6, 4, 2, 3, seed=63), {}),
]


@pytest.mark.parametrize("name,w,kw", RATE_CASES, ids=[c[0] for c in RATE_CASES])
def test_cfl_rate_matches_oracle(dgw, name, w, kw):
    """dgw_cfl_rate against the oracle on the workload field and on a random field whose enrichment
    coefficients are as large as the standard ones (the largest rate then sits in a wall cell)."""
    om, gm = _meshes(dgw, w, **kw)
    nef = 1 if kw.get("enrich_l", 1) == 0 else 8
    u0 = I.workload_velocity(om.node_coords(), om.n_e, w, n_layers=kw.get("n_layers", 1), nef=nef)
    ur = I.uniform(w.seed, om.n_u, -1.0, 1.0, stream=64)
    for u in (u0, ur):
        ref = om.cfl_rate(u)
        got = gm.cfl_rate(torch.tensor(u, device="cuda"))
        assert abs(got / ref - 1.0) < 1e-12, (got, ref)


ADAPTIVE_CASES = [
    ("channel_q2_4x4x2", I.Workload("ad", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=65), {}, False),
    ("bump_q2_6x4x2_high_order_bc", I.bump_workload("adb", 6, 4, 2, 2, seed=66), {}, True),
]


@pytest.mark.parametrize("name,w,kw,hobc", ADAPTIVE_CASES, ids=[c[0] for c in ADAPTIVE_CASES])
def test_adaptive_dual_splitting_matches_oracle(dgw, name, w, kw, hobc):
    """Adaptive steps (the CFL step binds: dt_max is large) against the oracle: the step sizes to
    1e-12 (they follow from u^n, so the GPU's rounding in u^n moves them by ~1e-8 relative at most in
    later steps) and the fields as in the constant-step test."""
    om, gm = _meshes(dgw, w, **kw)
    u0 = I.workload_velocity(om.node_coords(), om.n_e, w)
    force = (w.tau_w / (0.5 * w.ly), 0.0, 0.0)
    ref = O.DualSplitting(om, u0, dt=1.0, cr=0.14, force=force, rtol=1e-13, high_order_pressure_bc=hobc,
                          adaptive=True)
    ns = dgw.DualSplitting(gm, torch.tensor(u0, device="cuda"), dt=1.0, cr=0.14, force=force, rtol_pressure=1e-12,
                           rtol_projection=1e-12, rtol_viscous=1e-12, pressure_mode=0, high_order_pressure_bc=hobc,
                           adaptive_dt=True)
    pscale = None
    for step in range(3):
        info = ns.step()
        ur, pr = ref.step()
        assert info["dt"] < 1.0
        assert abs(info["dt"] / ref.dts[-1] - 1.0) < (1e-12 if step == 0 else 1e-7), (step, info["dt"], ref.dts[-1])
        u = ns.velocity().cpu().numpy()
        p = ns.pressure().cpu().numpy()
        pscale = pscale or np.linalg.norm(pr)
        du = _l2(om, u - ur, ur)
        dp = np.linalg.norm(p - pr) / pscale
        assert du < 1e-8 and dp < 1e-6, (step, du, dp, info)
    assert len(set(ref.dts)) > 1   # the step changed, so the variable-step constants were used


def test_time_step_reports_a_capped_solve(dgw):
    """With max_iter below what the solves of a step need at rtol 1e-12 the step fails with
    DGW_ENOTCONV (raised by the binding) instead of returning an unconverged field; the same
    integrator created with enough iterations takes the step."""
    w = I.Workload("cap", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=67)
    om, gm = _meshes(dgw, w)
    u0 = torch.tensor(I.workload_velocity(om.node_coords(), om.n_e, w), device="cuda")
    force = (w.tau_w, 0.0, 0.0)
    capped = dgw.DualSplitting(gm, u0, dt=2e-3, force=force, rtol_pressure=1e-12, rtol_projection=1e-12,
                               rtol_viscous=1e-12, max_iter=3, pressure_mode=0)
    with pytest.raises(dgw.DGWError) as err:
        capped.step()
    assert err.value.status == -3
    ok = dgw.DualSplitting(gm, u0, dt=2e-3, force=force, rtol_pressure=1e-12, rtol_projection=1e-12,
                           rtol_viscous=1e-12, max_iter=2000, pressure_mode=0)
    info = ok.step()
    assert info["projection_iterations"] > 3
