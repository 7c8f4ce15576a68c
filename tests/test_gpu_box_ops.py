"""Degree-specialised box kernels (standard cells; on the rows next to a wall layer they add the enriched
neighbour's u~ on the faces between) against the oracle, element by element: the divergence, the viscous
and the convective operator in FP64, in double-float (DGW_DF64) and in FP32, on meshes whose rows exercise
every path of those kernels and of the general kernel beside them: interior rows between one or two
enriched layers, a row whose two y-neighbours are both enriched, enrichment with l = 1 and l = 0, the wall
rows of meshes without enrichment (mirror state, x10 wall penalty), a single cell periodic onto itself in
x, odd and even cell counts along x (1 to 8 cells per CTA), degrees 1 to 5."""
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


CASES = [
    # nx, ny, nz, k, enriched layers per wall
    (8, 8, 4, 1, 1),
    (6, 7, 3, 2, 1),
    (5, 8, 2, 3, 1),
    (4, 6, 3, 4, 1),
    (2, 6, 2, 5, 1),
    (4, 3, 3, 3, 0),
    (1, 4, 1, 2, 0),
    (3, 5, 2, 4, 0),
    (8, 10, 2, 4, 2),
    (4, 3, 2, 3, 1),   # the middle row: enriched neighbours above and below
]


L0_CASES = [(6, 7, 3, 2, 1), (4, 6, 3, 4, 2), (4, 3, 2, 3, 1)]


@pytest.mark.parametrize("nx,ny,nz,k,layers,el", [c + (1,) for c in CASES] + [c + (0,) for c in L0_CASES],
                         ids=[f"{c[0]}x{c[1]}x{c[2]}_q{c[3]}_layers{c[4]}" for c in CASES]
                         + [f"{c[0]}x{c[1]}x{c[2]}_q{c[3]}_layers{c[4]}_l0" for c in L0_CASES])
def test_box_kernels_match_oracle(dgw, nx, ny, nz, k, layers, el):
    w = I.Workload("box", nx, ny, nz, k, 590.0, 1.0 / 12000.0, seed=40 + k)
    om = O.Mesh(**w.mesh_kwargs(), n_layers=layers, enrich_l=el)
    gm = dgw.mesh_for(w, n_layers=layers, enrich_l=el)
    assert (gm.n_p, gm.n_u) == (om.n_p, om.n_u)
    dev = torch.device("cuda:0")
    u = I.uniform(w.seed, gm.n_u, -1.0, 1.0, stream=5)
    u[3 * gm.n_p:] *= 0.05
    ud = torch.tensor(u, device=dev)
    # divergence
    refd = om.divergence(u)
    b = torch.empty(gm.n_p, dtype=torch.float64, device=dev)
    _cmp(gm.divergence(ud, b).cpu().numpy(), refd, TOL64, "divergence fp64")
    bd = gm.divergence(ud, torch.empty_like(b), prec=dgw.DGW_DF64).cpu().numpy()
    _cmp(bd, refd, TOL64, "divergence df64")
    # viscous, nu_t frozen from u
    gm.update_eddy_viscosity(ud)
    refv = om.viscous(u, u)
    y = torch.empty(gm.n_u, dtype=torch.float64, device=dev)
    y64 = gm.viscous(ud, y).cpu().numpy()
    _cmp(y64, refv, TOL64, "viscous fp64")
    ydf = gm.viscous(ud, torch.empty_like(y), prec=dgw.DGW_DF64).cpu().numpy()
    _cmp(ydf, refv, TOL64, "viscous df64")
    assert np.linalg.norm(ydf - y64) / np.linalg.norm(y64) < 1e-13
    y32 = torch.empty(gm.n_u, dtype=torch.float32, device=dev)
    _cmp(gm.viscous(ud.float(), y32).cpu().numpy(), refv, TOL32, "viscous fp32")
    # convective: the random field changes the sign of u.n on most faces, so both branches of the
    # Lax-Friedrichs Lambda are taken
    refc = om.convective(u)
    yc64 = gm.convective(ud, torch.empty_like(y)).cpu().numpy()
    _cmp(yc64, refc, TOL64, "convective fp64")
    ycdf = gm.convective(ud, torch.empty_like(y), prec=dgw.DGW_DF64).cpu().numpy()
    _cmp(ycdf, refc, TOL64, "convective df64")
    assert np.linalg.norm(ycdf - yc64) / np.linalg.norm(yc64) < 1e-13
    _cmp(gm.convective(ud.float(), torch.empty_like(y32)).cpu().numpy(), refc, TOL32, "convective fp32")


def test_box_kernels_smooth_field_of_the_workload(dgw):
    """The physical velocity of the Q2 8x8x8 workload (smooth, nearly divergence-free): the outputs
    are small differences of large terms, compared with the FP64 tolerance relative to the output."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    om = O.Mesh(**w.mesh_kwargs())
    gm = dgw.mesh_for(w)
    u = I.velocity_field(om.node_coords(), om.n_e, w)
    ud = torch.tensor(u, device="cuda")
    gm.update_eddy_viscosity(ud)
    refv = om.viscous(u, u)
    for prec in (None, dgw.DGW_DF64):
        y = torch.empty(gm.n_u, dtype=torch.float64, device="cuda")
        _cmp(gm.viscous(ud, y, prec=prec).cpu().numpy(), refv, TOL64, f"viscous {prec}")


def test_df64_rejected_where_unsupported(dgw):
    gm = dgw.mesh_for(I.bump_workload("b", 4, 4, 2, 2, seed=3))
    u = torch.zeros(gm.n_u, dtype=torch.float64, device="cuda")
    with pytest.raises(dgw.DGWError):
        gm.viscous(u, torch.empty_like(u), prec=dgw.DGW_DF64)
    with pytest.raises(dgw.DGWError):
        gm.convective(u, torch.empty_like(u), prec=dgw.DGW_DF64)
    with pytest.raises(dgw.DGWError):
        gm.divergence(u, torch.empty(gm.n_p, dtype=torch.float64, device="cuda"), prec=dgw.DGW_DF64)
