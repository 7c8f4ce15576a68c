"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: values printed in the paper,
textbook rules computed by other code (NumPy, SciPy), closed-form integrals, invariants of the
weak forms, brute-force assembly on tiny meshes, and convergence rates.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1705_08813_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------
# 1-D rules
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 12])
def test_gauss_rule_matches_numpy(n):
    x, w = O.gauss(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, 0.5 * (xr + 1.0), atol=1e-15, rtol=0)
    assert np.allclose(w, 0.5 * wr, atol=1e-15, rtol=0)
    # exact for degree 2n-1 monomials on [0, 1]
    for p in range(2 * n):
        assert abs(np.dot(w, x ** p) - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_lobatto_nodes_are_roots_of_legendre_derivative(n):
    x = O.lobatto(n)
    ref = np.sort(np.concatenate([[-1.0, 1.0], np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots()]))
    assert np.allclose(x, 0.5 * (ref + 1.0), atol=1e-14, rtol=0)


# ---------------------------------------------------------------------------------------------
# Wall laws (Sec. 3.2, Appendix A)
# ---------------------------------------------------------------------------------------------

def _table_a1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "psi_vandriest_tableA1.txt")) if l[0] != "#"]
    return np.array([[float(r[1]), float(r[2])] for r in rows])


def test_vandriest_table_chain_reproduces_printed_values():
    """psi_i + 9-point Gauss integral over [y_i, y_{i+1}] must give the printed psi_{i+1} to the
    stated 1e-12 accuracy (Appendix A, Table A1): pins the integrand, kappa, A+ and the rule."""
    t = _table_a1()
    for i in range(len(t) - 1):
        v = O.psi_vandriest_from(i, t[i + 1, 0])
        assert abs(v / t[i + 1, 1] - 1.0) <= 1e-12, (i, v, t[i + 1, 1])


def test_vandriest_against_adaptive_quadrature():
    """psi at arbitrary y+ up to 5000 against an adaptive integration (SciPy) of eq. (psi),
    anchored at the printed Table A1 values."""
    from scipy.integrate import quad
    t = _table_a1()

    def f(y):
        a = 2 * 0.41 * y * (1 - math.exp(-y / 26.0))
        return 2.0 / (1.0 + math.sqrt(1.0 + a * a))

    for yp in [0.3, 3.0, 7.5, 17.0, 40.0, 100.0, 250.0, 700.0, 1800.0, 4000.0, 5000.0]:
        i = int(np.searchsorted(t[:, 0], yp, side="right") - 1)
        ref = t[i, 1] + quad(f, t[i, 0], yp, epsabs=1e-15, epsrel=1e-15, limit=200)[0]
        v, d = O.psi_vandriest(yp)
        assert abs(v / ref - 1.0) <= 1e-12
        assert abs(d - f(yp)) <= 1e-15
    # wall behaviour u+(0) = 0, du+/dy+(0) = 1 (Sec. 3.2)
    assert O.psi_vandriest(0.0) == (0.0, 1.0)


def test_spalding_inverse_boundary_and_log_law():
    k, B = 0.41, 5.17
    assert O.psi_spalding(0.0) == (0.0, 1.0)
    v, d = O.psi_spalding(1e-6)
    assert abs(v - 1e-6) < 1e-15 and abs(d - 1.0) < 1e-5
    for yp in [1e-3, 0.5, 5.0, 11.0, 30.0, 100.0, 1e3, 5e3, 2e4]:
        psi, dpsi = O.psi_spalding(yp)
        kp = k * psi
        fwd = psi + math.exp(-k * B) * (math.exp(kp) - 1 - kp - kp ** 2 / 2 - kp ** 3 / 6)
        assert abs(fwd / yp - 1.0) < 1e-14
        # derivative against a central difference of the inverse
        h = 1e-5 * max(yp, 1.0)
        fd = (O.psi_spalding(yp + h)[0] - O.psi_spalding(yp - h)[0]) / (2 * h)
        assert abs(dpsi / fd - 1.0) < 1e-6
    # log law for large y+: psi -> ln(y+)/kappa + B
    for yp in [5e3, 2e4]:
        assert abs(O.psi_spalding(yp)[0] - (math.log(yp) / k + B)) < 0.05


# ---------------------------------------------------------------------------------------------
# Geometry (Sec. 5.1 channel; bump channel of the curved workload)
# ---------------------------------------------------------------------------------------------

def test_channel_volume_exact():
    m = O.Mesh(4, 5, 3, 3, gamma=1.8)
    assert abs(m.volume() - 4 * math.pi ** 2) < 1e-12 * 4 * math.pi ** 2


def test_bump_volume_closed_form():
    # 9 x [yw(x), 3.036] x 4.5 with yw = 0.3 cos^2(pi (x-4.5)/2) on |x-4.5| < 1: the bump area is
    # 0.3 * 1 (integral of cos^2 over one period); isoparametric Q4 mapping error is tiny.
    m = O.Mesh(24, 4, 2, 4, lx=9.0, ly=3.036, lz=4.5, geometry=1, n_layers=0)
    ref = 9.0 * 3.036 * 4.5 - 4.5 * 0.3
    assert abs(m.volume() - ref) < 1e-6 * ref


def test_bump_nodes_lie_on_the_walls_with_rows_upward():
    """Cell rows count upward from the bump wall (the layout the ABI fixes): the lowest nodes of row 0
    lie on y_w(x) = 0.3 cos^2(pi (x - 4.5) / 2) for |x - 4.5| < 1 (0 elsewhere), the highest nodes of
    the top row on y = 3.036, and every node column rises monotonically from row to row."""
    nx, ny, nz, k = 12, 4, 2, 3
    m = O.Mesh(nx, ny, nz, k, lx=9.0, ly=3.036, lz=4.5, geometry=1, n_layers=0)
    n = k + 1
    X = m.node_coords().reshape(nz, ny, nx, n, n, n, 3)        # [kz][j][i][c][b][a]
    x, y = X[..., 0], X[..., 1]
    s = x - 4.5
    yw = np.where(np.abs(s) < 1.0, 0.3 * np.cos(np.pi * s / 2.0) ** 2, 0.0)
    assert np.abs(y[:, 0, :, :, 0, :] - yw[:, 0, :, :, 0, :]).max() < 1e-14
    assert np.abs(y[:, ny - 1, :, :, n - 1, :] - 3.036).max() < 1e-14
    col = np.transpose(y, (0, 2, 3, 5, 1, 4)).reshape(nz, nx, n, n, ny * n)   # y up each node column
    assert np.all(np.diff(col, axis=-1) >= -1e-14)
    # x and z: the map is the identity along them, nodes at the Gauss-Lobatto points of each cell,
    # local index a along x and c along z ascending
    gl = O.lobatto(n)            # pinned against the roots of P'_{n-1} above
    xr = 9.0 * (np.arange(nx)[None, None, :, None, None, None] + gl[None, None, None, None, None, :]) / nx
    zr = 4.5 * (np.arange(nz)[:, None, None, None, None, None] + gl[None, None, None, :, None, None]) / nz
    assert np.abs(x - xr).max() < 1e-13 and np.abs(X[..., 2] - zr).max() < 1e-13
    assert yw.max() > 0.29


def test_penalty_on_curved_cells_against_the_mapped_cell():
    """tau = (k+1)^2 A(dK) / V(K) (interior faces weighted 1/2, walls 1) on the curved bump cells, with
    A and V integrated here to convergence (16 Gauss points per direction) over the isoparametric cell
    rebuilt from the node coordinates (Lagrange interpolation on the Gauss-Lobatto nodes, dA =
    |det J| |grad xi_d|). The oracle's k+2 point rules agree to 1e-6 (they are exact on boxes); a rule
    of k points would be off by about 2e-5."""
    nx, ny, nz, k = 12, 4, 2, 3
    m = O.Mesh(nx, ny, nz, k, lx=9.0, ly=3.036, lz=4.5, geometry=1, n_layers=0)
    n = k + 1
    X = m.node_coords().reshape(m.nc, n, n, n, 3)               # [c][cc][b][a]
    gl = O.lobatto(n)

    def lag(s):
        v, d = np.ones(n), np.zeros(n)
        for a in range(n):
            for b in range(n):
                if b != a:
                    v[a] *= (s - gl[b]) / (gl[a] - gl[b])
            for c in range(n):
                if c != a:
                    t = 1.0 / (gl[a] - gl[c])
                    for b in range(n):
                        if b != a and b != c:
                            t *= (s - gl[b]) / (gl[a] - gl[b])
                    d[a] += t
        return v, d

    def jac(c, xi):
        L = [lag(x) for x in xi]
        return np.array([[np.einsum("zyx,z,y,x", X[c, ..., e], *(L[2][dz], L[1][dy], L[0][dx]))
                          for (dx, dy, dz) in ((1, 0, 0), (0, 1, 0), (0, 0, 1))] for e in range(3)])

    q = 16
    xq, wq = np.polynomial.legendre.leggauss(q)
    xq, wq = 0.5 * (xq + 1), 0.5 * wq
    tau = m.cell_tau()
    for c in [4, 5, 6, 7, 4 + nx * (ny - 1), 5 + nx]:           # bump columns, bottom, top and inner rows
        j = (c // nx) % ny
        V = sum(abs(np.linalg.det(jac(c, (xq[a], xq[b], xq[e])))) * wq[a] * wq[b] * wq[e]
                for a in range(q) for b in range(q) for e in range(q))
        A = 0.0
        for d in range(3):
            t1, t2 = [e for e in range(3) if e != d]
            for side in (0, 1):
                wall = d == 1 and ((side == 0 and j == 0) or (side == 1 and j == ny - 1))
                for p in range(q):
                    for r in range(q):
                        xi = [0.0, 0.0, 0.0]
                        xi[d], xi[t1], xi[t2] = float(side), xq[p], xq[r]
                        J = jac(c, xi)
                        dA = abs(np.linalg.det(J)) * np.linalg.norm(np.linalg.inv(J)[d])
                        A += (1.0 if wall else 0.5) * dA * wq[p] * wq[r]
        assert abs(tau[c] / (n * n * A / V) - 1.0) < 1e-6, (c, tau[c], n * n * A / V)


# ---------------------------------------------------------------------------------------------
# SIPG Laplacian, eq. (ipflux)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("geometry", [0, 1])
def test_laplace_constants_in_null_space(geometry):
    kw = dict(lx=9.0, ly=3.036, lz=4.5, geometry=1) if geometry else {}
    m = O.Mesh(4, 3, 2, 3, n_layers=0, **kw)
    y = m.laplace(np.ones(m.n_p))
    d = m.laplace_diag()
    assert np.abs(y).max() < 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("dims,k,geometry", [((1, 1, 1), 1, 0), ((2, 1, 1), 2, 0), ((2, 3, 2), 1, 0),
                                               ((3, 2, 2), 2, 0), ((2, 2, 1), 3, 0), ((3, 2, 1), 2, 1)])
def test_laplace_bruteforce_symmetric_psd(dims, k, geometry):
    kw = dict(lx=9.0, ly=3.036, lz=4.5, geometry=1) if geometry else {}
    m = O.Mesh(*dims, k, n_layers=0, **kw)
    n = m.n_p
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        A[:, j] = m.laplace(e)
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-13 * scale
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev[0] >= -1e-12 * ev[-1]
    assert ev[1] > 1e-8 * ev[-1]            # exactly one (near-)zero eigenvalue: the constants
    assert np.allclose(np.diag(A), m.laplace_diag(), rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("op", ["laplace", "divergence", "convective", "viscous", "vmass"])
def test_default_rules_are_exact_on_box_cells(op):
    """On affine box cells without enrichment every integrand of a DG field of degree k is a
    polynomial that the method's rules integrate exactly (Sec. 4.4: k+1 Gauss points for the linear
    terms, floor(3k/2)+1 for the convective term), so adding two points per direction to every
    cell and face rule (extra_q = 2) changes no output beyond rounding, for random fields. The
    Lax-Friedrichs dissipation max(|u^-.n|, |u^+.n|) [[u]] is not a polynomial on a face where the
    normal velocity varies and jumps, so the convective case takes continuous random cubics in y,
    whose normal velocity is constant on every y-face (walls included) and whose jumps vanish inside."""
    kw = dict(n_layers=0, gamma=1.8, nu=1e-3)
    base = O.Mesh(3, 4, 2, 3, **kw)
    over = O.Mesh(3, 4, 2, 3, extra_q=2, **kw)
    p = I.uniform(21, base.n_p, -1, 1)
    u = I.uniform(22, base.n_u, -1, 1)
    if op == "convective":
        cf = I.uniform(23, 12, -1, 1).reshape(3, 4)
        u = _std_field(base, *[lambda x, y, z, a=a: cf[a, 0] + cf[a, 1] * y + cf[a, 2] * y ** 2 + cf[a, 3] * y ** 3
                               for a in range(3)])
    f = {"laplace": lambda m: m.laplace(p), "divergence": lambda m: m.divergence(u),
         "convective": lambda m: m.convective(u), "viscous": lambda m: m.viscous(u, u),
         "vmass": lambda m: m.vmass(u)}[op]
    a, b = f(base), f(over)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max(), op


def test_laplace_bilinear_form_of_smooth_fields_closed_form():
    """For continuous fields the SIPG face terms vanish and q^T A p = int grad q . grad p."""
    m = O.Mesh(3, 5, 2, 3, n_layers=0, gamma=1.8)
    X = m.node_coords()
    y = X[:, 1]
    q = y ** 2
    p = y ** 2 + y
    val = q @ m.laplace(p)
    ref = (2 * math.pi) * math.pi * (8.0 / 3.0)      # Lx Lz int_{-1}^{1} 2y (2y + 1) dy
    assert abs(val - ref) < 1e-12 * ref


@pytest.mark.slow
@pytest.mark.parametrize("k,n0,gamma", [(1, 8, 1e-3), (2, 4, 1.0), (3, 3, 1.0)])
def test_laplace_manufactured_solution_converges_at_k_plus_1(k, n0, gamma):
    """p* = cos(pi y) cos(x) cos(2z) (zero mean, homogeneous Neumann at y = +-1). k = 1 needs
    finer meshes to leave the pre-asymptotic range, so it runs on a uniform mesh."""
    errs = []
    for n in (n0, 2 * n0):
        m = O.Mesh(n, n, n, k, n_layers=0, gamma=gamma)
        X = m.node_coords()
        ps = np.cos(math.pi * X[:, 1]) * np.cos(X[:, 0]) * np.cos(2 * X[:, 2])
        b = m.mass((math.pi ** 2 + 5.0) * ps)
        p, it, rr = m.solve(b, rtol=1e-12)
        assert rr <= 1e-11
        e = p - ps
        e -= np.sum(m.mass(e)) / m.volume()
        errs.append(math.sqrt(e @ m.mass(e)))
    rate = math.log2(errs[0] / errs[1])
    assert rate >= k + 1 - 0.3, (errs, rate)


# ---------------------------------------------------------------------------------------------
# Velocity divergence (Sec. 4.2)
# ---------------------------------------------------------------------------------------------

def _std_field(m, fx, fy, fz):
    X = m.node_coords()
    n3 = (m.k + 1) ** 3
    u = np.zeros(m.n_u)
    std = u[: 3 * m.n_p].reshape(m.nc, 3, n3)
    for a, f in enumerate((fx, fy, fz)):
        std[:, a, :] = f(X[:, 0], X[:, 1], X[:, 2]).reshape(m.nc, n3)
    return u


def test_constant_fields_on_curved_cells():
    """On the isoparametric bump cells the metric terms of a constant field integrate exactly (the
    cofactors of a Q_k map times a derivative of the basis stay within the k+1 point rules), so the
    discrete integration by parts holds cell by cell: the divergence of a constant vector is zero in
    every output (wall faces use {{u}} = u^-), and the convective term of a constant vector is zero in
    every cell without a wall face (interior fluxes u (u.n) match the volume term). A wrong face
    normal, area weight or inverse Jacobian on a curved face breaks both."""
    m = O.Mesh(12, 4, 2, 3, lx=9.0, ly=3.036, lz=4.5, geometry=1, n_layers=0)
    c = np.array([0.7, -0.4, 0.25])
    u = np.zeros(m.n_u)
    u[: 3 * m.n_p].reshape(m.nc, 3, -1)[:] = c[None, :, None]
    scale = np.abs(m.divergence(I.uniform(3, m.n_u, -1, 1))).max()
    assert np.abs(m.divergence(u)).max() < 1e-13 * scale
    y = m.convective(u)[: 3 * m.n_p].reshape(m.nc, 3, -1)
    j = (np.arange(m.nc) // 12) % 4
    inner = (j > 0) & (j < 3)
    assert np.abs(y[~inner]).max() > 1e-3             # the mirrored walls do carry a flux
    assert np.abs(y[inner]).max() < 1e-13 * np.abs(y[~inner]).max()


def test_divergence_closed_form_with_wall_flux():
    """For continuous u: sum_i q_i b_i = -int q div(u); the wall rule {{u}} = u^- matters since
    u.n != 0 on the walls."""
    m = O.Mesh(3, 4, 2, 2, n_layers=0)
    u = _std_field(m, lambda x, y, z: y ** 2, lambda x, y, z: 1 + y ** 2, lambda x, y, z: y + 0 * x)
    q = m.node_coords()[:, 1] + 1.0
    val = q @ m.divergence(u)
    ref = -(2 * math.pi * math.pi) * (4.0 / 3.0)      # -Lx Lz int 2y (y+1) dy
    assert abs(val - ref) < 1e-12 * abs(ref)


def test_divergence_enrichment_volume_term():
    """u = psi(y+) e_y from enrichment only: with q = y the face terms cancel or vanish (psi(0)=0)
    and sum_i q_i b_i = int_{wall cells} psi(y+) dV (compare with adaptive quadrature of psi)."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    u = np.zeros(m.n_u)
    enr = u[3 * m.n_p:].reshape(m.n_e, 3, 8)
    enr[:, 1, :] = 1.0
    q = m.node_coords()[:, 1]
    val = q @ m.divergence(u)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    ref = 2 * (2 * math.pi * math.pi) * quad(lambda s: O.psi_spalding(s * w.u_tau / w.nu)[0], 0.0, dy,
                                             epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    assert abs(val / ref - 1.0) < 1e-6, (val, ref)


@pytest.mark.parametrize("comp", [0, 2])
def test_divergence_enrichment_tangential_components(comp):
    """Enrichment along x (or z) with vertex coefficients f = cos(2 pi s / L) of the vertex coordinate
    s: u = psi(y+) F(s) e_s, F the piecewise-linear interpolant of f, continuous and periodic. With the
    continuous periodic q = G(s), G interpolating g = sin(2 pi s / L), every face term cancels or has
    u.n = 0, so sum_i q_i b_i = int G'(s) F(s) psi dV
    = 2 L_t int_0^dy psi dy * sum_cells (g_{i+1} - g_i)(f_i + f_{i+1}) / 2 (L_t the other in-plane
    length), the psi integral by adaptive quadrature."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    nx, nz = w.nx, w.nz
    L, Lt, ncs = (w.lx, w.lz, nx) if comp == 0 else (w.lz, w.lx, nz)
    h = L / ncs
    f = lambda s: np.cos(2 * np.pi * s / L)
    g = lambda s: np.sin(2 * np.pi * s / L)
    u = np.zeros(m.n_u)
    enr = u[3 * m.n_p:].reshape(m.n_e, 3, 8)
    for layer in range(2):                      # enriched cells: bottom layer, then top, x fastest
        for kz in range(nz):
            for i in range(nx):
                e = layer * nx * nz + i + nx * kz
                for v in range(8):
                    vx, vz = v & 1, (v >> 2) & 1
                    s = (i + vx) * h if comp == 0 else (kz + vz) * h
                    enr[e, comp, v] = f(s)
    s = m.node_coords()[:, comp]
    n3 = (w.k + 1) ** 3
    c = np.repeat(np.arange(m.nc), n3)          # nodes are stored cell by cell, cells x fastest
    ci = c % nx if comp == 0 else c // (nx * w.ny)
    t = s / h - ci
    q = g(ci * h) + (g((ci + 1) * h) - g(ci * h)) * t
    val = q @ m.divergence(u)
    edges = np.arange(ncs) * h
    lin = np.sum((g(edges + h) - g(edges)) * (f(edges) + f(edges + h)) / 2.0)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    ipsi = quad(lambda y: O.psi_spalding(y * w.u_tau / w.nu)[0], 0.0, dy, epsabs=1e-14, epsrel=1e-13,
                limit=200)[0]
    ref = 2 * Lt * ipsi * lin
    assert abs(ref) > 1e-3
    assert abs(val / ref - 1.0) < 1e-6, (val, ref)


# ---------------------------------------------------------------------------------------------
# Velocity mass term (Sec. 4.2, M_e(v, u) = (v, u) per cell)
# ---------------------------------------------------------------------------------------------
def test_vmass_standard_part_integrates_polynomials():
    """Sum_i phi_i = 1: summing M u over the standard test functions of component a gives int u_a,
    exact for a polynomial field (the channel volume factor 2 pi^2 times the y-integral)."""
    m = O.Mesh(3, 4, 2, 2, n_layers=0)
    u = _std_field(m, lambda x, y, z: y ** 2, lambda x, y, z: 1 + 0 * y, lambda x, y, z: y + 0 * x)
    y = m.vmass(u)[: 3 * m.n_p].reshape(m.nc, 3, -1)
    ref = [(2 * math.pi * math.pi) * (2.0 / 3.0), (2 * math.pi * math.pi) * 2.0, 0.0]
    for a in range(3):
        assert abs(y[:, a, :].sum() - ref[a]) < 1e-12 * 2 * math.pi * math.pi * 2


def test_vmass_enrichment_integrates_psi():
    """u = psi(y+) e_x from enrichment only (all 8 weights 1): the standard test functions of component
    x sum to int_{wall cells} psi dV and the enriched ones psi N_B (sum_B N_B = 1) to int psi^2 dV -
    both compared with adaptive quadrature of Spalding's law; the other components stay zero."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    u = np.zeros(m.n_u)
    enr = u[3 * m.n_p:].reshape(m.n_e, 3, 8)
    enr[:, 0, :] = 1.0
    y = m.vmass(u)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    ref = 2 * (2 * math.pi * math.pi) * quad(lambda s: O.psi_spalding(s * w.u_tau / w.nu)[0], 0.0, dy,
                                             epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    std = y[: 3 * m.n_p].reshape(m.nc, 3, -1)
    ye = y[3 * m.n_p:].reshape(m.n_e, 3, 8)
    assert abs(std[:, 0, :].sum() / ref - 1.0) < 1e-6
    ref2 = 2 * (2 * math.pi * math.pi) * quad(lambda s: O.psi_spalding(s * w.u_tau / w.nu)[0] ** 2, 0.0, dy,
                                              epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    assert abs(ye[:, 0, :].sum() / ref2 - 1.0) < 1e-6
    assert np.abs(std[:, 1:, :]).max() == 0.0 and np.abs(ye[:, 1:, :]).max() == 0.0


@pytest.mark.parametrize("geometry", [0, 1])
def test_vmass_symmetric_positive_definite(geometry):
    """(v, u) is a symmetric positive definite bilinear form on standard plus enriched DoFs:
    brute-force assembly on a tiny mesh."""
    kw = dict(lx=9.0, ly=3.036, lz=4.5, geometry=1) if geometry else {}
    m = O.Mesh(2, 2, 1, 1, nu=1e-3, tau_w=1e-2, **kw)
    A = np.column_stack([m.vmass(e) for e in np.eye(m.n_u)])
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0.0


# ---------------------------------------------------------------------------------------------
# Convective term (Sec. 4.2, local Lax-Friedrichs flux)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("comp", [0, 2])
def test_convective_vanishes_for_shear_flow_with_enrichment(comp):
    """u = f(y) e_c (standard part) + u_tau psi(y+) e_c (enrichment), c = x or z: div(u x u) = 0
    and u.n = 0 on y-faces, so F^c(v, u) = 0 for every standard and enriched test function. The
    discrete integration by parts along c holds only if the faces normal to c use the same
    wall-normal rule as the volume (Sec. 4.4)."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    f = [lambda x, y, z: 0 * y] * 3
    f[comp] = lambda x, y, z: 1 - y ** 2
    u = _std_field(m, *f)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, comp, :] = w.u_tau
    y = m.convective(u)
    assert np.abs(y).max() < 1e-14


@pytest.mark.parametrize("k,f,g,w", [
    (2, lambda y: 1 + y + y ** 2, lambda y: 1 - y ** 2, lambda y: y ** 2),
    (3, lambda y: 1 + y + y ** 3, lambda y: y - y ** 3, lambda y: y ** 3)], ids=["k2", "k3"])
def test_convective_over_integration_is_exact_for_polynomials(k, f, g, w):
    """Sec. 4.4 over-integrates the convective term with floor(3k/2) + 1 points per direction, which
    integrates (u x u) : grad v (degree 3k - 1 per direction) exactly for fields of degree k. With
    u = (f(y), g(y), 0) (continuous, g(+-1) = 0 so u.n = 0 on the walls and every face term cancels or
    vanishes) and the continuous test field w(y) for component x:
    sum_i w_i y_x[i] = -L_x L_z int f g w' dy, which is -(8/15) L_x L_z for both cases:
    k = 2: (1 + y + y^2)(1 - y^2) 2y, k = 3: (1 + y + y^3)(y - y^3) 3y^2 (degree 8 on the graded,
    affine-per-cell rows: k + 1 = 4 points are not exact, 5 are)."""
    m = O.Mesh(3, 5, 2, k, n_layers=0, gamma=1.8)
    u = _std_field(m, lambda x, y, z: f(y), lambda x, y, z: g(y), lambda x, y, z: 0 * y)
    y = m.convective(u)[: 3 * m.n_p].reshape(m.nc, 3, -1)
    wy = w(m.node_coords()[:, 1]).reshape(m.nc, -1)
    val = np.sum(wy * y[:, 0, :])
    ref = -(8.0 / 15.0) * 2 * math.pi * math.pi
    assert abs(val - ref) < 1e-12 * abs(ref), (val, ref)


def test_convective_wall_normal_transport_by_the_enrichment():
    """u = e_x (standard part) plus a wall-normal enrichment u_y = c psi(y+) (1 - eta) in the bottom
    wall cells (weights c on the wall-side vertices, 0 on the others; eta the cell's local y). The field
    is continuous (psi(0) = 0 on the wall, the weights vanish at the cell's upper face) and u.n = 0 on
    the walls, so every face term cancels and, with the continuous test field w = y for component x,
    sum_i w_i y_x[i] = -int u_x u_y dV = -c L_x L_z int_0^dy psi (1 - s/dy) ds. With the enriched test
    functions of component x summed over the bottom layer (the test function psi e_x) the interface
    flux is u_x u_y = 0 there, so the sum is -int u_y dpsi/dy dV
    = -c L_x L_z (u_tau/nu) int_0^dy psi psi' (1 - s/dy) ds. Both integrals by adaptive quadrature; the
    second also by the 8-point Gauss rule of the wall-normal direction, which the oracle must match to
    rounding."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    c = 0.37
    u = _std_field(m, lambda x, y, z: 1 + 0 * y, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    enr = u[3 * m.n_p:].reshape(m.n_e, 3, 8)
    nb = w.nx * w.nz                            # bottom layer first
    for v in range(8):
        if (v >> 1) & 1 == 0:
            enr[:nb, 1, v] = c
    y = m.convective(u)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    sc = w.u_tau / w.nu
    area = w.lx * w.lz
    std = y[: 3 * m.n_p].reshape(m.nc, 3, -1)
    wy = m.node_coords()[:, 1].reshape(m.nc, -1)
    val = np.sum(wy * std[:, 0, :])
    ref = -c * area * quad(lambda s: O.psi_spalding(s * sc)[0] * (1 - s / dy), 0.0, dy,
                           epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    assert abs(val / ref - 1.0) < 1e-6, (val, ref)
    ye = y[3 * m.n_p:].reshape(m.n_e, 3, 8)
    val_e = ye[:nb, 0, :].sum()
    f = lambda s: np.prod(O.psi_spalding(s * sc)) * (1 - s / dy)
    ref_e = -c * area * sc * quad(f, 0.0, dy, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    assert abs(val_e / ref_e - 1.0) < 2e-5, (val_e, ref_e)   # psi psi' is less smooth: rule error
    # the same integral by the q_w = 8 point Gauss rule (NumPy) the wall cells use wall-normal
    xg, wg = np.polynomial.legendre.leggauss(8)
    rule = -c * area * sc * 0.5 * dy * sum(wq * f(0.5 * dy * (xq + 1)) for xq, wq in zip(xg, wg))
    assert abs(val_e / rule - 1.0) < 1e-12, (val_e, rule)


@pytest.mark.parametrize("b,total", [(0.0, 16.0), (1.0, 28.0)])
def test_convective_conservation_equals_wall_flux(b, total):
    """sum over all standard test functions of component d = sum of wall fluxes (interior fluxes
    cancel). With the mirror state u+ = -u- the wall flux is u_y (u.n) + 2 |u.n| u_y. For
    u = (0, 1 + b y + y^2, 0): b = 0 gives 12 (top, u_y = 2) + 4 (bottom); b = 1 gives 27 (top, u_y = 3)
    + 1 (bottom, u_y = 1), which also fixes the sign of u.n on the y-faces."""
    m = O.Mesh(2, 3, 2, 2, n_layers=0)
    u = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: 1 + b * y + y ** 2, lambda x, y, z: 0 * y)
    y = m.convective(u)[: 3 * m.n_p].reshape(m.nc, 3, -1)
    sums = y.sum(axis=(0, 2))
    area = 2 * math.pi * math.pi
    assert abs(sums[1] - total * area) < 1e-12 * total * area
    assert abs(sums[0]) < 1e-12 and abs(sums[2]) < 1e-12


@pytest.mark.parametrize("alpha,beta", [(0.3, 0.7), (0.8, 0.25)])
def test_convective_interior_flux_with_sign_changing_normal_velocity(alpha, beta):
    """Two cells along x (periodic, so both x-faces are interior), constant u = alpha e_x in cell 0
    and -beta e_x in cell 1: on every x-face u^-.n and u^+.n have opposite signs. The local
    Lax-Friedrichs flux of Sec. 4.2, F = 1/2 (u^- (u^-.n) + u^+ (u^+.n)) + Lambda/2 (u^- - u^+) with
    Lambda = max(2|u^-.n|, 2|u^+.n|), is evaluated here by hand; y- and z-faces carry no flux
    (u.n = 0 on both sides). With Gauss-Lobatto nodes the integral of a nodal basis function over a
    face is the product of the 1-D Lobatto weights, so every output has a closed form:
    y_{c,x,(a,b,c)} = W_bc [delta_{a,k} (F_R - u_c^2) + delta_{a,0} (F_L + u_c^2)], u_c the cell's
    x-velocity, F_R, F_L the x-fluxes through its right and left face (outward normals)."""
    k = 2
    m = O.Mesh(2, 1, 1, k, n_layers=0)
    n = k + 1
    u = np.zeros(m.n_u)
    std = u[: 3 * m.n_p].reshape(m.nc, 3, n ** 3)
    uc = [alpha, -beta]
    std[0, 0, :] = uc[0]
    std[1, 0, :] = uc[1]
    y = m.convective(u)[: 3 * m.n_p].reshape(m.nc, 3, n, n, n)   # [cell][comp][z][y][x]

    def flux(um, up, nrm):
        unm, unp = um * nrm, up * nrm
        lam = max(2 * abs(unm), 2 * abs(unp))
        return 0.5 * (um * unm + up * unp) + 0.5 * lam * (um - up)

    # independent Lobatto weights on [0, 1]: integrals of the Lagrange polynomials on the nodes
    z = np.concatenate(([-1.0], np.polynomial.legendre.Legendre.basis(k).deriv().roots(), [1.0]))
    wl = 2.0 / (k * (k + 1) * np.polynomial.legendre.legval(z, [0] * k + [1]) ** 2) / 2.0
    W = np.outer(wl, wl) * (2.0 * math.pi)          # [z][y] weights times the face area Ly Lz
    for c in range(2):
        o = 1 - c
        FR = flux(uc[c], uc[o], 1.0)                   # right face: n = +e_x
        FL = flux(uc[c], uc[o], -1.0)                  # left face: n = -e_x
        ref = np.zeros((n, n, n))
        ref[:, :, k] = W * (FR - uc[c] ** 2)
        ref[:, :, 0] = W * (FL + uc[c] ** 2)
        assert np.abs(y[c, 0] - ref).max() < 1e-13 * np.abs(ref).max()
        assert np.abs(y[c, 1:]).max() < 1e-14
        # the cell's total: the hand value 2 max(alpha, beta) (alpha + beta) L_y L_z with the sign
        # of its own velocity (a min in Lambda or a dropped 1/2 changes it)
        tot = y[c, 0].sum()
        expect = (1 if c == 0 else -1) * 2 * max(alpha, beta) * (alpha + beta) * 2 * math.pi
        assert abs(tot - expect) < 1e-13 * abs(expect)


# ---------------------------------------------------------------------------------------------
# Viscous multiscale term, eq. (viscous_multiscale)
# ---------------------------------------------------------------------------------------------

def test_viscous_bilinear_form_of_smooth_fields_closed_form():
    """No enrichment, continuous u and v vanishing on the walls: all face terms vanish and
    -F^nu(v, u) = int 2 nu eps(v):eps(u) = nu Lx Lz int u_x' v_x' dy."""
    nu = 1e-3
    m = O.Mesh(2, 3, 2, 3, n_layers=0, nu=nu)
    u = _std_field(m, lambda x, y, z: 1 - y ** 2, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    v = _std_field(m, lambda x, y, z: (1 - y ** 2) * (1 + y), lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    val = v @ m.viscous(np.zeros(m.n_u), u)
    ref = nu * 2 * math.pi * math.pi * (8.0 / 3.0)
    assert abs(val / ref - 1.0) < 1e-12


def test_viscous_wall_penalty_on_constant_field():
    """u = v = e_x: eps = 0, interior jumps 0; the mirror gives [[u]] = 2 e_x on both walls, so
    -F^nu(v,u) = sum_walls int 10 tau nu * 2 (penalty x10 on Dirichlet faces, Sec. 4.2)."""
    nu = 1e-3
    m = O.Mesh(2, 3, 2, 2, n_layers=0, nu=nu)
    one = lambda x, y, z: 1 + 0 * y
    zero = lambda x, y, z: 0 * y
    u = _std_field(m, one, zero, zero)
    val = u @ m.viscous(np.zeros(m.n_u), u)
    tau = m.cell_tau().reshape(2, 3, 2)      # [z][y][x]
    area_cell = (2 * math.pi / 2) * (math.pi / 2)
    ref = sum(10.0 * tau[:, j, :].sum() * nu * 2.0 * area_cell for j in (0, 2))
    assert abs(val / ref - 1.0) < 1e-12


def test_viscous_symmetric_part_is_volume_plus_penalty_and_psd():
    """Skew-symmetric consistency/adjoint pairs (Sec. 4.2-4.3): the symmetric part of -F^nu
    couples neighbouring cells only through penalty terms (standard functions not on the shared
    face have zero coupling), and it is positive semi-definite with the clipped viscosity."""
    nu = 1e-4
    m = O.Mesh(2, 3, 2, 2, n_layers=1, nu=nu, tau_w=1e-2, gamma=1.8)
    uf = np.zeros(m.n_u)
    uf[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = 0.1
    uf[3 * m.n_p:] += 0.02 * I.uniform(5, m.n_e * 24, -1, 1)
    n = m.n_u
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        A[:, j] = m.viscous(uf, e)
    S = 0.5 * (A + A.T)
    ev = np.linalg.eigvalsh(S)
    assert ev[0] >= -1e-11 * ev[-1]
    # the clip must actually be active somewhere for this frozen field (nu_t > 3 nu)
    assert max(m.nut_cell(uf, e).max() for e in range(m.n_e)) > 3 * nu
    # structural zeros: x-neighbours (0,j,k) and (1,j,k); local nodes with lx = 0 of cell 0 lie on
    # the face shared through the periodic boundary, lx = 2 on the interior face; lx = 1 is on
    # neither, so its symmetric coupling to every standard function of cell 1 must vanish.
    n1, n3 = 3, 27
    lx = np.arange(n3) % n1
    for comp in range(3):
        rows = 0 * 3 * n3 + comp * n3 + np.where(lx == 1)[0]
        cols = np.arange(1 * 3 * n3, 2 * 3 * n3)
        assert np.abs(S[np.ix_(rows, cols)]).max() <= 1e-14 * np.abs(S).max()
    # and the skew part does couple them (the consistency/adjoint terms are present)
    K = 0.5 * (A - A.T)
    rows = np.where(lx == 1)[0]
    assert np.abs(K[np.ix_(rows, np.arange(3 * n3, 6 * n3))]).max() > 1e-6 * np.abs(S).max()


class _BoxFields:
    """Independent evaluation (NumPy, not the oracle's tabulation) of ubar, u~ and their physical
    gradients at reference points of the box cells of a channel mesh with one enriched layer per
    wall and a constant wall shear stress tau_w: Lagrange polynomials on Gauss-Lobatto nodes for
    ubar (Sec. 4.2), u~ = psi(y+) sum_B N_B u~_B with y_h the distance to the wall and
    y+ = y_h sqrt(tau_w) / nu, grad u~ = sum_B u~_B (psi grad N_B + N_B psi' grad y+) (Sec. 3.1-3.2).
    psi and psi' come from the wall-law routine pinned on its own (Spalding)."""

    def __init__(self, m, nx, ny, nz, k, nu, tau_w):
        self.m, self.nx, self.ny, self.nz, self.k, self.nu, self.tau_w = m, nx, ny, nz, k, nu, tau_w
        self.n = k + 1
        z = np.concatenate(([-1.0], np.polynomial.legendre.Legendre.basis(k).deriv().roots(), [1.0]))
        self.gll = 0.5 * (np.sort(z) + 1.0)
        X = m.node_coords().reshape(m.nc, -1, 3)
        self.lo, self.hi = X.min(axis=1), X.max(axis=1)

    def lagrange(self, s):
        """values and derivatives of the n Lagrange polynomials on the Lobatto nodes at s"""
        x, n = self.gll, self.n
        v, d = np.ones(n), np.zeros(n)
        for a in range(n):
            for b in range(n):
                if b == a:
                    continue
                v[a] *= (s - x[b]) / (x[a] - x[b])
            for c in range(n):
                if c == a:
                    continue
                t = 1.0 / (x[a] - x[c])
                for b in range(n):
                    if b != a and b != c:
                        t *= (s - x[b]) / (x[a] - x[b])
                d[a] += t
        return v, d

    def enr_index(self, c):
        i, j, kz = c % self.nx, (c // self.nx) % self.ny, c // (self.nx * self.ny)
        if j == 0:
            return i + self.nx * kz
        if j == self.ny - 1:
            return self.nx * self.nz + i + self.nx * kz
        return -1

    def eval(self, u, c, xi):
        """(ubar, grad ubar, u~, grad u~) at reference point xi of cell c; G[a][e] = d u_a / d x_e"""
        m, n = self.m, self.n
        h = self.hi[c] - self.lo[c]
        L = [self.lagrange(xi[d]) for d in range(3)]
        U = u[: 3 * m.n_p].reshape(m.nc, 3, n, n, n)[c]           # [comp][z][y][x]
        ub = np.einsum("azyx,z,y,x->a", U, L[2][0], L[1][0], L[0][0])
        gb = np.stack([np.einsum("azyx,z,y,x->a", U, L[2][0], L[1][0], L[0][1]) / h[0],
                       np.einsum("azyx,z,y,x->a", U, L[2][0], L[1][1], L[0][0]) / h[1],
                       np.einsum("azyx,z,y,x->a", U, L[2][1], L[1][0], L[0][0]) / h[2]], axis=1)
        ut, gt = np.zeros(3), np.zeros((3, 3))
        e = self.enr_index(c)
        if e >= 0:
            y = self.lo[c][1] + xi[1] * h[1]
            bottom = (c // self.nx) % self.ny == 0
            yh = y + 1.0 if bottom else 1.0 - y
            st = math.sqrt(self.tau_w)
            yp = yh * st / self.nu
            gyp = np.array([0.0, (1.0 if bottom else -1.0) * st / self.nu, 0.0])
            psi, dpsi = O.psi_spalding(yp)
            E = u[3 * m.n_p:].reshape(-1, 3, 8)[e]
            for v in range(8):
                f = [xi[d] if (v >> d) & 1 else 1.0 - xi[d] for d in range(3)]
                df = [1.0 if (v >> d) & 1 else -1.0 for d in range(3)]
                N = f[0] * f[1] * f[2]
                gN = np.array([df[0] * f[1] * f[2] / h[0], f[0] * df[1] * f[2] / h[1], f[0] * f[1] * df[2] / h[2]])
                ut += psi * N * E[:, v]
                gt += np.outer(E[:, v], psi * gN + N * dpsi * gyp)
        return ub, gb, ut, gt


def _eps(G):
    return 0.5 * (G + G.T)


def test_viscous_energy_identity_as_a_value():
    """Energy identity of eq. (viscous_multiscale) (Sec. 4.2-4.3, P7): testing -F^nu with u itself,
    every consistency term cancels against the adjoint term of the other side (also on the
    mirrored walls), so
      u^T (-F^nu) u = sum_points dV [2 nu eps(ubar):eps(ubar) + 2 nuhat eps(ubar):eps(u~)
                                     + 2 (nu + nu_t) eps(u~):eps(u~)]
                      + sum_interior faces int tau_F nu |u^- - u^+|^2 + sum_walls int 2 tau_F nu |u^-|^2,
    nuhat = min(nu + nu_t, 2 sqrt(nu (nu + nu_t))) (eq. minvt), tau_F = max(tau^-, tau^+) inside and
    10 tau on walls. The right side is summed here from the independent point evaluation, with the
    same quadrature (k+1 Gauss points, q_w wall-normal in and next to enriched cells), nu_t from
    the frozen field, and tau from its definition (k+1)^2 A/V. The clip is active (nu_t > 3 nu) and
    the ubar/u~ cross term is large, so exchanging nuhat and nu + nu_t in the two enriched volume
    terms changes the value by far more than the tolerance (asserted below)."""
    nx, ny, nz, k, qw = 2, 3, 2, 2, 8
    nu, tau_w = 1e-4, 1e-2
    m = O.Mesh(nx, ny, nz, k, n_layers=1, nu=nu, tau_w=tau_w, gamma=1.8, q_wall=qw)
    uf = np.zeros(m.n_u)
    uf[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = 0.1
    uf[3 * m.n_p:] += 0.02 * I.uniform(5, m.n_e * 24, -1, 1)
    u = I.uniform(6, m.n_u, -1, 1)
    u[3 * m.n_p:] *= 0.5
    val = u @ m.viscous(uf, u)
    F = _BoxFields(m, nx, ny, nz, k, nu, tau_w)
    n = k + 1
    # penalty parameter from its definition: (k+1)^2 A(dK)/V(K), interior faces weighted 1/2
    tau = np.zeros(m.nc)
    for c in range(m.nc):
        h = F.hi[c] - F.lo[c]
        j = (c // nx) % ny
        A = 0.0
        for d in range(3):
            t = [e for e in range(3) if e != d]
            for side in (0, 1):
                wall = d == 1 and ((side == 0 and j == 0) or (side == 1 and j == ny - 1))
                A += (1.0 if wall else 0.5) * h[t[0]] * h[t[1]]
        tau[c] = n * n * A / np.prod(h)
    assert np.abs(tau - m.cell_tau()).max() < 1e-12 * tau.max()

    def gauss(q):
        x, w = np.polynomial.legendre.leggauss(q)
        return 0.5 * (x + 1), 0.5 * w

    vol = np.zeros(3)      # the three volume parts: nu eps(ub):eps(ub), nuhat cross, (nu+nut) eps(ut):eps(ut)
    swapped = 0.0
    for c in range(m.nc):
        h = F.hi[c] - F.lo[c]
        e = F.enr_index(c)
        nq = [n, qw if e >= 0 else n, n]
        (x0, w0), (x1, w1), (x2, w2) = gauss(nq[0]), gauss(nq[1]), gauss(nq[2])
        nut = m.nut_cell(uf, e).reshape(nq[2], nq[1], nq[0]) if e >= 0 else None
        for i2 in range(nq[2]):
            for i1 in range(nq[1]):
                for i0 in range(nq[0]):
                    dV = np.prod(h) * w0[i0] * w1[i1] * w2[i2]
                    ub, gb, ut, gt = F.eval(u, c, (x0[i0], x1[i1], x2[i2]))
                    eb, et = _eps(gb), _eps(gt)
                    vol[0] += dV * 2 * nu * np.sum(eb * eb)
                    if e >= 0:
                        nt = nut[i2, i1, i0]
                        nuh = min(nu + nt, 2 * math.sqrt(nu * (nu + nt)))
                        vol[1] += dV * 2 * nuh * np.sum(eb * et)
                        vol[2] += dV * 2 * (nu + nt) * np.sum(et * et)
                        swapped += dV * (2 * (nu + nt) * np.sum(eb * et) + 2 * nuh * np.sum(et * et))
    pen = 0.0
    for c in range(m.nc):
        i, j, kz = c % nx, (c // nx) % ny, c // (nx * ny)
        h = F.hi[c] - F.lo[c]
        for d in range(3):
            for side in (0, 1):
                # every interior face once (from its lower cell), both walls
                if d == 1:
                    jn = j + (1 if side else -1)
                    if 0 <= jn < ny and side == 0:
                        continue
                    nb = None if not (0 <= jn < ny) else i + nx * (jn + ny * kz)
                elif side == 0:
                    continue
                else:
                    nb = ((i + 1) % nx + nx * (j + ny * kz)) if d == 0 else (i + nx * (j + ny * ((kz + 1) % nz)))
                t1 = 1 if d == 0 else 0
                t2 = 1 if d == 2 else 2
                enr = F.enr_index(c) >= 0 or (nb is not None and F.enr_index(nb) >= 0)
                q1 = qw if (t1 == 1 and enr) else n
                q2 = qw if (t2 == 1 and enr) else n
                (a1, b1), (a2, b2) = gauss(q1), gauss(q2)
                for p2 in range(q2):
                    for p1 in range(q1):
                        xi = [0.0, 0.0, 0.0]
                        xi[d] = float(side)
                        xi[t1], xi[t2] = a1[p1], a2[p2]
                        dA = h[t1] * h[t2] * b1[p1] * b2[p2]
                        ub, _, ut, _ = F.eval(u, c, xi)
                        um = ub + ut
                        if nb is None:
                            pen += dA * 2 * 10 * tau[c] * nu * um @ um
                        else:
                            xo = list(xi)
                            xo[d] = 1.0 - side
                            ubo, _, uto, _ = F.eval(u, nb, xo)
                            jmp = um - ubo - uto
                            pen += dA * max(tau[c], tau[nb]) * nu * jmp @ jmp
    ref = vol.sum() + pen
    assert abs(val - ref) < 1e-12 * abs(ref), (val, ref)
    # the identity distinguishes the two enriched volume coefficients
    alt = vol[0] + swapped + pen
    assert abs(alt - ref) > 1e-6 * abs(ref)
    assert max(m.nut_cell(uf, e).max() for e in range(m.n_e)) > 3 * nu


def _nut_point(F, uf, c, xi):
    """nu_t = l_mix^2 sqrt(2 eps(u~):eps(u~)) of the frozen field at reference point xi of cell c
    (eq. mix, lmix, ydes: kappa = 0.41, A+ = 26, C_DES = 0.85, beta = 6, h = cell height / (k+1)),
    from the independent point evaluation; 0 outside the enriched cells."""
    if F.enr_index(c) < 0:
        return 0.0
    _, _, _, gt = F.eval(uf, c, xi)
    et = _eps(gt)
    h = F.hi[c] - F.lo[c]
    y = F.lo[c][1] + xi[1] * h[1]
    yh = y + 1.0 if (c // F.nx) % F.ny == 0 else 1.0 - y
    yp = yh * math.sqrt(F.tau_w) / F.nu
    hd = 0.85 * h[1] / (F.k + 1)
    ydes = (yh ** -6 + hd ** -6) ** (-1.0 / 6.0) if yh > 0 else 0.0
    lmix = 0.41 * ydes * (1.0 - math.exp(-yp / 26.0))
    return lmix * lmix * math.sqrt(2.0 * np.sum(et * et))


def test_viscous_bilinear_form_with_harmonic_mean_viscosity():
    """The whole bilinear form v^T (-F^nu) u of eq. (viscous_multiscale) for independent random v and u
    and a frozen field whose nu_t differs from cell to cell, summed here from the independent point
    evaluation. On faces between two enriched cells (and on their mirrored walls) the weighted average
    of eq. (harmweights), w^- = (nu + nu_t^+) / (2 nu + nu_t^- + nu_t^+), makes every weighted flux
    w^- kappa^- = w^+ kappa^+ = H / 2 with H = 2 kappa^- kappa^+ / (kappa^- + kappa^+) the harmonic
    mean of kappa = nu + nu_t of the two sides; this reference is written in that form:
      consistency  -(H/2) (2 eps(u~^-) + 2 eps(u~^+)) n . v^-,
      adjoint       (H/2) (grad v~^- n . [[u]] + n . grad v~^- [[u]]),
    together with the standard average nu (eps(ubar^-) + eps(ubar^+)) n, the standard adjoint term
    nu/2 (grad vbar n . j + n . grad vbar j) (j = [[ubar]], plus [[u~]] on the interface faces), the
    interface term -nu (eps(ubar^-) + eps(ubar^+)) n . v~^-, and the penalty tau nu [[u]] . v^-
    (tau = max of both sides inside, 10 tau on walls). Volume: 2 nu eps(vbar):eps(ubar)
    + 2 nuhat eps(vbar):eps(u~) + 2 (nu + nu_t) eps(v~):eps(u~). Replacing the harmonic mean by the
    arithmetic one changes the value by far more than the tolerance (asserted)."""
    nx, ny, nz, k, qw = 2, 3, 2, 2, 8
    nu, tau_w = 1e-4, 1e-2
    m = O.Mesh(nx, ny, nz, k, n_layers=1, nu=nu, tau_w=tau_w, gamma=1.8, q_wall=qw)
    uf = np.zeros(m.n_u)
    uf[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = 0.1
    uf[3 * m.n_p:] += 0.1 * I.uniform(7, m.n_e * 24, -1, 1)
    u = I.uniform(8, m.n_u, -1, 1)
    v = I.uniform(9, m.n_u, -1, 1)
    val = v @ m.viscous(uf, u)
    F = _BoxFields(m, nx, ny, nz, k, nu, tau_w)
    n = k + 1
    tau = m.cell_tau()      # pinned against its definition in the energy identity

    def gauss(q):
        x, w = np.polynomial.legendre.leggauss(q)
        return 0.5 * (x + 1), 0.5 * w

    ref = 0.0
    for c in range(m.nc):
        h = F.hi[c] - F.lo[c]
        e = F.enr_index(c)
        nq = [n, qw if e >= 0 else n, n]
        (x0, w0), (x1, w1), (x2, w2) = gauss(nq[0]), gauss(nq[1]), gauss(nq[2])
        nut = m.nut_cell(uf, e).reshape(nq[2], nq[1], nq[0]) if e >= 0 else None
        for i2 in range(nq[2]):
            for i1 in range(nq[1]):
                for i0 in range(nq[0]):
                    xi = (x0[i0], x1[i1], x2[i2])
                    dV = np.prod(h) * w0[i0] * w1[i1] * w2[i2]
                    _, gb, _, gt = F.eval(u, c, xi)
                    _, gvb, _, gvt = F.eval(v, c, xi)
                    ref += dV * 2 * nu * np.sum(_eps(gvb) * _eps(gb))
                    if e >= 0:
                        nt = _nut_point(F, uf, c, xi)
                        assert abs(nt - nut[i2, i1, i0]) <= 1e-12 * max(nt, 1e-300) + 1e-300
                        nuh = min(nu + nt, 2 * math.sqrt(nu * (nu + nt)))
                        ref += dV * 2 * nuh * np.sum(_eps(gvb) * _eps(gt))
                        ref += dV * 2 * (nu + nt) * np.sum(_eps(gvt) * _eps(gt))
    # faces, each from both sides (the test function lives on the side it is evaluated from)
    face = 0.0
    arith = 0.0      # change of the enriched-face terms with the arithmetic mean of kappa
    for c in range(m.nc):
        i, j, kz = c % nx, (c // nx) % ny, c // (nx * ny)
        h = F.hi[c] - F.lo[c]
        enr_c = F.enr_index(c) >= 0
        for d in range(3):
            t1 = 1 if d == 0 else 0
            t2 = 1 if d == 2 else 2
            for side in (0, 1):
                step = 1 if side else -1
                if d == 0:
                    nb = (i + step) % nx + nx * (j + ny * kz)
                elif d == 2:
                    nb = i + nx * (j + ny * ((kz + step) % nz))
                else:
                    nb = i + nx * (j + step + ny * kz) if 0 <= j + step < ny else None
                enr_o = enr_c if nb is None else F.enr_index(nb) >= 0
                both, iface = enr_c and enr_o, enr_c != enr_o
                tf = 10 * tau[c] if nb is None else max(tau[c], tau[nb])
                nvec = np.zeros(3)
                nvec[d] = 1.0 if side else -1.0
                q1 = qw if (t1 == 1 and (enr_c or enr_o)) else n
                q2 = qw if (t2 == 1 and (enr_c or enr_o)) else n
                (a1, b1), (a2, b2) = gauss(q1), gauss(q2)
                for p2 in range(q2):
                    for p1 in range(q1):
                        xi = [0.0, 0.0, 0.0]
                        xi[d] = float(side)
                        xi[t1], xi[t2] = a1[p1], a2[p2]
                        dA = h[t1] * h[t2] * b1[p1] * b2[p2]
                        ub, gb, ut, gt = F.eval(u, c, xi)
                        vb, gvb, vt, gvt = F.eval(v, c, xi)
                        ks = nu + _nut_point(F, uf, c, xi)
                        if nb is None:        # mirror state: u+ = -u-, grad u+ = grad u-, nu_t+ = nu_t-
                            ubo, gbo, uto, gto, ko = -ub, gb, -ut, gt, ks
                        else:
                            xo = list(xi)
                            xo[d] = 1.0 - side
                            ubo, gbo, uto, gto = F.eval(u, nb, xo)
                            ko = nu + _nut_point(F, uf, nb, xo)
                        jb, jt = ub - ubo, ut - uto
                        jtot = jb + jt
                        sb = nu * (_eps(gb) + _eps(gbo)) @ nvec             # {{2 nu eps(ubar)}} n
                        jadj = jb + (jt if iface else 0.0)
                        # standard test function: consistency, adjoint, penalty
                        t = vb @ (-sb + tf * nu * jtot)
                        t += 0.5 * nu * (jadj @ gvb @ nvec + nvec @ gvb @ jadj)
                        # enriched test function
                        t += vt @ (tf * nu * jtot) - (vt @ sb if iface else 0.0)
                        if both:
                            # enriched flux with the harmonic mean H of kappa (and, for the
                            # sensitivity check, with the arithmetic mean)
                            terms = []
                            for mean in (2 * ks * ko / (ks + ko), 0.5 * (ks + ko)):
                                st = 0.5 * mean * (2 * _eps(gt) + 2 * _eps(gto)) @ nvec
                                terms.append(-(vb + vt) @ st
                                             + 0.5 * mean * (jtot @ gvt @ nvec + nvec @ gvt @ jtot))
                            t += terms[0]
                            arith += dA * (terms[1] - terms[0])
                        face += dA * t
    ref += face
    assert abs(val - ref) < 1e-12 * abs(ref), (val, ref)
    # the weights matter: the arithmetic mean of kappa moves the value far beyond the tolerance
    assert abs(arith) > 1e-6 * abs(ref), (arith, ref)


# ---------------------------------------------------------------------------------------------
# Enrichment and eddy viscosity (Sec. 3, Sec. 2.2)
# ---------------------------------------------------------------------------------------------

def test_enrichment_reproduces_wall_law_profile():
    """ubar = 0 and u~_B = u_tau e_x: the field in every wall cell is u_tau psi(y+) e_x with
    y+ = (distance to the wall) u_tau / nu (Sec. 3.1, eq. enrichment)."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = w.u_tau
    X = m.node_coords().reshape(m.nc, -1, 3)
    for c in [0, 5, 63, 7 * 8 + 3, 8 * 8 * 3 + 8 * 7 + 2]:
        ys = X[c, :, 1]
        for xi in ([0.1, 0.0, 0.7], [0.5, 0.37, 0.2], [0.9, 0.99, 0.4]):
            r = m.eval_point(u, c, xi)
            yphys = ys.min() + xi[1] * (ys.max() - ys.min())
            yp = (1.0 - abs(yphys)) * w.u_tau / w.nu
            assert abs(r["yplus"] - yp) < 1e-10 * max(yp, 1)
            assert abs(r["u"][0] - w.u_tau * O.psi_spalding(yp)[0]) < 1e-14
            assert abs(r["psi"] - O.psi_spalding(yp)[0]) < 1e-11 * max(1.0, abs(r["psi"]))
            assert abs(r["u"][1]) < 1e-300 and abs(r["u"][2]) < 1e-300


def test_eddy_viscosity_log_layer_limit():
    """Mixing length with the enriched log-law profile: in the log layer (y+ ~ 2000, damping ~ 1,
    y << C_DES h) nu_t -> kappa u_tau y, the textbook Prandtl result."""
    m = O.Mesh(1, 2, 1, 1, gamma=1e-3, nu=1e-5, tau_w=1.0, n_layers=1)
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = 1.0
    nut = m.nut_cell(u, 0)            # points x fastest, then 8 wall-normal, then z
    gy, _ = O.gauss(8)
    nq = 2
    y0 = gy[0] * 1.0                   # bottom cell spans [-1, 0] (gamma -> 0 is uniform)
    v = nut.reshape(nq, 8, nq)[0, 0, 0]
    assert abs(v / (0.41 * y0) - 1.0) < 0.05
    assert np.all(nut >= 0)


def test_eddy_viscosity_des_limiter_and_wall_branches():
    """y_DES = (y^-6 + (C_DES h)^-6)^(-1/6) (eq. ydes, h = wall-normal cell width / (k+1)) tends
    to C_DES h far from the wall (y >> C_DES h: the mixing length saturates at the grid scale) and
    to y near it. With the enriched log-law field u~ = u_tau psi(y+) e_x the strain is closed-form,
    sqrt(2 eps:eps) = u_tau^2 psi'(y+) / nu, so nu_t = (kappa y_DES (1 - exp(-y+/26)))^2 u_tau^2
    psi' / nu (eq. mix, lmix) must approach both limits at the points of the wall cell."""
    k, nu, tau_w = 4, 1e-5, 1.0
    m = O.Mesh(1, 2, 1, k, gamma=1e-3, nu=nu, tau_w=tau_w, n_layers=1)
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = 1.0     # u_tau = 1
    nut = m.nut_cell(u, 0).reshape(k + 1, 8, k + 1)[0, :, 0]   # along the wall normal
    gy, _ = O.gauss(8)
    X = m.node_coords().reshape(m.nc, -1, 3)
    dy = X[0, :, 1].max() - X[0, :, 1].min()
    ch = 0.85 * dy / (k + 1)
    far = near = 0
    for y, v in zip(gy * dy, nut):
        yp = y * math.sqrt(tau_w) / nu
        psi, dpsi = O.psi_spalding(yp)
        core = (0.41 * (1 - math.exp(-yp / 26.0))) ** 2 * dpsi / nu
        if y >= 4 * ch:
            assert abs(v / (core * ch ** 2) - 1) < 2e-4, (y, v)      # (1/4)^6 / 3 away from the limit
            far += 1
        if y <= 0.25 * ch:
            assert abs(v / (core * y ** 2) - 1) < 2e-4, (y, v)
            near += 1
    assert far >= 2 and near >= 1


def test_oracle_operators_overwrite_their_output():
    """Every operator writes its whole output: called on a buffer full of garbage it returns what it
    returns on a zeroed buffer (the Python wrappers always pass zeros, so this is checked through
    the C entry points directly)."""
    import ctypes
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(2, 3, 2, 2, lx=w.lx, lz=w.lz, nu=w.nu, tau_w=w.tau_w)
    p = I.uniform(11, m.n_p, -1, 1)
    u = I.uniform(12, m.n_u, -1, 1)
    tau_d = I.uniform(13, m.nc, 0.5, 1.0)
    ptr = O._ptr
    calls = {
        "laplace": (m.n_p, lambda y: m.lib.dgo_laplace(m.h, ptr(p), ptr(y))),
        "laplace_diag": (m.n_p, lambda y: m.lib.dgo_laplace_diag(m.h, ptr(y))),
        "mass": (m.n_p, lambda y: m.lib.dgo_mass(m.h, ptr(p), ptr(y))),
        "divergence": (m.n_p, lambda y: m.lib.dgo_divergence(m.h, ptr(u), ptr(y))),
        "convective": (m.n_u, lambda y: m.lib.dgo_convective(m.h, ptr(u), ptr(y))),
        "viscous": (m.n_u, lambda y: m.lib.dgo_viscous(m.h, ptr(u), ptr(u), ptr(y))),
        "vmass": (m.n_u, lambda y: m.lib.dgo_vmass(m.h, ptr(u), ptr(y))),
        "gradient": (m.n_u, lambda y: m.lib.dgo_gradient(m.h, ptr(p), ptr(y))),
        "curl": (m.n_u, lambda y: m.lib.dgo_curl(m.h, ptr(u), ptr(y))),
        "divdiv": (m.n_u, lambda y: m.lib.dgo_divdiv(m.h, ptr(tau_d), ptr(u), ptr(y))),
        "inverse_mass": (m.n_u, lambda y: m.lib.dgo_inverse_mass(m.h, ptr(u), ptr(y))),
    }
    for name, (size, call) in calls.items():
        clean = np.zeros(size)
        call(clean)
        dirty = np.full(size, 1e30)
        call(dirty)
        assert np.array_equal(clean, dirty), name
        assert np.abs(clean).max() > 0.0, name


def test_active_cell_mask_restricts_outputs_to_those_cells():
    """The sampling mask (used for sampled full-size parity and the CPU baseline) computes the outputs
    of the masked cells exactly as the whole operator does and leaves the other cells' outputs zero;
    clearing the mask restores the whole operator."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(3, 4, 2, 2, lx=w.lx, lz=w.lz, nu=w.nu, tau_w=w.tau_w)
    u = I.uniform(41, m.n_u, -1, 1)
    p = I.uniform(42, m.n_p, -1, 1)
    full = {"laplace": m.laplace(p), "divergence": m.divergence(u), "convective": m.convective(u),
            "viscous": m.viscous(u, u)}
    cells = [0, 5, 13, 23]
    m.set_active(cells)
    mask = np.zeros(m.nc, dtype=bool)
    mask[cells] = True
    n3 = (2 + 1) ** 3
    part = {"laplace": m.laplace(p), "divergence": m.divergence(u), "convective": m.convective(u),
            "viscous": m.viscous(u, u)}
    m.set_active(None)
    for name in full:
        a, b = full[name], part[name]
        std_n = m.n_p if name in ("laplace", "divergence") else 3 * m.n_p
        per = 1 if name in ("laplace", "divergence") else 3
        sa = a[:std_n].reshape(m.nc, per * n3)
        sb = b[:std_n].reshape(m.nc, per * n3)
        assert np.array_equal(sa[mask], sb[mask]), name
        assert np.abs(sb[~mask]).max() == 0.0, name
    assert np.array_equal(m.convective(u), full["convective"])


def test_oracle_solve_reaches_tolerance_zero_mean():
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(3, 4, 3, 2, n_layers=0, nu=w.nu)
    b = I.pressure_rhs(m.n_p, 7)
    p, it, rr = m.solve(b, rtol=1e-12)
    assert rr <= 1e-12 and abs(p.mean()) < 1e-14 and it > 0


# ---------------------------------------------------------------------------------------------
# Constant enrichment weights, l = 0 (Sec. 3.1 with N^0 = 1; the setting of every simulation of
# Sec. 5 except the one comparison of Sec. 5.1): one coefficient per component and wall cell
# ---------------------------------------------------------------------------------------------

def _l0_mesh(w, **kw):
    return O.Mesh(**w.mesh_kwargs(), enrich_l=0, **kw)


def test_l0_layout_has_one_coefficient_per_component():
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m0, m1 = _l0_mesh(w), O.Mesh(**w.mesh_kwargs())
    assert m0.n_e == m1.n_e > 0 and m0.n_p == m1.n_p
    assert m0.n_u == 3 * m0.n_p + 3 * m0.n_e and m1.n_u == 3 * m1.n_p + 24 * m1.n_e


def test_l0_enrichment_reproduces_wall_law_profile():
    """ubar = 0 and u~ = u_tau e_x: the field in every wall cell is u_tau psi(y+) e_x (eq. enrichment
    with a constant weight)."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = _l0_mesh(w)
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3)[:, 0] = w.u_tau
    X = m.node_coords().reshape(m.nc, -1, 3)
    for c in [0, 5, 63, 8 * 8 * 3 + 8 * 7 + 2]:
        ys = X[c, :, 1]
        for xi in ([0.1, 0.0, 0.7], [0.5, 0.37, 0.2], [0.9, 0.99, 0.4]):
            r = m.eval_point(u, c, xi)
            yphys = ys.min() + xi[1] * (ys.max() - ys.min())
            yp = (1.0 - abs(yphys)) * w.u_tau / w.nu
            assert abs(r["u"][0] - w.u_tau * O.psi_spalding(yp)[0]) < 1e-14
            assert abs(r["u"][1]) < 1e-300 and abs(r["u"][2]) < 1e-300


def test_l0_mass_and_divergence_integrate_psi():
    """u~ = e_x (then e_y), ubar = 0: the enriched mass output of component x is int psi^2 over the
    wall cells, the standard outputs sum to int psi, and with q = y the divergence gives int psi
    (face terms vanish or cancel as for l = 1) - all against adaptive quadrature of Spalding's law."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = _l0_mesh(w)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    area = 2 * (2 * math.pi * math.pi)

    def integral(f):
        return area * quad(lambda s: f(O.psi_spalding(s * w.u_tau / w.nu)[0]), 0.0, dy,
                           epsabs=1e-14, epsrel=1e-13, limit=200)[0]

    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3)[:, 0] = 1.0
    y = m.vmass(u)
    std = y[: 3 * m.n_p].reshape(m.nc, 3, -1)
    ye = y[3 * m.n_p:].reshape(m.n_e, 3)
    assert abs(std[:, 0, :].sum() / integral(lambda p: p) - 1.0) < 1e-6
    assert abs(ye[:, 0].sum() / integral(lambda p: p * p) - 1.0) < 1e-6
    assert np.abs(ye[:, 1:]).max() == 0.0
    u[:] = 0.0
    u[3 * m.n_p:].reshape(m.n_e, 3)[:, 1] = 1.0
    val = m.node_coords()[:, 1] @ m.divergence(u)
    assert abs(val / integral(lambda p: p) - 1.0) < 1e-6


@pytest.mark.parametrize("comp", [0, 2])
def test_l0_convective_vanishes_for_shear_flow(comp):
    """The shear-flow invariant of the convective term (div(u x u) = 0, u.n = 0 on y-faces) with the
    constant-weight enrichment."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = _l0_mesh(w)
    f = [lambda x, y, z: 0 * y] * 3
    f[comp] = lambda x, y, z: 1 - y ** 2
    u = _std_field(m, *f)
    u[3 * m.n_p:].reshape(m.n_e, 3)[:, comp] = w.u_tau
    assert np.abs(m.convective(u)).max() < 1e-14


def test_l0_viscous_symmetric_part_psd_and_mass_spd():
    """Brute-force assembly on a tiny enriched mesh with l = 0: the symmetric part of -F^nu is
    positive semi-definite (clipped viscosity active) and the mass matrix is SPD."""
    nu = 1e-4
    m = O.Mesh(2, 3, 2, 2, n_layers=1, nu=nu, tau_w=1e-2, gamma=1.8, enrich_l=0)
    uf = np.zeros(m.n_u)
    uf[3 * m.n_p:].reshape(m.n_e, 3)[:, 0] = 0.1
    uf[3 * m.n_p:] += 0.02 * I.uniform(6, m.n_e * 3, -1, 1)
    E = np.eye(m.n_u)
    A = np.column_stack([m.viscous(uf, e) for e in E])
    S = 0.5 * (A + A.T)
    ev = np.linalg.eigvalsh(S)
    assert ev[0] >= -1e-11 * ev[-1]
    assert max(m.nut_cell(uf, e).max() for e in range(m.n_e)) > 3 * nu
    Mm = np.column_stack([m.vmass(e) for e in E])
    assert np.abs(Mm - Mm.T).max() < 1e-14 * np.abs(Mm).max()
    assert np.linalg.eigvalsh(Mm).min() > 0.0


@pytest.mark.parametrize("geometry", [0, 1])
def test_l0_equals_l1_with_equal_weights(geometry):
    """sum_B N_B = 1: an l = 1 field whose 8 weights of a component are equal is the l = 0 field with
    that coefficient, and the l = 0 test function psi e_a is the sum of the 8 l = 1 test functions.
    So every operator (and nu_t) of l = 0 equals the l = 1 operator with replicated inputs and
    summed enriched outputs - the oracle's two basis branches checked against each other."""
    if geometry:
        w = I.bump_workload("b0", 6, 4, 2, 2, seed=23)
    else:
        w = I.Workload("l0", 3, 4, 2, 3, 395.0, 1.0 / 6000.0, seed=24)
    m0, m1 = _l0_mesh(w), O.Mesh(**w.mesh_kwargs())
    ne, np3 = m0.n_e, 3 * m0.n_p
    u0 = I.workload_velocity(m0.node_coords(), ne, w, nef=1)
    u0[np3:] += 0.1 * w.u_tau * I.uniform(w.seed, 3 * ne, -1, 1, stream=51)
    u1 = np.concatenate([u0[:np3], np.repeat(u0[np3:], 8)])
    r = I.uniform(w.seed, m0.n_u, -1, 1, stream=52)
    r1 = np.concatenate([r[:np3], np.repeat(r[np3:], 8)])

    def fold(y1):
        return np.concatenate([y1[:np3], y1[np3:].reshape(-1, 8).sum(axis=1)])

    pairs = [(m0.vmass(r), fold(m1.vmass(r1))), (m0.convective(u0), fold(m1.convective(u1))),
             (m0.viscous(u0, r), fold(m1.viscous(u1, r1)))]
    for y0, y1 in pairs:
        assert np.abs(y0 - y1).max() <= 1e-13 * np.abs(y1).max()
    d0, d1 = m0.divergence(u0), m1.divergence(u1)
    assert np.abs(d0 - d1).max() <= 1e-13 * np.abs(d1).max()
    for e in range(0, ne, max(ne // 4, 1)):
        n0, n1 = m0.nut_cell(u0, e), m1.nut_cell(u1, e)
        assert np.abs(n0 - n1).max() <= 1e-13 * max(np.abs(n1).max(), 1e-300)


# ---------------------------------------------------------------------------------------------
# Wall shear stress on the linear wall nodes (Sec. 3.2): tau_w,B = |int N_B tau_w dA| / int N_B dA
# ---------------------------------------------------------------------------------------------

def test_wall_shear_of_parabolic_profile_is_exact():
    """u = (1 - y^2) e_x (no enrichment): nu |du/dy| = 2 nu on both walls, so every node gets 2 nu
    (a polynomial the Q_k space and the face rule hold exactly)."""
    nu = 1e-3
    m = O.Mesh(5, 4, 3, 2, n_layers=0, nu=nu)
    assert m.n_wall_nodes == 2 * 5 * 3
    u = _std_field(m, lambda x, y, z: 1 - y ** 2, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    tn = m.wall_shear(u)
    assert np.abs(tn / (2 * nu) - 1.0).max() < 1e-12


@pytest.mark.parametrize("enrich_l", [1, 0])
def test_wall_shear_reproduces_the_enrichment_tau(enrich_l):
    """ubar = 0, u~ = u_tau e_x with the prescribed tau_w = u_tau^2: at the wall psi = 0, psi'(0) = 1
    and dy+/dy = u_tau / nu, so nu du/dy = u_tau^2 = tau_w at every wall point and node."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs(), enrich_l=enrich_l)
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3, -1)[:, 0, :] = w.u_tau
    tn = m.wall_shear(u)
    assert np.abs(tn / w.tau_w - 1.0).max() < 1e-12


def test_wall_shear_weights_nodes_with_the_hat_functions():
    """u = (1 - y^2)(1 + a sin(2 pi x / L_x)) e_x: the traction 2 nu (1 + a sin) integrated against the
    periodic hat of node x_i on a uniform grid of spacing h gives
    2 nu (1 + a sin(kappa x_i) * 2 (1 - cos kappa h) / (kappa h)^2); the discrete field is the
    degree-5 interpolant of the sine, hence the tolerance."""
    nu, a, nx = 1e-3, 0.5, 16
    m = O.Mesh(nx, 2, 2, 5, n_layers=0, nu=nu)
    lx = 2 * math.pi
    kap = 2 * math.pi / lx
    u = _std_field(m, lambda x, y, z: (1 - y ** 2) * (1 + a * np.sin(kap * x)), lambda x, y, z: 0 * y,
                   lambda x, y, z: 0 * y)
    tn = m.wall_shear(u).reshape(2, 2, nx)            # [wall][k][i]
    h = lx / nx
    xi = np.arange(nx) * h
    ref = 2 * nu * (1 + a * np.sin(kap * xi) * 2 * (1 - math.cos(kap * h)) / (kap * h) ** 2)
    for wall in range(2):
        for kz in range(2):
            assert np.abs(tn[wall, kz] / ref - 1.0).max() < 1e-6


def test_wall_shear_is_the_magnitude_of_the_hat_weighted_traction_vector():
    """u = (1 - y^2) ((1 + a sin(2 pi z / L_z)) e_x + c e_y + b e_z): the wall traction nu du/dn is a
    vector with three components, varying along z. Each node gets the magnitude of its hat-weighted
    mean traction, 2 nu sqrt((1 + a s sin(kappa z_k))^2 + c^2 + b^2) with s = 2 (1 - cos kappa h) /
    (kappa h)^2 the hat's factor for the sine (uniform spacing h along z)."""
    nu, a, b, c, nz = 1e-3, 0.5, 0.7, 0.4, 16
    m = O.Mesh(2, 2, nz, 5, n_layers=0, nu=nu)
    lz = math.pi
    kap = 2 * math.pi / lz
    u = _std_field(m, lambda x, y, z: (1 - y ** 2) * (1 + a * np.sin(kap * z)), lambda x, y, z: (1 - y ** 2) * c,
                   lambda x, y, z: (1 - y ** 2) * b + 0 * x)
    tn = m.wall_shear(u).reshape(2, nz, 2)            # [wall][k][i]
    h = lz / nz
    s = 2 * (1 - math.cos(kap * h)) / (kap * h) ** 2
    zk = np.arange(nz) * h
    ref = 2 * nu * np.sqrt((1 + a * s * np.sin(kap * zk)) ** 2 + c ** 2 + b ** 2)
    for wall in range(2):
        for i in range(2):
            assert np.abs(tn[wall, :, i] / ref - 1.0).max() < 1e-6


def test_set_tau_nodes_interpolates_bilinearly_along_the_wall():
    """Nodal tau_w: y+ at a point of a wall cell is y_h sqrt(tau_h) / nu with tau_h the bilinear
    interpolant of the four wall nodes below it (off-wall vertices carry the value of the wall node
    that defines their wall distance, the node of the same column on the channel)."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    tn = w.tau_w * (1.0 + 0.5 * I.uniform(3, m.n_wall_nodes, -1.0, 1.0))
    m.set_tau_nodes(tn)
    u = np.zeros(m.n_u)
    nx, nz = 8, 8
    X = m.node_coords().reshape(m.nc, -1, 3)
    for (i, j, kz) in [(0, 0, 0), (7, 0, 7), (3, 7, 5), (6, 7, 0)]:
        c = i + nx * (j + 8 * kz)
        wall = 0 if j == 0 else 1
        T = tn.reshape(2, nz, nx)[wall]
        ys = X[c, :, 1]
        for xi in ([0.2, 0.3, 0.7], [0.9, 0.05, 0.4]):
            r = m.eval_point(u, c, xi)
            th = ((1 - xi[0]) * (1 - xi[2]) * T[kz, i] + xi[0] * (1 - xi[2]) * T[kz, (i + 1) % nx]
                  + (1 - xi[0]) * xi[2] * T[(kz + 1) % nz, i] + xi[0] * xi[2] * T[(kz + 1) % nz, (i + 1) % nx])
            yphys = ys.min() + xi[1] * (ys.max() - ys.min())
            yp = (1.0 - abs(yphys)) * math.sqrt(th) / w.nu
            assert abs(r["yplus"] / yp - 1.0) < 1e-12


def test_enrichment_gradient_is_the_derivative_of_the_enrichment():
    """With a nodal tau_w varying along the wall, grad u~ = sum_B u~_B (psi grad N_B + N_B psi' grad y+)
    and grad y+ = (sqrt(tau_h) grad y_h + y_h grad tau_h / (2 sqrt(tau_h))) / nu must be the derivative
    of the field u~ itself: nu_t = l_mix^2 sqrt(2 eps(u~):eps(u~)) (eq. mix, lmix, ydes) evaluated with
    central differences of u~ (and y+ from the point evaluation, pinned above) matches the oracle's
    nu_t at points of wall cells on both walls."""
    nx, ny, nz, k = 4, 4, 4, 2
    nu, tau_w = 1e-3, 1e-2
    m = O.Mesh(nx, ny, nz, k, nu=nu, tau_w=tau_w, n_layers=1)
    m.set_tau_nodes(tau_w * (1.0 + 0.5 * I.uniform(14, m.n_wall_nodes, -1.0, 1.0)))
    u = np.zeros(m.n_u)
    u[3 * m.n_p:] = I.uniform(15, 24 * m.n_e, -1.0, 1.0)
    X = m.node_coords().reshape(m.nc, -1, 3)
    dlt = 1e-5
    for c in [0, 1 + nx * ny * 2, 2 + nx * (ny - 1) + nx * ny * 3, 1 + nx * (ny - 1)]:   # both walls
        lo, hi = X[c].min(axis=0), X[c].max(axis=0)
        h = hi - lo
        for xi in ([0.3, 0.4, 0.6], [0.8, 0.15, 0.25], [0.55, 0.9, 0.7]):
            G = np.zeros((3, 3))
            for d in range(3):
                a, b = list(xi), list(xi)
                a[d] += dlt
                b[d] -= dlt
                G[:, d] = (m.eval_point(u, c, a)["util"] - m.eval_point(u, c, b)["util"]) / (2 * dlt * h[d])
            E = 0.5 * (G + G.T)
            r = m.eval_point(u, c, xi)
            y = lo[1] + xi[1] * h[1]
            yh = 1.0 - abs(y)
            ydes = (yh ** -6 + (0.85 * h[1] / (k + 1)) ** -6) ** (-1.0 / 6.0)
            lmix = 0.41 * ydes * (1.0 - math.exp(-r["yplus"] / 26.0))
            ref = lmix ** 2 * math.sqrt(2.0 * np.sum(E * E))
            assert abs(r["nut"] / ref - 1.0) < 1e-7, (c, xi, r["nut"], ref)


def test_wall_distance_and_nodal_tau_on_the_bump():
    """On the bump every vertex of an enriched cell takes the distance to, and the tau_w of, the
    closest wall vertex of either wall (periodic copies included), found here by brute force over the
    node coordinates; y+ at a point is y_h sqrt(tau_h) / nu with y_h and tau_h the trilinear
    interpolants of those vertex values (Sec. 3.2)."""
    nx, ny, nz, k = 12, 4, 2, 2
    nu, tau_w = 1e-3, 2e-2
    m = O.Mesh(nx, ny, nz, k, lx=9.0, ly=3.036, lz=4.5, geometry=1, n_layers=1, nu=nu, tau_w=tau_w)
    tn = tau_w * (1.0 + 0.5 * I.uniform(4, m.n_wall_nodes, -1.0, 1.0))
    m.set_tau_nodes(tn)
    n = k + 1
    X = m.node_coords().reshape(nz, ny, nx, n, n, n, 3)          # [kz][j][i][c][b][a]
    # wall vertices (wi, wk) = 0..nx, 0..nz with their node index wall * nx * nz + wi % nx + nx * (wk % nz)
    wall_pts, wall_idx = [], []
    for wall, (j, b) in enumerate(((0, 0), (ny - 1, n - 1))):
        for wk in range(nz + 1):
            for wi in range(nx + 1):
                p = X[min(wk, nz - 1), j, min(wi, nx - 1), (n - 1) if wk == nz else 0, b,
                      (n - 1) if wi == nx else 0].copy()
                wall_pts.append(p)
                wall_idx.append(wall * nx * nz + wi % nx + nx * (wk % nz))
    wall_pts, wall_idx = np.array(wall_pts), np.array(wall_idx)
    u = np.zeros(m.n_u)
    checked = 0
    for (i, j, kz) in [(0, 0, 0), (4, 0, 1), (5, 0, 0), (6, 0, 1), (7, 0, 0), (11, 0, 1), (5, ny - 1, 0)]:
        c = i + nx * (j + ny * kz)
        d = np.zeros(8)
        t = np.zeros(8)
        for v in range(8):
            vx, vy, vz = v & 1, (v >> 1) & 1, v >> 2
            p = X[kz, j, i, (n - 1) * vz, (n - 1) * vy, (n - 1) * vx]
            dist = np.linalg.norm(wall_pts - p, axis=1)
            q = int(np.argmin(dist))
            d[v], t[v] = dist[q], tn[wall_idx[q]]
        for xi in ([0.2, 0.3, 0.7], [0.9, 0.05, 0.4], [0.5, 0.8, 0.1]):
            N = np.array([(xi[0] if v & 1 else 1 - xi[0]) * (xi[1] if (v >> 1) & 1 else 1 - xi[1])
                          * (xi[2] if v >> 2 else 1 - xi[2]) for v in range(8)])
            yp = (N @ d) * math.sqrt(N @ t) / nu
            r = m.eval_point(u, c, xi)
            assert abs(r["yplus"] / yp - 1.0) < 1e-12, (i, j, kz, xi, r["yplus"], yp)
            checked += 1
    assert checked == 21


# ---------------------------------------------------------------------------------------------
# Cell-wise L2 projection onto the space of a new wall shear stress (Sec. 3.2, eq. l2). The cell
# systems are ill-conditioned (psi N_B is close to the polynomials where the cell spans few wall
# units), so the pins compare functions in the L2 norm, not coefficients.
# ---------------------------------------------------------------------------------------------

def _l2_rel(m, a, b):
    d = a - b
    return math.sqrt(abs(d @ m.vmass(d)) / (b @ m.vmass(b)))


def test_projection_onto_the_same_space_is_the_identity():
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    u = I.workload_velocity(m.node_coords(), m.n_e, w)
    u[3 * m.n_p:] += 0.2 * w.u_tau * I.uniform(4, 24 * m.n_e, -1, 1)
    un = m.project(np.full(m.n_wall_nodes, w.tau_w), u)
    assert _l2_rel(m, un, u) < 1e-12
    nw = [c for c in range(m.nc) if (c // 8) % 8 not in (0, 7)]     # cells off the wall: copied
    std = lambda v: v[: 3 * m.n_p].reshape(m.nc, -1)[nw]
    assert np.array_equal(std(un), std(u))


@pytest.mark.parametrize("geometry", [0, 1])
def test_projection_keeps_a_polynomial_field(geometry):
    """A standard Q_k field (no enrichment part) lies in every enriched space: projecting it onto the
    space of a varying nodal tau_w leaves the function unchanged."""
    if geometry:
        w = I.bump_workload("bp", 6, 4, 2, 3, seed=31)
    else:
        w = I.Workload("pp", 4, 4, 2, 3, 395.0, 1.0 / 6000.0, seed=32)
    m = O.Mesh(**w.mesh_kwargs())
    u = _std_field(m, lambda x, y, z: 1 + y ** 3 - 0.5 * x * y, lambda x, y, z: y * z, lambda x, y, z: x ** 2)
    tn = w.tau_w * (1.0 + 0.6 * I.uniform(5, m.n_wall_nodes, -1, 1))
    un = m.project(tn, u)          # the mesh now holds tn, so vmass measures in the new space
    assert _l2_rel(m, un, u) < 1e-11


def test_projection_matches_the_integrals_of_the_old_wall_law():
    """u_old = psi_old(y+) e_x (ubar = 0, all weights 1) with tau_old, projected onto tau_new = 2 tau_old:
    the Galerkin conditions for v = 1 and v = psi_new give int u_new = int psi_old and
    int u_new psi_new = int psi_old psi_new over the wall cells, against adaptive quadrature."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = 1.0
    un = m.project(np.full(m.n_wall_nodes, 2.0 * w.tau_w), u)
    y = m.vmass(un)
    ut_old, ut_new = w.u_tau, math.sqrt(2.0) * w.u_tau
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    area = 2 * (2 * math.pi * math.pi)
    ps = lambda s, ut: O.psi_spalding(s * ut / w.nu)[0]
    r1 = area * quad(lambda s: ps(s, ut_old), 0.0, dy, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    r2 = area * quad(lambda s: ps(s, ut_old) * ps(s, ut_new), 0.0, dy, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    std = y[: 3 * m.n_p].reshape(m.nc, 3, -1)
    ye = y[3 * m.n_p:].reshape(m.n_e, 3, 8)
    assert abs(std[:, 0, :].sum() / r1 - 1.0) < 1e-6
    assert abs(ye[:, 0, :].sum() / r2 - 1.0) < 1e-6
    assert np.abs(un[: 3 * m.n_p].reshape(m.nc, 3, -1)[:, 1:, :]).max() == 0.0


@pytest.mark.parametrize("full_q", [False, True])
def test_projection_keeps_the_moments_against_every_standard_test_function(full_q):
    """Galerkin condition of eq. (l2) for the standard test functions, which both spaces share: for a
    random old field (standard and enriched coefficients varying in every direction) projected onto a
    random nodal tau_w, int phi_i u_new (new space) = int phi_i u_old (old space) for every standard
    phi_i, both integrals taken by the (separately pinned) velocity mass operator with the mesh holding
    the old and then the new tau_w. With the default point set the in-plane directions are collocated
    (k+1 points for k+1 functions), so only the q_w^3 rule exercises the in-plane weights."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(4, 4, 3, 2, lx=w.lx, lz=w.lz, nu=w.nu, tau_w=w.tau_w, full_quadrature=full_q)
    u = I.uniform(31, m.n_u, -1, 1)
    u[3 * m.n_p:] *= 0.3
    y_old = m.vmass(u)[: 3 * m.n_p]
    un = m.project(w.tau_w * (1.0 + 0.3 * I.uniform(32, m.n_wall_nodes, -1, 1)), u)
    y_new = m.vmass(un)[: 3 * m.n_p]
    assert np.abs(y_new - y_old).max() < 1e-9 * np.abs(y_old).max()
    assert np.abs(un - u).max() > 1e-3                  # the space did change


# ---------------------------------------------------------------------------------------------
# Switch-off of the wall model where the wall-nearest cell lies below a y+ threshold (Sec. 3.2)
# ---------------------------------------------------------------------------------------------

def test_switched_off_mesh_equals_the_mesh_without_enrichment():
    """With every wall column switched off the operators on the standard DoFs are those of the same
    mesh built without enrichment, and the enrichment outputs are zero; switching back on restores
    the enriched operators exactly."""
    w = I.Workload("so", 4, 4, 2, 2, 180.0, 1.0 / 3250.0, seed=33)
    m, m0 = O.Mesh(**w.mesh_kwargs()), O.Mesh(**w.mesh_kwargs(), n_layers=0)
    u = I.workload_velocity(m.node_coords(), m.n_e, w)
    u[3 * m.n_p:] += 0.1 * I.uniform(7, 24 * m.n_e, -1, 1)
    np3 = 3 * m.n_p
    before = [m.convective(u), m.viscous(u, u), m.vmass(u)]
    m.set_switch(1e30)
    assert m.active().sum() == 0
    for f, f0 in ((m.convective, m0.convective), (m.vmass, m0.vmass)):
        y, y0 = f(u), f0(u[:np3])
        assert np.array_equal(y[:np3], y0) and not np.any(y[np3:])
    y, y0 = m.viscous(u, u), m0.viscous(u[:np3], u[:np3])
    assert np.array_equal(y[:np3], y0) and not np.any(y[np3:])
    assert np.array_equal(m.divergence(u), m0.divergence(u[:np3]))
    m.set_switch(0.0)
    assert m.active().sum() == m.n_e
    for y, f in zip(before, (m.convective, lambda v: m.viscous(v, v), m.vmass)):
        assert np.array_equal(f(u), y)


def test_switch_off_criterion_on_the_channel():
    """Channel: y_h = xi_1 dy in a bottom wall cell, tau_h is bilinear in (xi_0, xi_2) and constant in
    xi_1, so the largest y+ over the points is at the largest wall-normal Gauss point and the largest
    in-plane value of tau_h; a column is on iff that maximum reaches the threshold."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    nx, nz = 8, 8
    tn = w.tau_w * 10.0 ** I.uniform(8, m.n_wall_nodes, -1.0, 1.0)
    m.set_tau_nodes(tn)
    thr = 25.0
    m.set_switch(thr)
    gx, _ = O.gauss(3)
    gq, _ = O.gauss(8)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    on = m.active()
    T = tn.reshape(2, nz, nx)
    for e in range(m.n_e):
        wall, r = divmod(e, nx * nz)
        kz, i = divmod(r, nx)
        t4 = [T[wall, kz, i], T[wall, kz, (i + 1) % nx], T[wall, (kz + 1) % nz, i], T[wall, (kz + 1) % nz, (i + 1) % nx]]
        th = max((1 - a) * (1 - b) * t4[0] + a * (1 - b) * t4[1] + (1 - a) * b * t4[2] + a * b * t4[3]
                 for a in gx for b in gx)
        ymax = (gq[-1] if wall == 0 else 1.0 - gq[0]) * dy * math.sqrt(th) / w.nu
        assert on[e] == (ymax >= thr), (e, ymax)
    assert 0 < on.sum() < m.n_e


def test_projection_into_switched_off_cells_keeps_polynomials():
    """Projecting onto a space whose wall columns are partly switched off: a polynomial field is
    unchanged and the enrichment coefficients of the switched-off cells are zero."""
    w = I.Workload("sp", 4, 4, 2, 3, 395.0, 1.0 / 6000.0, seed=34)
    m = O.Mesh(**w.mesh_kwargs())
    m.set_switch(60.0)
    u = _std_field(m, lambda x, y, z: 1 + y ** 3 - 0.5 * x * y, lambda x, y, z: y * z, lambda x, y, z: x ** 2)
    tn = w.tau_w * 10.0 ** I.uniform(9, m.n_wall_nodes, -2.0, 0.3)
    un = m.project(tn, u)
    on = m.active()
    assert 0 < on.sum() < m.n_e
    assert _l2_rel(m, un, u) < 1e-11
    ue = un[3 * m.n_p:].reshape(m.n_e, -1)
    assert not np.any(ue[on == 0])


# ---------------------------------------------------------------------------------------------
# Projection-step operators (Sec. 4.2): pressure gradient P, div-div penalty D, and the inverse
# mass of the explicit convective step
# ---------------------------------------------------------------------------------------------

def test_gradient_of_continuous_pressure_is_the_volume_integral():
    """For continuous p the face terms and -(div v, p) integrate by parts to (v, grad p) (also on
    walls, where {{p}} = p^-): v . P(p) = int v . grad p; p = y^3/3 + y, v = (0, y^2, 0)."""
    m = O.Mesh(3, 4, 2, 3, n_layers=0)
    p = (lambda X: X[:, 1] ** 3 / 3 + X[:, 1])(m.node_coords())
    v = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: y ** 2, lambda x, y, z: 0 * y)
    ref = 2 * math.pi * math.pi * (2.0 / 5 + 2.0 / 3)
    assert abs(v @ m.gradient(p) / ref - 1.0) < 1e-12


def test_gradient_is_the_transpose_of_the_divergence_where_v_n_vanishes():
    """On interior faces P(v, p) = -C(p, v) term by term (same average); the volume terms agree by
    integration by parts, exact for polynomial fields with these rules; on walls they differ by
    (p, v.n). With v_y zero on the wall node layers v.n = 0 there, so v . P(p) = p . (-C v) for a
    discontinuous random p and a random standard v (enriched cells still use their point sets)."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    n1 = m.k + 1
    p = I.uniform(1, m.n_p, -1, 1)
    v = I.uniform(2, m.n_u, -1, 1)
    v[3 * m.n_p:] = 0.0
    std = v[: 3 * m.n_p].reshape(8, 8, 8, 3, n1, n1, n1)     # cz, cy, cx, comp, lz, ly, lx
    std[:, 0, :, 1, :, 0, :] = 0.0
    std[:, 7, :, 1, :, n1 - 1, :] = 0.0
    lhs, rhs = v @ m.gradient(p), p @ m.divergence(v)
    assert abs(lhs - rhs) < 1e-12 * (abs(v) @ np.abs(m.gradient(p)))


def test_gradient_enriched_test_functions_against_the_point_rule():
    """p = y (continuous): the enriched outputs of component y sum to
    -int d(psi)/dy y dV + (psi y n_y) on the face away from the wall (psi = 0 on the wall; the enriched
    test functions psi N_v e_y sum to psi e_y). The volume integral is the q_w-point Gauss rule of the
    wall-normal direction, written out here with NumPy's rule and the oracle's pinned psi, psi'."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    y = m.gradient(m.node_coords()[:, 1].copy())
    ye = y[3 * m.n_p:].reshape(m.n_e, 3, 8)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    s = w.u_tau / w.nu
    xq, wq = np.polynomial.legendre.leggauss(8)
    xq, wq = 0.5 * (xq + 1.0), 0.5 * wq
    vol = -sum(wi * dy * O.psi_spalding(xi * dy * s)[1] * s * (-1.0 + xi * dy) for xi, wi in zip(xq, wq))
    face = O.psi_spalding(dy * s)[0] * (-1.0 + dy)
    ref = 2 * (2 * math.pi * math.pi) * (vol + face)
    assert abs(ye[:, 1, :].sum() / ref - 1.0) < 1e-12


def test_divdiv_closed_form_null_space_and_tau():
    """D(u, u) = sum_K tau_K int (div u)^2 for u = (0, y^2, 0) with constant tau (= c int 4 y^2);
    D u = 0 for divergence-free shear flows with equal-weight enrichment; tau_D of a uniform flow U
    is U h dt / Cr with h the cube root of the cell volume."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    c = 0.37
    tau = np.full(m.nc, c)
    u = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: y ** 2, lambda x, y, z: 0 * y)
    ref = c * 2 * math.pi * math.pi * 8.0 / 3.0
    assert abs(u @ m.divdiv(tau, u) / ref - 1.0) < 1e-12
    s = _std_field(m, lambda x, y, z: 1 - y ** 2, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    s[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = w.u_tau
    assert np.abs(m.divdiv(tau, s)).max() < 1e-13
    U, dt, cr = 0.8, 1e-3, 0.14
    uu = _std_field(m, lambda x, y, z: U + 0 * y, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    X = m.node_coords().reshape(m.nc, -1, 3)
    vol = np.array([(np.ptp(X[k, :, 0])) * np.ptp(X[k, :, 1]) * np.ptp(X[k, :, 2]) for k in range(m.nc)])
    assert np.allclose(m.tau_divdiv(uu, dt, cr), U * np.cbrt(vol) * dt / cr, rtol=1e-12, atol=0)


def test_tau_divdiv_of_wall_cells_with_enrichment():
    """tau_D = (volume average of |u|) h dt / Cr (eq. tauD, h the cube root of the cell volume) in wall
    cells where u = (U, V, W) + psi(y+) (a, b, c): the average of
    sqrt((U + a psi)^2 + (V + b psi)^2 + (W + c psi)^2) over the cell is taken along y by the q_w = 8
    point Gauss rule (NumPy) the wall cells use; every component's sign enters."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    U, V, W = 0.3, -0.2, 0.1
    a, b, c = 0.05, 0.04, -0.03
    u = _std_field(m, lambda x, y, z: U + 0 * y, lambda x, y, z: V + 0 * y, lambda x, y, z: W + 0 * y)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:] = np.array([a, b, c])[None, :, None]
    dt, cr = 1e-3, 0.14
    tau = m.tau_divdiv(u, dt, cr)
    X = m.node_coords().reshape(m.nc, -1, 3)
    h = X[0].max(axis=0) - X[0].min(axis=0)                 # a bottom wall cell
    sc = w.u_tau / w.nu
    xg, wg = np.polynomial.legendre.leggauss(8)
    mean = 0.0
    for xq, wq in zip(xg, wg):
        ps = O.psi_spalding(0.5 * (xq + 1) * h[1] * sc)[0]
        mean += 0.5 * wq * math.sqrt((U + a * ps) ** 2 + (V + b * ps) ** 2 + (W + c * ps) ** 2)
    ref = mean * np.cbrt(np.prod(h)) * dt / cr
    assert abs(tau[0] / ref - 1.0) < 1e-12, (tau[0], ref)
    top = w.nx * (w.ny - 1)                                  # a top wall cell: the same by symmetry
    assert abs(tau[top] / ref - 1.0) < 1e-12


def test_divdiv_of_the_wall_normal_enrichment():
    """u = psi(y+) e_y from enrichment only (all weights 1): div u = psi'(y+) u_tau / nu, so
    u^T D u = tau int (div u)^2 over the wall cells = 2 tau L_x L_z (u_tau/nu)^2 int_0^dy psi'^2 ds
    (by the 8-point wall-normal Gauss rule to rounding, and by adaptive quadrature within the rule's
    error). For the x and z components the enriched test functions of a cell sum to psi e_x (psi e_z),
    whose divergence is zero, so their outputs sum to zero in every cell."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    c = 0.37
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 1, :] = 1.0
    y = m.divdiv(np.full(m.nc, c), u)
    sc = w.u_tau / w.nu
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    f = lambda s: O.psi_spalding(s * sc)[1] ** 2
    xg, wg = np.polynomial.legendre.leggauss(8)
    rule = 0.5 * dy * sum(wq * f(0.5 * dy * (xq + 1)) for xq, wq in zip(xg, wg))
    ref = 2 * c * w.lx * w.lz * sc ** 2 * rule
    val = u @ y
    assert abs(val / ref - 1.0) < 1e-12, (val, ref)
    exact = 2 * c * w.lx * w.lz * sc ** 2 * quad(f, 0.0, dy, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    assert abs(val / exact - 1.0) < 1e-4
    ye = y[3 * m.n_p:].reshape(m.n_e, 3, 8)
    big = np.abs(ye[:, 1, :]).max()
    for a in (0, 2):
        assert np.abs(ye[:, a, :].sum(axis=1)).max() < 1e-12 * big


@pytest.mark.parametrize("geometry", [0, 1])
def test_inverse_mass_inverts_the_mass_operator(geometry):
    """M^-1 (M u) = u for a velocity with enrichment, measured as functions (L2 norm): the wall-cell
    systems are ill-conditioned, so coefficients may move along nearly null directions."""
    if geometry:
        w = I.bump_workload("im", 5, 4, 2, 2, seed=36)
    else:
        w = I.Workload("im", 3, 4, 2, 3, 395.0, 1.0 / 6000.0, seed=37)
    m = O.Mesh(**w.mesh_kwargs())
    u = I.workload_velocity(m.node_coords(), m.n_e, w)
    u[3 * m.n_p:] += 0.2 * w.u_tau * I.uniform(w.seed, u.size - 3 * m.n_p, -1, 1)
    x = m.inverse_mass(m.vmass(u))
    assert _l2_rel(m, x, u) < 1e-10


# ---------------------------------------------------------------------------------------------
# Dual-splitting step (Sec. 4.1, eqs. convstepspat, poissonspat, projectionspat, helmholtzspat)
# ---------------------------------------------------------------------------------------------

def test_dual_splitting_keeps_poiseuille_flow_steady():
    """Laminar channel flow u = U (1 - y^2) e_x driven by f = 2 nu U e_x is a steady solution: the
    convective term vanishes for the shear flow, u^ = u + dt f / gamma_0 is divergence-free (p = 0),
    the div-div term vanishes, and -F^nu(u) = M f for the quadratic profile (Q2, exact quadrature).
    A wrong sign, a BDF coefficient that does not sum to gamma_0 or a dropped dt/gamma_0 breaks it."""
    nu, U = 1e-2, 1.0
    m = O.Mesh(4, 4, 2, 2, n_layers=0, nu=nu)
    u0 = _std_field(m, lambda x, y, z: U * (1 - y ** 2), lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    for hobc in (False, True):   # the high-order pressure data vanish too: g = f.n = 0 on the walls
        ds = O.DualSplitting(m, u0, dt=5e-3, force=(2 * nu * U, 0.0, 0.0), high_order_pressure_bc=hobc)
        for _ in range(3):
            u, p = ds.step()
        assert _l2_rel(m, u, u0) < 1e-11
        assert np.abs(p).max() < 1e-10


def test_cfl_rate_of_a_uniform_flow_is_the_thinnest_row_closed_form():
    """For a constant velocity (U, V, W) without enrichment on the boxes of the graded channel,
    |J^-1 u|_2 = sqrt((U/h_x)^2 + (V/h_y)^2 + (W/h_z)^2) at every point of a cell, so the rate is
    that of the thinnest row (cell sizes read from the node coordinates)."""
    m = O.Mesh(4, 6, 3, 2, n_layers=0)
    U, V, W = 1.0, 0.5, -0.25
    u = _std_field(m, lambda x, y, z: U + 0 * y, lambda x, y, z: V + 0 * y, lambda x, y, z: W + 0 * y)
    X = m.node_coords().reshape(m.nc, -1, 3)
    h = X.max(axis=1) - X.min(axis=1)
    ref = np.sqrt((U / h[:, 0]) ** 2 + (V / h[:, 1]) ** 2 + (W / h[:, 2]) ** 2).max()
    assert abs(m.cfl_rate(u) / ref - 1.0) < 1e-13
    assert abs(m.cfl_rate(-3.0 * u) / (3.0 * ref) - 1.0) < 1e-13


def test_cfl_rate_with_a_mean_flow_and_enrichment_in_every_component():
    """ubar = (U, V, W) everywhere plus u~ = psi(y+) (a, b, c) in the wall cells (all weights equal):
    the velocity at a wall-cell point is (U + a psi, V + b psi, W + c psi), so the rate is the largest of
    sqrt(((U + a psi_q)/h_x)^2 + ((V + b psi_q)/h_y)^2 + ((W + c psi_q)/h_z)^2) over the q_w wall-normal
    points and of the plain value in the other rows (a sign error in any component changes it)."""
    k, nu, tau_w = 2, 1e-3, 4e-2
    m = O.Mesh(2, 4, 2, k, nu=nu, tau_w=tau_w, n_layers=1)
    U, V, W = 0.3, -0.2, 0.1
    a, b, c = 0.05, 0.4, -0.3
    u = _std_field(m, lambda x, y, z: U + 0 * y, lambda x, y, z: V + 0 * y, lambda x, y, z: W + 0 * y)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:] = np.array([a, b, c])[None, :, None]
    X = m.node_coords().reshape(m.nc, -1, 3)
    h = X.max(axis=1) - X.min(axis=1)
    ut = math.sqrt(tau_w)
    gy, _ = O.gauss(8)
    rates = [np.sqrt((U / h[cc, 0]) ** 2 + (V / h[cc, 1]) ** 2 + (W / h[cc, 2]) ** 2) for cc in range(m.nc)]
    hw = h[0]                                            # wall rows: the same sizes at both walls
    for yq in gy:
        ps = O.psi_spalding(yq * hw[1] * ut / nu)[0]
        rates.append(math.sqrt(((U + a * ps) / hw[0]) ** 2 + ((V + b * ps) / hw[1]) ** 2 + ((W + c * ps) / hw[2]) ** 2))
    assert abs(m.cfl_rate(u) / max(rates) - 1.0) < 1e-12


def test_cfl_rate_on_curved_cells():
    """u = (U, V (1 + x / 9), W) on the bump: the rate is the largest |J^-1 u| over the linear point set,
    J^-1 and x rebuilt here from the node coordinates (Lagrange interpolation on the Gauss-Lobatto
    nodes). On the bump's slopes J^-1 is not diagonal; the x-dependent u_y breaks the mirror symmetry of
    the bump, so the sign of every off-diagonal term matters."""
    nx, ny, nz, k = 12, 3, 1, 2
    m = O.Mesh(nx, ny, nz, k, lx=9.0, ly=3.036, lz=4.5, geometry=1, n_layers=0)
    U, V, W = 1.0, 0.6, -0.3
    u = _std_field(m, lambda x, y, z: U + 0 * x, lambda x, y, z: V * (1 + x / 9.0), lambda x, y, z: W + 0 * x)
    n = k + 1
    X = m.node_coords().reshape(m.nc, n, n, n, 3)
    gl = O.lobatto(n)

    def lag(s):
        v, d = np.ones(n), np.zeros(n)
        for i in range(n):
            for j in range(n):
                if j != i:
                    v[i] *= (s - gl[j]) / (gl[i] - gl[j])
            for c in range(n):
                if c != i:
                    t = 1.0 / (gl[i] - gl[c])
                    for j in range(n):
                        if j != i and j != c:
                            t *= (s - gl[j]) / (gl[i] - gl[j])
                    d[i] += t
        return v, d

    gq, _ = O.gauss(n)
    best = 0.0
    for c in range(m.nc):
        for x2 in gq:
            for x1 in gq:
                for x0 in gq:
                    L = [lag(x0), lag(x1), lag(x2)]
                    J = np.array([[np.einsum("zyx,z,y,x", X[c, ..., e], L[2][dz], L[1][dy], L[0][dx])
                                   for (dx, dy, dz) in ((1, 0, 0), (0, 1, 0), (0, 0, 1))] for e in range(3)])
                    xp = np.einsum("zyx,z,y,x", X[c, ..., 0], L[2][0], L[1][0], L[0][0])
                    vel = np.array([U, V * (1 + xp / 9.0), W])
                    best = max(best, np.linalg.norm(np.linalg.solve(J, vel)))
    assert abs(m.cfl_rate(u) / best - 1.0) < 1e-12


def test_cfl_rate_includes_the_enrichment_at_the_wall_normal_points():
    """With ubar = 0 and u~_B = u_tau e_x the velocity is u_tau psi(y+) e_x, largest at the outermost
    of the q_w wall-normal Gauss points of a wall cell: rate = u_tau psi(y+_q) / h_x there."""
    k, nu, tau_w = 2, 1e-3, 4e-2
    m = O.Mesh(2, 4, 2, k, nu=nu, tau_w=tau_w, n_layers=1)
    u = np.zeros(m.n_u)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = math.sqrt(tau_w)
    X = m.node_coords().reshape(m.nc, -1, 3)
    hx = X[0, :, 0].max() - X[0, :, 0].min()
    hy = X[0, :, 1].max() - X[0, :, 1].min()
    gy, _ = O.gauss(8)
    ut = math.sqrt(tau_w)
    ref = max(ut * O.psi_spalding(y * hy * ut / nu)[0] for y in gy) / hx
    assert abs(m.cfl_rate(u) / ref - 1.0) < 1e-12


def test_variable_step_bdf2_and_extrapolation_constants():
    """gamma_0, alpha_i: dt_n times the derivative at t_{n+1} of the quadratic interpolant through three
    unevenly spaced times (NumPy polynomial fit); beta_i: the linear extrapolation; omega = 1 gives the
    constant-step constants exactly."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        d1, d0 = rng.uniform(0.1, 2.0, 2)     # dt_{n-1}, dt_n
        t = np.array([0.0, d1, d1 + d0])       # t_{n-1}, t_n, t_{n+1}
        g0, a0, a1, b0, b1 = O.bdf2_variable(d0 / d1)
        for j in range(3):                     # the quadratic interpolant of the j-th unit vector
            y = np.zeros(3); y[j] = 1.0
            c = np.polyfit(t, y, 2)
            deriv = d0 * np.polyval(np.polyder(c), t[2])
            ref = [-a1, -a0, g0][j]            # u^{n-1}: -alpha_1, u^n: -alpha_0, u^{n+1}: gamma_0
            assert abs(deriv - ref) < 1e-10 * max(1.0, abs(ref))
        c = np.polyfit(t[:2], [1.0, 0.0], 1)    # extrapolation weight of u^{n-1}
        assert abs(np.polyval(c, t[2]) - b1) < 1e-12
        c = np.polyfit(t[:2], [0.0, 1.0], 1)
        assert abs(np.polyval(c, t[2]) - b0) < 1e-12
    assert O.bdf2_variable(1.0) == (1.5, 2.0, -0.5, 2.0, -1.0)


def test_adaptive_dual_splitting_reduces_to_the_constant_step():
    """When the CFL step is larger than dt the adaptive integrator takes dt in every step and equals the
    constant-step one (velocities bit for bit; the pressure to the rounding of the oracle's threaded
    CG reductions); when it binds, dt_n = Cr / (k^1.5 rate(u^n)) and Poiseuille flow
    still stays steady (variable BDF2 constants sum to zero on a steady state)."""
    nu, U = 1e-2, 1.0
    m = O.Mesh(4, 4, 2, 2, n_layers=0, nu=nu)
    u0 = _std_field(m, lambda x, y, z: U * (1 - y ** 2), lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    force = (2 * nu * U, 0.0, 0.0)
    a = O.DualSplitting(m, u0, dt=5e-3, cr=100.0, force=force, adaptive=True)
    b = O.DualSplitting(m, u0, dt=5e-3, cr=100.0, force=force)
    for _ in range(3):
        ua, pa = a.step()
        ub, pb = b.step()
        assert np.array_equal(ua, ub)
        assert np.abs(pa - pb).max() <= 1e-12 * max(np.abs(pb).max(), 1e-300) or np.abs(pa - pb).max() < 1e-14
    assert a.dts == [5e-3] * 3
    c = O.DualSplitting(m, u0, dt=1.0, cr=0.14, force=force, adaptive=True)
    for _ in range(3):
        u, p = c.step()
    rate = m.cfl_rate(u0)
    assert abs(c.dts[0] / (0.14 / (2 ** 1.5 * rate)) - 1.0) < 1e-14
    assert _l2_rel(m, u, u0) < 1e-11


# ---------------------------------------------------------------------------------------------
# Vorticity and the high-order pressure Neumann data (Sec. 4.1 eq. bc_d_pres)
# ---------------------------------------------------------------------------------------------

def test_curl_weak_form_closed_forms():
    """(v, curl u) for u = (-y^2, 0, 0): curl u = (0, 0, 2y), and v = (0, 0, y) gives int 2 y^2; a
    gradient field u = grad(y^2) has no curl."""
    m = O.Mesh(3, 4, 2, 2, n_layers=0)
    u = _std_field(m, lambda x, y, z: -y ** 2, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    v = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y, lambda x, y, z: y)
    ref = 2 * math.pi * math.pi * 4.0 / 3.0
    assert abs(v @ m.curl(u) / ref - 1.0) < 1e-12
    g = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: 2 * y, lambda x, y, z: 0 * y)
    assert np.abs(m.curl(g)).max() < 1e-13


def test_curl_of_a_linear_field_with_every_gradient_entry():
    """The curl term has no face integrals, so cell-wise linear fields need no continuity: for
    u = (a z + d y, b x + e z, c y + f x) every entry of grad u is set and curl u = (c - e, a - f, b - d),
    so the standard outputs of component i summed over all test functions give V curl_i."""
    m = O.Mesh(3, 4, 2, 2, n_layers=0)
    a, b, c, d, e, f = 0.3, -0.7, 1.1, 0.4, 0.9, -0.2
    u = _std_field(m, lambda x, y, z: a * z + d * y, lambda x, y, z: b * x + e * z, lambda x, y, z: c * y + f * x)
    y = m.curl(u)[: 3 * m.n_p].reshape(m.nc, 3, -1).sum(axis=(0, 2))
    vol = 4 * math.pi ** 2
    ref = vol * np.array([c - e, a - f, b - d])
    assert np.abs(y - ref).max() < 1e-12 * vol


def test_vorticity_of_a_polynomial_is_exact_with_enrichment():
    """u = (y^3 - y, 0, y^2) (Q3): curl u = (2y, 0, 1 - 3y^2) lies in the velocity space (enrichment
    coefficients zero), so its L2 projection is itself (compared as functions)."""
    w = I.Workload("vo", 3, 4, 2, 3, 395.0, 1.0 / 6000.0, seed=46)
    m = O.Mesh(**w.mesh_kwargs())
    u = _std_field(m, lambda x, y, z: y ** 3 - y, lambda x, y, z: 0 * y, lambda x, y, z: y ** 2)
    ref = _std_field(m, lambda x, y, z: 2 * y, lambda x, y, z: 0 * y, lambda x, y, z: 1 - 3 * y ** 2)
    assert _l2_rel(m, m.vorticity(u), ref) < 1e-10


def test_pressure_neumann_convective_part():
    """u = (0, y, 0): div(u x u) = (0, 2y, 0), curl u = 0, so g = -beta 2y n_y = -2 beta on both walls
    and the wall integrals of q = 1 sum to -2 beta times the wall area of both walls."""
    m = O.Mesh(3, 4, 2, 2, n_layers=0)
    u = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: y, lambda x, y, z: 0 * y)
    beta = 1.5
    y = m.pressure_neumann(u, m.vorticity(u), beta)
    ref = -2 * beta * 2 * (2 * math.pi * math.pi)
    assert abs(y.sum() / ref - 1.0) < 1e-12


def test_pressure_neumann_convective_part_with_enrichment():
    """ubar = (0, V, W z) and u~ = psi(y+) (0, b, 0) (all weights b), omega = 0: at a wall psi = 0, so
    u = ubar there while grad u~ = b psi'(0) grad y+ = +-b (u_tau/nu) e_y (sign of the wall's normal
    distance), and div(u x u) . e_y = u_y div u + u . grad u_y = V (2 s b + W) on the bottom wall and
    V (W - 2 s b) on the top wall (s = u_tau / nu). With n = -e_y and +e_y the wall integrals of q = 1
    are L_x L_z beta V (2 s b + W) and L_x L_z beta V (2 s b - W), each wall on its own."""
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs())
    V, W, b, beta = 0.4, 0.3, 1e-3, 1.5
    u = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: V + 0 * y, lambda x, y, z: W * z)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 1, :] = b
    y = m.pressure_neumann(u, np.zeros(m.n_u), beta).reshape(w.nz, w.ny, w.nx, -1)
    s = w.u_tau / w.nu
    area = w.lx * w.lz
    bottom, top = y[:, 0].sum(), y[:, w.ny - 1].sum()
    assert abs(bottom / (area * beta * V * (2 * s * b + W)) - 1.0) < 1e-12
    assert abs(top / (area * beta * V * (2 * s * b - W)) - 1.0) < 1e-12


def test_pressure_neumann_on_the_sloped_bump_wall():
    """u = (a x, 0, 0) cell by cell on the bump (the data are per wall face, so no continuity is needed):
    div(u x u) = (2 a^2 x, 0, 0), and on the bump wall n dA = (y_w'(x), -1, 0) dx dz, so the bottom
    wall's integral of q = 1 is -2 beta a^2 L_z int x y_w'(x) dx = 2 beta a^2 L_z int y_w dx (periodic,
    y_w = 0 at the ends), with y_w the mesh's Q_k wall, whose bump area is 9 * 3.036 - V / L_z (V the
    separately pinned volume; both integrals are exact for the polynomial map); the flat top wall gets
    nothing. A body force f = (0, f_y, 0) adds f . n: -f_y L_x L_z on the bump wall (n_y dA = -dx dz
    there, whatever the slope) and +f_y L_x L_z on the top wall. The viscous part nu curl(omega) . n
    reaches the bump wall through n_x: with omega = (0, c x z, 0) it is -beta nu c L_z A_w."""
    m = O.Mesh(12, 4, 1, 3, lx=9.0, ly=3.036, lz=4.5, geometry=1, n_layers=0)
    a, beta, fy = 0.7, 1.5, 0.25
    u = _std_field(m, lambda x, y, z: a * x, lambda x, y, z: 0 * y, lambda x, y, z: 0 * y)
    y = m.pressure_neumann(u, np.zeros(m.n_u), beta).reshape(1, 4, 12, -1)
    area = 9.0 * 3.036 - m.volume() / 4.5
    assert abs(area / 0.3 - 1.0) < 1e-2
    ref = 2 * beta * a * a * 4.5 * area
    assert abs(y[:, 0].sum() / ref - 1.0) < 1e-11
    assert abs(y[:, 3].sum()) < 1e-12 * ref
    yf = m.pressure_neumann(u, np.zeros(m.n_u), beta, f=(0.0, fy, 0.0)).reshape(1, 4, 12, -1)
    assert abs(yf[:, 0].sum() / (ref - fy * 9.0 * 4.5) - 1.0) < 1e-11
    assert abs(yf[:, 3].sum() / (fy * 9.0 * 4.5) - 1.0) < 1e-11
    # viscous part: u = 0 and omega = (0, c x z, 0) cell by cell, curl omega = (-c x, 0, c z), so the
    # bump wall gets -beta nu int (-c x) n_x dA = beta nu c L_z int x y_w' dx = -beta nu c L_z A_w
    nu, c = m.params.nu, 0.9
    om = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: c * x * z, lambda x, y, z: 0 * y)
    yv = m.pressure_neumann(np.zeros(m.n_u), om, beta).reshape(1, 4, 12, -1)
    refv = -beta * nu * c * 4.5 * area
    assert abs(yv[:, 0].sum() / refv - 1.0) < 1e-11
    assert abs(yv[:, 3].sum()) < 1e-12 * abs(refv)


def test_pressure_neumann_viscous_part():
    """u = (0, sin(kx), 0): curl u = (0, 0, k cos kx), curl curl u = (0, k^2 sin kx, 0), the convective
    part vanishes; with q = y sin(kx), sum of q g over both walls = -2 beta nu k^2 (L_x/2) L_z. The
    vorticity is the L2 projection of the interpolated sine's curl (tolerance: interpolation error)."""
    nu, beta = 1e-2, 2.0
    m = O.Mesh(16, 2, 1, 4, n_layers=0, nu=nu)
    kap = 1.0
    u = _std_field(m, lambda x, y, z: 0 * y, lambda x, y, z: np.sin(kap * x), lambda x, y, z: 0 * y)
    X = m.node_coords()
    q = X[:, 1] * np.sin(kap * X[:, 0])
    y = m.pressure_neumann(u, m.vorticity(u), beta)
    ref = -2 * beta * nu * kap ** 2 * math.pi * math.pi
    # the degree-4 interpolant of the sine on h = 2 pi / 16 differs by ~(h/2)^5 / 5! ~ 2e-6, and the
    # curl-curl takes two derivatives of it
    assert abs(q @ y / ref - 1.0) < 1e-4


# ---------------------------------------------------------------------------------------------
# Paper-literal enriched quadrature (Sec. 4.4: q_w points in every direction of enriched cells and
# per tangential direction of faces touching them)
# ---------------------------------------------------------------------------------------------

def test_full_enriched_quadrature_keeps_the_pinned_invariants():
    """With q_w^3 points in the wall cells: the shear-flow invariant of the convective term, the psi and
    psi^2 integrals of the mass, and polynomial exactness of the Laplace-free operators hold as before;
    for polynomial fields (no enrichment content) both rules integrate exactly, so the standard outputs
    agree with the default rule to rounding."""
    from scipy.integrate import quad
    w = I.WORKLOADS["channel_q2_8x8x8"]
    m = O.Mesh(**w.mesh_kwargs(), full_quadrature=True)
    m0 = O.Mesh(**w.mesh_kwargs())
    f = [lambda x, y, z: 0 * y] * 3
    f[0] = lambda x, y, z: 1 - y ** 2
    u = _std_field(m, *f)
    u[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = w.u_tau
    assert np.abs(m.convective(u)).max() < 1e-14
    e = np.zeros(m.n_u)
    e[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :] = 1.0
    y = m.vmass(e)
    dy = 1.0 + math.tanh(1.8 * (2.0 / 8 - 1.0)) / math.tanh(1.8)
    ref2 = 2 * (2 * math.pi * math.pi) * quad(lambda s: O.psi_spalding(s * w.u_tau / w.nu)[0] ** 2, 0.0, dy,
                                              epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    assert abs(y[3 * m.n_p:].reshape(m.n_e, 3, 8)[:, 0, :].sum() / ref2 - 1.0) < 1e-6
    p = _std_field(m, lambda x, y, z: y ** 2, lambda x, y, z: 1 + y + 0 * x, lambda x, y, z: y * z)
    for op in ("vmass", "divergence"):
        a, b = getattr(m, op)(p), getattr(m0, op)(p)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
