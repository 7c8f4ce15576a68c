"""Plain FP64 CPU oracle for the DG wall-model operators (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It wraps ``dgw_oracle.c`` (plain C, OpenMP over cells, full 3-D tabulation of the
basis at every quadrature point, no sum factorisation) through ctypes and shares nothing with the
CUDA library.

Paper: Krank, Kronbichler & Wall, arXiv 1705.08813. Each C function cites the section or
equation it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgw_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP). Returns the path of the shared library."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("k", ctypes.c_int), ("enrich_l", ctypes.c_int), ("q_wall", ctypes.c_int),
        ("geometry", ctypes.c_int), ("wall_law", ctypes.c_int), ("n_layers", ctypes.c_int),
        ("extra_q", ctypes.c_int), ("full_q", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("nu", ctypes.c_double), ("tau_w", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        vp = ctypes.c_void_p
        lib.dgo_mesh_create.restype = vp
        lib.dgo_mesh_create.argtypes = [ctypes.POINTER(Params)]
        lib.dgo_mesh_destroy.argtypes = [vp]
        lib.dgo_mesh_info.argtypes = [vp, lp, lp, lp]
        lib.dgo_node_coords.argtypes = [vp, dp]
        lib.dgo_cell_tau.argtypes = [vp, dp]
        for name in ("dgo_laplace", "dgo_divergence", "dgo_convective", "dgo_laplace_diag"):
            getattr(lib, name).argtypes = [vp, dp, dp] if name != "dgo_laplace_diag" else [vp, dp]
            getattr(lib, name).restype = ctypes.c_int
        lib.dgo_viscous.argtypes = [vp, dp, dp, dp]
        lib.dgo_mass.argtypes = [vp, dp, dp]
        lib.dgo_vmass.argtypes = [vp, dp, dp]
        lib.dgo_set_active.argtypes = [vp, ctypes.c_void_p]
        lib.dgo_solve_cg.argtypes = [vp, dp, dp, ctypes.c_double, ctypes.c_int, ip, dp]
        lib.dgo_eval_point.argtypes = [vp, dp, ctypes.c_int, dp, dp]
        lib.dgo_nut_cell.argtypes = [vp, dp, ctypes.c_int, dp]
        lib.dgo_nut_cell.restype = ctypes.c_int
        lib.dgo_wall_nodes.argtypes = [vp]
        lib.dgo_wall_nodes.restype = ctypes.c_int
        lib.dgo_set_tau_nodes.argtypes = [vp, dp]
        lib.dgo_wall_shear.argtypes = [vp, dp, dp]
        lib.dgo_wall_shear.restype = ctypes.c_int
        lib.dgo_project.argtypes = [vp, dp, dp, dp]
        lib.dgo_set_switch.argtypes = [vp, ctypes.c_double]
        lib.dgo_gradient.argtypes = [vp, dp, dp]
        lib.dgo_curl.argtypes = [vp, dp, dp]
        lib.dgo_pressure_neumann.argtypes = [vp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.dgo_divdiv.argtypes = [vp, dp, dp, dp]
        lib.dgo_tau_divdiv.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.dgo_cfl_rate.argtypes = [vp, dp]
        lib.dgo_cfl_rate.restype = ctypes.c_double
        lib.dgo_inverse_mass.argtypes = [vp, dp, dp]
        lib.dgo_inverse_mass.restype = ctypes.c_int
        lib.dgo_active.argtypes = [vp, ip]
        lib.dgo_active.restype = ctypes.c_int
        lib.dgo_project.restype = ctypes.c_int
        lib.dgo_volume.argtypes = [vp]
        lib.dgo_volume.restype = ctypes.c_double
        lib.dgo_psi_spalding.argtypes = [ctypes.c_double, dp]
        lib.dgo_psi_spalding.restype = ctypes.c_double
        lib.dgo_psi_vandriest.argtypes = [ctypes.c_double, dp]
        lib.dgo_psi_vandriest.restype = ctypes.c_double
        lib.dgo_psi_vd_from.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.dgo_psi_vd_from.restype = ctypes.c_double
        lib.dgo_gauss.argtypes = [ctypes.c_int, dp, dp]
        lib.dgo_lobatto.argtypes = [ctypes.c_int, dp]
        lib.dgo_num_threads.restype = ctypes.c_int
        lib.dgo_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gauss(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (nodes ascending, weights)."""
    x = np.zeros(n); w = np.zeros(n)
    _load().dgo_gauss(n, _ptr(x), _ptr(w))
    return x, w


def lobatto(n: int):
    """n Gauss-Lobatto nodes on [0, 1]."""
    x = np.zeros(n)
    _load().dgo_lobatto(n, _ptr(x))
    return x


def psi_spalding(yp: float):
    """Spalding wall law inverted for psi = u+(y+); returns (psi, dpsi/dy+)."""
    d = ctypes.c_double()
    v = _load().dgo_psi_spalding(float(yp), ctypes.byref(d))
    return v, d.value


def psi_vandriest(yp: float):
    """van Driest wall law, eq. (psi), evaluated as in Appendix A; returns (psi, dpsi/dy+)."""
    d = ctypes.c_double()
    v = _load().dgo_psi_vandriest(float(yp), ctypes.byref(d))
    return v, d.value


def psi_vandriest_from(i: int, yp: float) -> float:
    """psi_i + 9-point Gauss integral over [y_i+, y+] from Table A1 row i (eq. psinum)."""
    return _load().dgo_psi_vd_from(int(i), float(yp))


def set_threads(n: int) -> None:
    _load().dgo_set_threads(int(n))


def num_threads() -> int:
    return _load().dgo_num_threads()


class Mesh:
    """Oracle mesh of a channel (geometry 0) or bump channel (geometry 1)."""

    def __init__(self, nx, ny, nz, k, *, lx=2 * np.pi, ly=2.0, lz=np.pi, gamma=1.8, nu=1.0 / 3250,
                 tau_w=1.0, enrich_l=1, q_wall=8, geometry=0, wall_law=0, n_layers=1, extra_q=0,
                 full_quadrature=False):
        self.lib = _load()
        self.params = Params(nx, ny, nz, k, enrich_l, q_wall, geometry, wall_law, n_layers, extra_q,
                             1 if full_quadrature else 0, lx, ly, lz, gamma, nu, tau_w)
        h = self.lib.dgo_mesh_create(ctypes.byref(self.params))
        if not h:
            raise ValueError("oracle: invalid mesh parameters")
        self.h = ctypes.c_void_p(h)
        np_, nu_, ne_ = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        self.lib.dgo_mesh_info(self.h, ctypes.byref(np_), ctypes.byref(nu_), ctypes.byref(ne_))
        self.n_p, self.n_u, self.n_e = np_.value, nu_.value, ne_.value
        self.k = k
        self.nc = nx * ny * nz

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.dgo_mesh_destroy(h)
            self.h = None

    def set_active(self, cells=None) -> None:
        """Compute only the outputs of the given cells in later operator calls (None: all)."""
        if cells is None:
            self.lib.dgo_set_active(self.h, None)
            return
        mask = np.zeros(self.nc, dtype=np.uint8)
        mask[np.asarray(cells, dtype=np.int64)] = 1
        self._mask = mask
        self.lib.dgo_set_active(self.h, mask.ctypes.data_as(ctypes.c_void_p))

    def node_coords(self) -> np.ndarray:
        out = np.zeros((self.n_p, 3))
        self.lib.dgo_node_coords(self.h, _ptr(out))
        return out

    def cell_tau(self) -> np.ndarray:
        out = np.zeros(self.nc)
        self.lib.dgo_cell_tau(self.h, _ptr(out))
        return out

    def volume(self) -> float:
        return self.lib.dgo_volume(self.h)

    def laplace(self, p: np.ndarray) -> np.ndarray:
        p = np.ascontiguousarray(p, dtype=np.float64); y = np.zeros(self.n_p)
        self.lib.dgo_laplace(self.h, _ptr(p), _ptr(y))
        return y

    def mass(self, p: np.ndarray) -> np.ndarray:
        p = np.ascontiguousarray(p, dtype=np.float64); y = np.zeros(self.n_p)
        self.lib.dgo_mass(self.h, _ptr(p), _ptr(y))
        return y

    def vmass(self, u: np.ndarray) -> np.ndarray:
        """Velocity mass operator on standard and enriched DoFs (n_u values in, n_u out)."""
        u = np.ascontiguousarray(u, dtype=np.float64); y = np.zeros(self.n_u)
        self.lib.dgo_vmass(self.h, _ptr(u), _ptr(y))
        return y

    def laplace_diag(self) -> np.ndarray:
        y = np.zeros(self.n_p)
        self.lib.dgo_laplace_diag(self.h, _ptr(y))
        return y

    def divergence(self, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64); b = np.zeros(self.n_p)
        self.lib.dgo_divergence(self.h, _ptr(u), _ptr(b))
        return b

    def convective(self, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64); y = np.zeros(self.n_u)
        self.lib.dgo_convective(self.h, _ptr(u), _ptr(y))
        return y

    def viscous(self, u_frozen: np.ndarray, u: np.ndarray) -> np.ndarray:
        uf = np.ascontiguousarray(u_frozen, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64); y = np.zeros(self.n_u)
        self.lib.dgo_viscous(self.h, _ptr(uf), _ptr(u), _ptr(y))
        return y

    def solve(self, b: np.ndarray, rtol=1e-12, maxit=20000):
        b = np.ascontiguousarray(b, dtype=np.float64); p = np.zeros(self.n_p)
        it, rr = ctypes.c_int(), ctypes.c_double()
        self.lib.dgo_solve_cg(self.h, _ptr(b), _ptr(p), rtol, maxit, ctypes.byref(it), ctypes.byref(rr))
        return p, it.value, rr.value

    def eval_point(self, u: np.ndarray, cell: int, xi) -> dict:
        u = np.ascontiguousarray(u, dtype=np.float64)
        xi = np.ascontiguousarray(xi, dtype=np.float64); out = np.zeros(12)
        self.lib.dgo_eval_point(self.h, _ptr(u), int(cell), _ptr(xi), _ptr(out))
        return {"u": out[0:3], "ubar": out[3:6], "util": out[6:9], "psi": out[9],
                "yplus": out[10], "nut": out[11]}

    @property
    def n_wall_nodes(self) -> int:
        """Linear wall nodes: 2 walls x nx x nz (periodic), index wall * nx * nz + i + nx * k."""
        return self.lib.dgo_wall_nodes(self.h)

    def wall_shear(self, u: np.ndarray) -> np.ndarray:
        """Nodal wall shear stress tau_w,B = |int N_B nu (grad u) n dA| / int N_B dA (Sec. 3.2)."""
        u = np.ascontiguousarray(u, dtype=np.float64); out = np.zeros(self.n_wall_nodes)
        self.lib.dgo_wall_shear(self.h, _ptr(u), _ptr(out))
        return out

    def set_tau_nodes(self, tau_nodes: np.ndarray) -> None:
        """Set the wall shear stress of every wall node (enriched-cell vertices off the wall take the
        value of the wall node that defines their wall distance); changes the enrichment space."""
        tn = np.ascontiguousarray(tau_nodes, dtype=np.float64)
        assert tn.size == self.n_wall_nodes
        self.lib.dgo_set_tau_nodes(self.h, _ptr(tn))

    def project(self, tau_new: np.ndarray, u_old: np.ndarray) -> np.ndarray:
        """Cell-wise L2 projection of u_old (current space) onto the space of the nodal wall shear
        stress tau_new (eq. l2); the mesh keeps tau_new afterwards."""
        tn = np.ascontiguousarray(tau_new, dtype=np.float64)
        u = np.ascontiguousarray(u_old, dtype=np.float64); out = np.zeros(self.n_u)
        assert tn.size == self.n_wall_nodes
        if self.lib.dgo_project(self.h, _ptr(tn), _ptr(u), _ptr(out)) != 0:
            raise RuntimeError("singular cell system in the L2 projection")
        return out

    def gradient(self, p: np.ndarray) -> np.ndarray:
        """Pressure gradient P(v, p) = -(div v, p) + (v, {{p}} n), {{p}} = p^- on walls (n_p in, n_u out)."""
        p = np.ascontiguousarray(p, dtype=np.float64); y = np.zeros(self.n_u)
        self.lib.dgo_gradient(self.h, _ptr(p), _ptr(y))
        return y

    def curl(self, u: np.ndarray) -> np.ndarray:
        """y = (v, curl u)_K for every velocity test function; the vorticity is inverse_mass(y)."""
        u = np.ascontiguousarray(u, dtype=np.float64); y = np.zeros(self.n_u)
        self.lib.dgo_curl(self.h, _ptr(u), _ptr(y))
        return y

    def vorticity(self, u: np.ndarray) -> np.ndarray:
        """omega_h: L2 projection of curl u onto the velocity space."""
        return self.inverse_mass(self.curl(u))

    def pressure_neumann(self, u0, w0, b0, u1=None, w1=None, b1=0.0, f=(0.0, 0.0, 0.0)) -> np.ndarray:
        """Wall integrals (q, g), g = -(sum beta_i (div(u x u) + nu curl omega)(history i) - f) . n."""
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (u0, w0)]
        b = [np.ascontiguousarray(x if x is not None else u0, dtype=np.float64) for x in (u1, w1)]
        fv = np.ascontiguousarray(f, dtype=np.float64); y = np.zeros(self.n_p)
        self.lib.dgo_pressure_neumann(self.h, _ptr(a[0]), _ptr(b[0]), _ptr(a[1]), _ptr(b[1]), float(b0),
                                      float(b1 if u1 is not None else 0.0), _ptr(fv), _ptr(y))
        return y

    def cfl_rate(self, u: np.ndarray) -> float:
        """Largest |J^-1 (ubar + u~)|_2 over the linear volume point set of every cell: the speed in
        reference-cell lengths per unit time that sets the adaptive time step Cr / (k^1.5 rate)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        return float(self.lib.dgo_cfl_rate(self.h, _ptr(u)))

    def tau_divdiv(self, u: np.ndarray, dt: float, cr: float) -> np.ndarray:
        """Per-cell tau_D = |u|_K h dt / Cr (volume-averaged |u|, h = cube root of the cell volume)."""
        u = np.ascontiguousarray(u, dtype=np.float64); out = np.zeros(self.nc)
        self.lib.dgo_tau_divdiv(self.h, _ptr(u), float(dt), float(cr), _ptr(out))
        return out

    def divdiv(self, tau_d: np.ndarray, u: np.ndarray) -> np.ndarray:
        """Div-div penalty D(v, u) = (div v, tau_D div u) per cell."""
        t = np.ascontiguousarray(tau_d, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64); y = np.zeros(self.n_u)
        self.lib.dgo_divdiv(self.h, _ptr(t), _ptr(u), _ptr(y))
        return y

    def inverse_mass(self, r: np.ndarray) -> np.ndarray:
        """x = M^-1 r, cell by cell (dense cell systems)."""
        r = np.ascontiguousarray(r, dtype=np.float64); x = np.zeros(self.n_u)
        if self.lib.dgo_inverse_mass(self.h, _ptr(r), _ptr(x)) != 0:
            raise RuntimeError("singular cell mass matrix")
        return x

    def set_switch(self, yplus_off: float) -> None:
        """Switch the wall model off in every wall column whose wall-nearest cell has y+ < yplus_off at
        all of its points (0: never); re-evaluated whenever tau_w changes."""
        self.lib.dgo_set_switch(self.h, float(yplus_off))

    def active(self) -> np.ndarray:
        """Per enriched index: 1 if the enrichment is switched on."""
        out = np.zeros(max(self.n_e, 1), dtype=np.int32)
        self.lib.dgo_active(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return out[: self.n_e]

    def nut_cell(self, u: np.ndarray, e: int) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64); out = np.zeros(4096)
        n = self.lib.dgo_nut_cell(self.h, _ptr(u), int(e), _ptr(out))
        return out[:n]


def _gmres(apply, b, x0, prec, rtol, restart=60, maxit=3000):
    """Restarted right-preconditioned GMRES (Saad's algorithm, modified Gram-Schmidt), numpy."""
    x = x0.copy()
    nb = np.linalg.norm(b)
    it = 0
    while it < maxit:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * nb:
            return x, it
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        for j in range(restart):
            z = prec(V[j])
            Z.append(z)
            w = apply(z)
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            it += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(H[: j + 2, : j + 1] @ y - e1)
            if res <= rtol * nb * 0.5 or H[j + 1, j] == 0.0 or it >= maxit:
                break
            V.append(w / H[j + 1, j])
        x = x + sum(yi * zi for yi, zi in zip(y, Z))
    return x, it


def _pcg(apply, b, x0, prec, rtol, maxit=5000):
    """Preconditioned conjugate gradients (Hestenes-Stiefel), numpy."""
    x = x0.copy()
    r = b - apply(x)
    z = prec(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for it in range(maxit):
        if np.linalg.norm(r) <= rtol * nb:
            return x, it
        q = apply(p)
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = prec(r)
        rz2 = r @ z
        p = z + (rz2 / rz) * p
        rz = rz2
    raise RuntimeError("projection CG did not converge")


def bdf2_variable(omega):
    """(gamma_0, alpha_0, alpha_1, beta_0, beta_1) of the second-order BDF and extrapolation for the
    step ratio omega = dt_n / dt_{n-1} (Sec. 4.1: the constants follow the variable increments): the
    derivative at t_{n+1} of the quadratic through u^{n+1}, u^n, u^{n-1} times dt_n is
    gamma_0 u^{n+1} - alpha_0 u^n - alpha_1 u^{n-1}, and beta_0 u^n + beta_1 u^{n-1} is the linear
    extrapolation to t_{n+1}."""
    w = float(omega)
    return (1.0 + 2.0 * w) / (1.0 + w), 1.0 + w, -w * w / (1.0 + w), 1.0 + w, -w


class DualSplitting:
    """One constant-step BDF2/extrapolation step of the dual-splitting scheme after Sec. 4.1 with the
    Galerkin forms of Sec. 4.2, written with this module's operators (first order in the first step):
    convective step with the exact inverse mass, pressure Poisson solve (homogeneous Neumann data, or
    with high_order_pressure_bc the data of eq. bc_d_pres from u^{n-i} and their vorticities), the
    projection (M + D) u^^ = M u^ - (dt / gamma_0) P(p) by preconditioned CG, and the viscous
    Helmholtz step by GMRES, nu_t and tau_D from u^n. With update_wall_model the step starts with the
    wall shear stress of u^n, the L2 projection of u^n and u^{n-1} onto the new space and a new
    F^c(u^{n-1}). With adaptive the step is dt_n = min(dt, Cr / (k^1.5 cfl_rate(u^n))) and the
    constants those of bdf2_variable for dt_n / dt_{n-1}."""

    def __init__(self, mesh: "Mesh", u0, dt, cr=0.14, force=(0.0, 0.0, 0.0), rtol=1e-13,
                 update_wall_model=False, tau_nodes=None, high_order_pressure_bc=False, adaptive=False):
        self.m, self.dt, self.cr, self.rtol = mesh, float(dt), float(cr), float(rtol)
        self.adaptive = bool(adaptive)
        self.dt_prev = None
        self.dts = []
        self.u = [np.array(u0, dtype=np.float64), None]
        self.fc_old = None
        self.p = np.zeros(mesh.n_p)
        self.steps = 0
        self.update = update_wall_model
        self.hobc = high_order_pressure_bc
        self.force = tuple(float(x) for x in force)
        self.tau = (np.full(mesh.n_wall_nodes, mesh.params.tau_w) if tau_nodes is None
                    else np.array(tau_nodes, dtype=np.float64))
        n3 = (mesh.k + 1) ** 3
        self.f = np.zeros(mesh.n_u)
        std = self.f[: 3 * mesh.n_p].reshape(mesh.nc, 3, n3)
        for a in range(3):
            std[:, a, :] = force[a]

    def step(self):
        m, dt = self.m, self.dt
        second = self.steps > 0
        if self.adaptive:
            rate = m.cfl_rate(self.u[0])
            if rate > 0.0:
                dt = min(dt, self.cr / (m.k ** 1.5 * rate))
        if not second:
            g0, a0, a1, b0, b1 = (1.0, 1.0, 0.0, 1.0, 0.0)
        elif self.adaptive:
            g0, a0, a1, b0, b1 = bdf2_variable(dt / self.dt_prev)
        else:
            g0, a0, a1, b0, b1 = (1.5, 2.0, -0.5, 2.0, -1.0)
        if self.update and m.n_e > 0:
            tn = m.wall_shear(self.u[0])
            old = self.tau
            un = m.project(tn, self.u[0])
            if second:
                m.set_tau_nodes(old)
                self.u[1] = m.project(tn, self.u[1])
                self.fc_old = m.convective(self.u[1])
            self.u[0] = un
            self.tau = tn
        un, unm = self.u
        fc = m.convective(un)
        if self.hobc:
            wn = m.vorticity(un)
            wnm = m.vorticity(unm) if second else None
        w = b0 * fc + (b1 * self.fc_old if second else 0.0)
        uh = (a0 * un + (a1 * unm if second else 0.0) + dt * self.f - dt * m.inverse_mass(w)) / g0
        b = (g0 / dt) * m.divergence(uh)
        if self.hobc:
            b = b + m.pressure_neumann(un, wn, b0, unm if second else None, wnm, b1 if second else 0.0, self.force)
        p, _, _ = m.solve(b, rtol=self.rtol, maxit=200000)
        tau_d = m.tau_divdiv(un, dt, self.cr)
        rhs = m.vmass(uh) - (dt / g0) * m.gradient(p)
        uhh, _ = _pcg(lambda v: m.vmass(v) + m.divdiv(tau_d, v), rhs, uh, m.inverse_mass, self.rtol)
        gam = g0 / dt
        rhs3 = gam * m.vmass(uhh)
        unew, _ = _gmres(lambda v: gam * m.vmass(v) + m.viscous(un, v), rhs3, uhh,
                         lambda v: m.inverse_mass(v) / gam, self.rtol)
        self.u = [unew, un]
        self.fc_old = fc
        self.p = p
        self.steps += 1
        self.dt_prev = dt
        self.dts.append(dt)
        return unew, p
