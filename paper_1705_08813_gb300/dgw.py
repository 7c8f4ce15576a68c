"""Thin ctypes binding of libdgw.so (argument marshalling only; every step runs in the CUDA
library). Device vectors are torch tensors; their data pointers and the current CUDA stream are
passed through the C ABI declared in include/dgw.h."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdgw.so")

DGW_FP64 = 0
DGW_FP32 = 1
DGW_DF64 = 2   # double vectors, double-float arithmetic on the FP32 units
STATUS = {0: "DGW_OK", -1: "DGW_EINVAL", -2: "DGW_ENOMEM", -3: "DGW_ENOTCONV", -4: "DGW_ETIMEOUT",
          -5: "DGW_EBUSY", -6: "DGW_ECUDA", -7: "DGW_EDEVICE"}

# every symbol include/dgw.h declares
EXPORTS = ["dgw_mesh_create", "dgw_mesh_destroy", "dgw_mesh_info", "dgw_mesh_node_coords",
           "dgw_update_eddy_viscosity", "dgw_apply_laplace", "dgw_apply_divergence",
           "dgw_apply_convective", "dgw_apply_viscous", "dgw_apply_divergence_prec", "dgw_pressure_solve", "dgw_last_error",
           "dgw_counters", "dgw_solver_describe", "dgw_pressure_solve_jacobi_noalloc", "dgw_pressure_solve_batch",
           "dgw_server_create", "dgw_submit", "dgw_poll", "dgw_server_stats", "dgw_server_destroy",
           "dgw_apply_mass", "dgw_helmholtz_solve", "dgw_wall_shear_stress", "dgw_set_wall_shear_stress",
           "dgw_project_velocity", "dgw_set_enrichment_switch", "dgw_enrichment_active",
           "dgw_apply_gradient", "dgw_tau_divdiv", "dgw_apply_divdiv", "dgw_apply_inverse_mass",
           "dgw_ns_create", "dgw_ns_destroy", "dgw_ns_step", "dgw_ns_state", "dgw_ns_copy_state",
           "dgw_apply_curl", "dgw_add_pressure_neumann", "dgw_cfl_rate"]

JOB_SOLVE, JOB_LAPLACE, JOB_DIVERGENCE, JOB_CONVECTIVE, JOB_VISCOUS = 0, 1, 2, 3, 4


class DGWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class NSParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("cr", ctypes.c_double), ("force", ctypes.c_double * 3),
                ("rtol_pressure", ctypes.c_double), ("rtol_projection", ctypes.c_double),
                ("rtol_viscous", ctypes.c_double), ("max_iter", ctypes.c_int), ("pressure_mode", ctypes.c_int),
                ("update_wall_model", ctypes.c_int), ("pressure_bc", ctypes.c_int), ("adaptive_dt", ctypes.c_int)]


class NSStepInfo(ctypes.Structure):
    _fields_ = [("pressure_iterations", ctypes.c_int), ("projection_iterations", ctypes.c_int),
                ("viscous_iterations", ctypes.c_int), ("ms", ctypes.c_double), ("dt", ctypes.c_double)]


class MeshParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("degree", ctypes.c_int), ("enrich_l", ctypes.c_int), ("q_wall", ctypes.c_int),
                ("geometry", ctypes.c_int), ("wall_law", ctypes.c_int), ("n_layers", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("stretch_gamma", ctypes.c_double), ("nu", ctypes.c_double), ("tau_w", ctypes.c_double),
                ("precision_mask", ctypes.c_int), ("full_quadrature", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mode", ctypes.c_int),
                ("cheb_degree", ctypes.c_int)]


class HelmholtzOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("restart", ctypes.c_int)]


class Job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("prec", ctypes.c_int), ("mesh", MeshParams),
                ("inp", ctypes.c_void_p), ("out", ctypes.c_void_p), ("aux", ctypes.c_void_p), ("opts", SolveOpts)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double), ("ms", ctypes.c_float),
                ("dof_applies", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libdgw.so; raises if the CUDA extension has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdgw.so not found at {path}: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, dp, lp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)
    lib.dgw_mesh_create.argtypes = [ctypes.POINTER(MeshParams), vp, ctypes.POINTER(vp)]
    lib.dgw_mesh_destroy.argtypes = [vp]
    lib.dgw_mesh_info.argtypes = [vp, lp, lp, lp, ctypes.POINTER(ctypes.c_size_t)]
    lib.dgw_mesh_node_coords.argtypes = [vp, dp]
    lib.dgw_update_eddy_viscosity.argtypes = [vp, vp, vp]
    lib.dgw_apply_laplace.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.dgw_apply_divergence.argtypes = [vp, vp, vp, vp]
    lib.dgw_apply_divergence_prec.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.dgw_apply_convective.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.dgw_apply_viscous.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.dgw_pressure_solve.argtypes = [vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.dgw_pressure_solve_batch.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                             ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.dgw_solver_describe.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp,
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int, vp]
    lib.dgw_pressure_solve_jacobi_noalloc.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int,
                                                      ctypes.POINTER(SolveInfo), vp]
    lib.dgw_apply_mass.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.dgw_wall_shear_stress.argtypes = [vp, vp, vp, vp]
    lib.dgw_set_wall_shear_stress.argtypes = [vp, vp, vp]
    lib.dgw_project_velocity.argtypes = [vp, vp, vp, vp, vp]
    lib.dgw_set_enrichment_switch.argtypes = [vp, ctypes.c_double, vp]
    lib.dgw_apply_gradient.argtypes = [vp, vp, vp, vp]
    lib.dgw_apply_curl.argtypes = [vp, vp, vp, vp]
    lib.dgw_add_pressure_neumann.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_double), vp, vp]
    lib.dgw_ns_create.argtypes = [vp, ctypes.POINTER(NSParams), vp, vp, ctypes.POINTER(vp)]
    lib.dgw_ns_destroy.argtypes = [vp]
    lib.dgw_ns_step.argtypes = [vp, ctypes.POINTER(NSStepInfo), vp]
    lib.dgw_ns_state.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int)]
    lib.dgw_ns_copy_state.argtypes = [vp, vp, vp, vp]
    lib.dgw_tau_divdiv.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, vp, vp]
    lib.dgw_cfl_rate.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.dgw_apply_divdiv.argtypes = [vp, vp, vp, vp, vp]
    lib.dgw_apply_inverse_mass.argtypes = [vp, vp, vp, vp]
    lib.dgw_enrichment_active.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), vp]
    lib.dgw_helmholtz_solve.argtypes = [vp, ctypes.c_double, vp, vp, ctypes.POINTER(HelmholtzOpts),
                                        ctypes.POINTER(SolveInfo), vp]
    lib.dgw_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]
    lib.dgw_submit.argtypes = [vp, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_long)]
    lib.dgw_poll.argtypes = [vp, ctypes.c_long, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(SolveInfo),
                             ctypes.POINTER(ctypes.c_double)]
    lib.dgw_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]
    lib.dgw_server_destroy.argtypes = [vp, ctypes.c_int]
    lib.dgw_last_error.restype = ctypes.c_char_p
    lib.dgw_counters.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]
    lib.dgw_counters.restype = None
    for name in EXPORTS:
        if name not in ("dgw_last_error", "dgw_counters"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise DGWError(status, (_lib.dgw_last_error() or b"").decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """A device-resident mesh of the channel with its metric and wall tables."""

    def __init__(self, nx, ny, nz, k, *, lx, ly=2.0, lz, gamma=1.8, nu, tau_w, n_layers=1, q_wall=8,
                 wall_law=0, enrich_l=1, geometry=0, fp32=True, full_quadrature=False, stream=None):
        lib = load()
        self.lib = lib
        self.params = MeshParams(nx, ny, nz, k, enrich_l, q_wall, geometry, wall_law, n_layers,
                                 lx, ly, lz, gamma, nu, tau_w, 3 if fp32 else 1, 1 if full_quadrature else 0)
        h = ctypes.c_void_p()
        _check(lib.dgw_mesh_create(ctypes.byref(self.params), _stream(stream), ctypes.byref(h)))
        self.h = h
        a, b, c, d = ctypes.c_long(), ctypes.c_long(), ctypes.c_long(), ctypes.c_size_t()
        _check(lib.dgw_mesh_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        self.n_p, self.n_u, self.n_e, self.hbm_bytes = a.value, b.value, c.value, d.value
        self.nc = nx * ny * nz
        self.k = k

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgw_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def node_coords(self):
        import numpy as np
        out = np.zeros((self.n_p, 3))
        _check(self.lib.dgw_mesh_node_coords(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    @staticmethod
    def _prec(t):
        import torch
        return DGW_FP64 if t.dtype == torch.float64 else DGW_FP32

    def update_eddy_viscosity(self, u, stream=None):
        import torch
        _check(self.lib.dgw_update_eddy_viscosity(self.h, _ptr(u, torch.float64, self.n_u, "u"), _stream(stream)))

    def laplace(self, p, y, stream=None, prec=None):
        """y = A_L p; prec defaults to the tensors' dtype (DGW_DF64: double tensors, double-float
        arithmetic)."""
        _check(self.lib.dgw_apply_laplace(self.h, self._prec(p) if prec is None else prec,
                                          _ptr(p, None, self.n_p, "p"), _ptr(y, p.dtype, self.n_p, "y"),
                                          _stream(stream)))
        return y

    def divergence(self, u, b, stream=None, prec=None):
        """b = -C(q, u) (FP64; prec=DGW_DF64: double-float arithmetic on the box rows)."""
        import torch
        if prec is None or prec == DGW_FP64:
            _check(self.lib.dgw_apply_divergence(self.h, _ptr(u, torch.float64, self.n_u, "u"),
                                                 _ptr(b, torch.float64, self.n_p, "b"), _stream(stream)))
        else:
            _check(self.lib.dgw_apply_divergence_prec(self.h, prec, _ptr(u, torch.float64, self.n_u, "u"),
                                                      _ptr(b, torch.float64, self.n_p, "b"), _stream(stream)))
        return b

    def convective(self, u, y, stream=None, prec=None):
        _check(self.lib.dgw_apply_convective(self.h, self._prec(u) if prec is None else prec,
                                             _ptr(u, None, self.n_u, "u"), _ptr(y, u.dtype, self.n_u, "y"),
                                             _stream(stream)))
        return y

    def viscous(self, u, y, stream=None, prec=None):
        _check(self.lib.dgw_apply_viscous(self.h, self._prec(u) if prec is None else prec,
                                          _ptr(u, None, self.n_u, "u"), _ptr(y, u.dtype, self.n_u, "y"),
                                          _stream(stream)))
        return y

    @property
    def n_wall_nodes(self) -> int:
        """Linear wall nodes: 2 walls x nx x nz, index wall * nx * nz + i + nx * k."""
        return 2 * self.params.nx * self.params.nz

    def wall_shear_stress(self, u, tau_nodes, stream=None):
        """Nodal wall shear stress tau_w,B of the velocity u (FP64) into tau_nodes (FP64 device)."""
        import torch
        _check(self.lib.dgw_wall_shear_stress(self.h, _ptr(u, torch.float64, self.n_u, "u"),
                                              _ptr(tau_nodes, torch.float64, self.n_wall_nodes, "tau_nodes"),
                                              _stream(stream)))
        return tau_nodes

    def set_wall_shear_stress(self, tau_nodes, stream=None):
        """New nodal wall shear stress: rebuilds the enrichment's wall tables (synchronising)."""
        import torch
        _check(self.lib.dgw_set_wall_shear_stress(self.h, _ptr(tau_nodes, torch.float64, self.n_wall_nodes,
                                                               "tau_nodes"), _stream(stream)))

    def project_velocity(self, tau_nodes, u_old, u_new, stream=None):
        """Set a new nodal wall shear stress and L2-project u_old (old space) into u_new (new space)."""
        import torch
        _check(self.lib.dgw_project_velocity(self.h, _ptr(tau_nodes, torch.float64, self.n_wall_nodes, "tau_nodes"),
                                             _ptr(u_old, torch.float64, self.n_u, "u_old"),
                                             _ptr(u_new, torch.float64, self.n_u, "u_new"), _stream(stream)))
        return u_new

    def gradient(self, p, y, stream=None):
        """y = P(v, p), the pressure gradient of the projection step (FP64)."""
        import torch
        _check(self.lib.dgw_apply_gradient(self.h, _ptr(p, torch.float64, self.n_p, "p"),
                                           _ptr(y, torch.float64, self.n_u, "y"), _stream(stream)))
        return y

    def curl(self, u, y, stream=None):
        """y = (v, curl u) per cell; the vorticity is inverse_mass(y)."""
        import torch
        _check(self.lib.dgw_apply_curl(self.h, _ptr(u, torch.float64, self.n_u, "u"),
                                       _ptr(y, torch.float64, self.n_u, "y"), _stream(stream)))
        return y

    def add_pressure_neumann(self, b, u0, w0, beta0, u1=None, w1=None, beta1=0.0, force=(0.0, 0.0, 0.0),
                             stream=None):
        """b += (q, g)_walls, the high-order pressure Neumann data of eq. bc_d_pres."""
        import torch
        f = (ctypes.c_double * 3)(*force)
        p1 = _ptr(u1, torch.float64, self.n_u, "u1") if u1 is not None else None
        q1 = _ptr(w1, torch.float64, self.n_u, "w1") if w1 is not None else None
        _check(self.lib.dgw_add_pressure_neumann(self.h, _ptr(u0, torch.float64, self.n_u, "u0"),
                                                 _ptr(w0, torch.float64, self.n_u, "w0"), ctypes.c_double(beta0),
                                                 p1, q1, ctypes.c_double(beta1), f,
                                                 _ptr(b, torch.float64, self.n_p, "b"), _stream(stream)))
        return b

    def cfl_rate(self, u, stream=None):
        """Largest |J^-1 (ubar + u~)|_2 over the linear volume point set (dgw_cfl_rate): the rate of the
        adaptive time step Cr / (k^1.5 rate)."""
        import torch
        r = ctypes.c_double()
        _check(self.lib.dgw_cfl_rate(self.h, _ptr(u, torch.float64, self.n_u, "u"), ctypes.byref(r), _stream(stream)))
        return r.value

    def tau_divdiv(self, u, dt, cr, tau_d, stream=None):
        """Per-cell tau_D = |u|_K h dt / Cr into tau_d (nc doubles)."""
        import torch
        _check(self.lib.dgw_tau_divdiv(self.h, _ptr(u, torch.float64, self.n_u, "u"), ctypes.c_double(dt),
                                       ctypes.c_double(cr), _ptr(tau_d, torch.float64, self.nc, "tau_d"),
                                       _stream(stream)))
        return tau_d

    def divdiv(self, tau_d, u, y, stream=None):
        """y = D(v, u) = (div v, tau_D div u) per cell."""
        import torch
        _check(self.lib.dgw_apply_divdiv(self.h, _ptr(tau_d, torch.float64, self.nc, "tau_d"),
                                         _ptr(u, torch.float64, self.n_u, "u"), _ptr(y, torch.float64, self.n_u, "y"),
                                         _stream(stream)))
        return y

    def inverse_mass(self, r, x, stream=None):
        """x = M^-1 r (exact, cell by cell)."""
        import torch
        _check(self.lib.dgw_apply_inverse_mass(self.h, _ptr(r, torch.float64, self.n_u, "r"),
                                               _ptr(x, torch.float64, self.n_u, "x"), _stream(stream)))
        return x

    def set_enrichment_switch(self, yplus_off: float, stream=None):
        """Switch the wall model off in wall columns whose wall-nearest cell has y+ < yplus_off."""
        _check(self.lib.dgw_set_enrichment_switch(self.h, ctypes.c_double(yplus_off), _stream(stream)))

    def enrichment_active(self, stream=None):
        """Per enriched cell: 1 if the wall model is switched on (numpy int32 array)."""
        import numpy as np
        out = np.zeros(max(self.n_e, 1), dtype=np.int32)
        cnt = ctypes.c_int()
        _check(self.lib.dgw_enrichment_active(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                              ctypes.byref(cnt), _stream(stream)))
        return out[: self.n_e]

    def mass(self, u, y, stream=None):
        _check(self.lib.dgw_apply_mass(self.h, self._prec(u), _ptr(u, None, self.n_u, "u"),
                                       _ptr(y, u.dtype, self.n_u, "y"), _stream(stream)))
        return y

    def helmholtz_solve(self, gamma, rhs, u, rtol=1e-10, max_iter=1000, restart=30, stream=None, check=True):
        """Solve gamma M u - F^nu(u) = rhs (u: initial guess in, solution out)."""
        import torch
        opts = HelmholtzOpts(rtol, max_iter, restart)
        info = SolveInfo()
        st = self.lib.dgw_helmholtz_solve(self.h, ctypes.c_double(gamma), _ptr(rhs, torch.float64, self.n_u, "rhs"),
                                          _ptr(u, torch.float64, self.n_u, "u"), ctypes.byref(opts),
                                          ctypes.byref(info), _stream(stream))
        if check:
            _check(st)
        return {"iterations": info.iterations, "rel_residual": info.rel_residual, "ms": info.ms, "status": st,
                "dof_applies": info.dof_applies}

    def pressure_solve(self, b, p, rtol=1e-10, max_iter=1000, mode=1, cheb_degree=5, stream=None, check=True):
        import torch
        opts = SolveOpts(rtol, max_iter, mode, cheb_degree)
        info = SolveInfo()
        st = self.lib.dgw_pressure_solve(self.h, _ptr(b, torch.float64, self.n_p, "b"),
                                         _ptr(p, torch.float64, self.n_p, "p"), ctypes.byref(opts),
                                         ctypes.byref(info), _stream(stream))
        if check:
            _check(st)
        return {"iterations": info.iterations, "rel_residual": info.rel_residual, "ms": info.ms, "status": st,
                "dof_applies": info.dof_applies}


def pressure_solve_batch(mesh, bs, ps, rtol=1e-10, max_iter=1000, cheb_degree=5, stream=None, check=True):
    """Mixed-precision solves of the right-hand sides bs (list of CUDA float64 tensors of n_p) into ps
    as one block (dgw_pressure_solve_batch). Returns one info dict per column."""
    import torch
    nc = len(bs)
    if nc != len(ps) or nc == 0:
        raise ValueError("bs and ps must be non-empty lists of equal length")
    B = (ctypes.c_void_p * nc)(*[_ptr(b, torch.float64, mesh.n_p, "b") for b in bs])
    P = (ctypes.c_void_p * nc)(*[_ptr(p, torch.float64, mesh.n_p, "p") for p in ps])
    opts = SolveOpts(rtol, max_iter, 1, cheb_degree)
    infos = (SolveInfo * nc)()
    st = mesh.lib.dgw_pressure_solve_batch(mesh.h, nc, B, P, ctypes.byref(opts), infos, _stream(stream))
    if check:
        _check(st)
    return [{"iterations": i.iterations, "rel_residual": i.rel_residual, "ms": i.ms, "status": st,
             "dof_applies": i.dof_applies} for i in infos]


def describe_solver(mesh, mode=1):
    """Multigrid hierarchy of `mode`: list of (cells, lmax of D^-1 A) per level, finest first."""
    lib = load()
    nl = ctypes.c_int()
    lm = (ctypes.c_double * 32)()
    cells = (ctypes.c_int * 32)()
    _check(lib.dgw_solver_describe(mesh.h, mode, ctypes.byref(nl), lm, cells, 32, None))
    return [(cells[i], lm[i]) for i in range(min(nl.value, 32))]


class Server:
    """Request loop: jobs (solves and applies on any channel mesh) admitted as worker slots and
    device memory free up; concurrent jobs overlap on the device."""

    def __init__(self, hbm_budget_bytes, max_inflight=4):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.dgw_server_create(int(hbm_budget_bytes), int(max_inflight), ctypes.byref(h)))
        self.h = h

    def submit(self, kind, params: MeshParams, inp, out, prec=DGW_FP64, rtol=1e-10, max_iter=500, mode=1,
               cheb_degree=5, aux=None):
        job = Job(kind, prec, params, ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                  ctypes.c_void_p(aux.data_ptr() if aux is not None else 0), SolveOpts(rtol, max_iter, mode, cheb_degree))
        t = ctypes.c_long()
        _check(self.lib.dgw_submit(self.h, ctypes.byref(job), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """None while pending, else dict(status, iterations, rel_residual, latency_ms)."""
        st, info, lat = ctypes.c_int(), SolveInfo(), ctypes.c_double()
        r = self.lib.dgw_poll(self.h, int(ticket), ctypes.byref(st), ctypes.byref(info), ctypes.byref(lat))
        if r == -5:
            return None
        _check(r)
        return {"status": st.value, "iterations": info.iterations, "rel_residual": info.rel_residual,
                "latency_ms": lat.value}

    def stats(self):
        a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(self.lib.dgw_server_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        return {"queued": a.value, "running": b.value, "meshes": c.value, "reserved_bytes": d.value}

    def close(self, timeout_ms=60000):
        if getattr(self, "h", None):
            _check(self.lib.dgw_server_destroy(self.h, int(timeout_ms)))
            self.h = None


def mesh_params(workload, n_layers=1, q_wall=8, wall_law=0, fp32=True) -> MeshParams:
    return MeshParams(workload.nx, workload.ny, workload.nz, workload.k, 1, q_wall, workload.geometry, wall_law, n_layers,
                      workload.lx, workload.ly, workload.lz, workload.gamma, workload.nu, workload.tau_w,
                      3 if fp32 else 1)


def counters():
    """(kernel launches, operator DoF applications) performed by the library so far."""
    lib = load()
    a, b = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    lib.dgw_counters(ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


class DualSplitting:
    """Time integrator of the dual-splitting scheme on a Mesh (dgw_ns_*): u0 is copied; velocity()
    and pressure() return copies of the current state as CUDA tensors."""

    def __init__(self, mesh: Mesh, u0, *, dt, cr=0.14, force=(0.0, 0.0, 0.0), rtol_pressure=1e-10,
                 rtol_projection=1e-10, rtol_viscous=1e-10, max_iter=2000, pressure_mode=1,
                 update_wall_model=False, high_order_pressure_bc=False, adaptive_dt=False, stream=None):
        import torch
        self.mesh, self.lib = mesh, mesh.lib
        self.params = NSParams(dt, cr, (ctypes.c_double * 3)(*force), rtol_pressure, rtol_projection, rtol_viscous,
                               max_iter, pressure_mode, 1 if update_wall_model else 0,
                               1 if high_order_pressure_bc else 0, 1 if adaptive_dt else 0)
        h = ctypes.c_void_p()
        _check(self.lib.dgw_ns_create(mesh.h, ctypes.byref(self.params), _ptr(u0, torch.float64, mesh.n_u, "u0"),
                                      _stream(stream), ctypes.byref(h)))
        self.h = h

    def step(self, stream=None) -> dict:
        info = NSStepInfo()
        _check(self.lib.dgw_ns_step(self.h, ctypes.byref(info), _stream(stream)))
        return {"pressure_iterations": info.pressure_iterations, "projection_iterations": info.projection_iterations,
                "viscous_iterations": info.viscous_iterations, "ms": info.ms, "dt": info.dt}

    def _state(self):
        u, p, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int()
        _check(self.lib.dgw_ns_state(self.h, ctypes.byref(u), ctypes.byref(p), ctypes.byref(n)))
        return u.value, p.value, n.value

    def velocity(self, stream=None):
        return self._copy_state(True, stream)

    def pressure(self, stream=None):
        return self._copy_state(False, stream)

    def _copy_state(self, vel, stream):
        import torch
        out = torch.empty(self.mesh.n_u if vel else self.mesh.n_p, dtype=torch.float64, device="cuda")
        ptr = ctypes.c_void_p(out.data_ptr())
        _check(self.lib.dgw_ns_copy_state(self.h, ptr if vel else None, None if vel else ptr, _stream(stream)))
        return out

    @property
    def steps(self) -> int:
        return self._state()[2]

    def close(self):
        if self.h:
            self.lib.dgw_ns_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_for(workload, **kw) -> Mesh:
    """Mesh of a workload preset (paper_1705_08813_gb300.inputs.Workload), channel or bump."""
    kw.setdefault("geometry", workload.geometry)
    return Mesh(workload.nx, workload.ny, workload.nz, workload.k, lx=workload.lx, ly=workload.ly,
                lz=workload.lz, gamma=workload.gamma, nu=workload.nu, tau_w=workload.tau_w, **kw)
