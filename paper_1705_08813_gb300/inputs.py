"""Seeded synthetic inputs for the DG wall-model operators.

This module holds no arithmetic of the method (no basis, quadrature, wall law psi or weak
form): it only turns seeds into numbers. It is shared by the tests, the benchmark and the
smoke check, and is the one module both the CUDA path and the CPU oracle consume.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply
rounds; a double in [0, 1) takes the top 53 bits.

Velocity inputs take the shape of the paper's channel workload (Sec. 5.1): a turbulent mean
profile along x plus a divergence-free Fourier perturbation. The mean profile is Reichardt's
explicit law of the wall, u+ = ln(1 + 0.4 y+)/0.4 + 7.8 (1 - e^{-y+/11} - (y+/11) e^{-y+/3}),
a closed form that is independent of the enrichment function the operators evaluate. In wall
cells the standard coefficients carry only the perturbation and every enrichment coefficient is
u_tau e_x, so the enriched field there is u_tau * psi(y+) e_x exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n raw 64-bit outputs of SplitMix64 started from seed (stream selects a sub-sequence)."""
    base = np.uint64((seed * 0x100000001B3 + stream * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = base + _GOLD * np.arange(1, n + 1, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, stream: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the top 53 bits of SplitMix64 outputs."""
    u = (splitmix64(seed, n, stream) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


# --------------------------------------------------------------------------------------------
# Workload presets (synthetic stand-ins for the paper's channel and periodic-hill flows)
# --------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    k: int
    re_tau: float
    nu: float
    lx: float = 2.0 * math.pi
    ly: float = 2.0
    lz: float = math.pi
    gamma: float = 1.8
    geometry: int = 0
    seed: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def u_tau(self) -> float:
        return self.re_tau * self.nu

    @property
    def tau_w(self) -> float:
        return self.u_tau ** 2

    def mesh_kwargs(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, k=self.k, lx=self.lx, ly=self.ly,
                    lz=self.lz, gamma=self.gamma, nu=self.nu, tau_w=self.tau_w,
                    geometry=self.geometry)


def _reichardt(yp):
    return np.log1p(0.4 * yp) / 0.4 + 7.8 * (1.0 - np.exp(-yp / 11.0) - (yp / 11.0) * np.exp(-yp / 3.0))


def nu_for_unit_centreline(re_tau: float) -> float:
    """nu such that the mean profile reaches U = 1 at the centreline (delta = 1): u_tau =
    1 / u+(Re_tau), nu = u_tau / Re_tau (Reichardt profile)."""
    return 1.0 / (float(_reichardt(np.float64(re_tau))) * re_tau)


# Bump channel (stand-in for the periodic hill of Sec. 5.2): box 9 x 3.036 x 4.5 with a cos^2 bump of
# height 0.3 on the lower wall; Re_tau = 395 on the half height delta = 1.518 with centreline
# velocity 1, so nu = delta u_tau / Re_tau.
BUMP_DELTA = 0.5 * 3.036


def bump_workload(name: str, nx: int, ny: int, nz: int, k: int, seed: int, re_tau: float = 395.0) -> Workload:
    return Workload(name, nx, ny, nz, k, re_tau, BUMP_DELTA * nu_for_unit_centreline(re_tau),
                    lx=9.0, ly=3.036, lz=4.5, geometry=1, seed=seed)


WORKLOADS = {
    "channel_q2_8x8x8": Workload("channel_q2_8x8x8", 8, 8, 8, 2, 180.0, 1.0 / 3250.0, seed=1),
    "channel_q4_32x24x24": Workload("channel_q4_32x24x24", 32, 24, 24, 4, 590.0, 1.0 / 12000.0, seed=2),
    "channel_q3_64x32x32": Workload("channel_q3_64x32x32", 64, 32, 32, 3, 950.0,
                                    nu_for_unit_centreline(950.0), seed=3),
    "bump_q4_48x32x24": bump_workload("bump_q4_48x32x24", 48, 32, 24, 4, seed=4),
}


# --------------------------------------------------------------------------------------------
# Fields
# --------------------------------------------------------------------------------------------

def _modes():
    out = []
    for l in range(1, 5):
        for m in range(-4, 5):
            for n in range(-4, 5):
                if m * m + n * n + l * l <= 16:
                    out.append((m, n, l))
    return out


def _unique_axes(nodes: np.ndarray, nx: int, ny: int, nz: int, k: int):
    """1-D node coordinate arrays of a tensor-product channel mesh, from nodal positions in the
    canonical layout [cell (x fastest, then y, then z)][lz][ly][lx]."""
    n1 = k + 1
    X = nodes.reshape(nz, ny, nx, n1, n1, n1, 3)
    xs = X[0, 0, :, 0, 0, :, 0].reshape(-1)      # (nx, lx)
    ys = X[0, :, 0, 0, :, 0, 1].reshape(-1)      # (ny, ly)
    zs = X[:, 0, 0, :, 0, 0, 2].reshape(-1)      # (nz, lz)
    return xs, ys, zs


def _perturbation_grid(xs, ys, zs, w: Workload):
    """Divergence-free u' = curl A on the tensor grid (xs, ys, zs); A_i = W(y) sum_modes
    a sin(l pi (y+1)/2) cos(2 pi m x/Lx + 2 pi n z/Lz + phi); W = (1-y^2)^2. Returns (3, Nz, Ny, Nx)."""
    modes = _modes()
    nm = len(modes)
    a = uniform(w.seed, 3 * nm, -1.0, 1.0, stream=11).reshape(3, nm)
    ph = uniform(w.seed, 3 * nm, 0.0, 2.0 * math.pi, stream=12).reshape(3, nm)
    half = 0.5 * w.ly
    yy = ys / half                                  # walls at +-1
    W = (1.0 - yy ** 2) ** 2
    dW = -4.0 * yy * (1.0 - yy ** 2) / half
    eta = 0.5 * math.pi * (yy + 1.0)
    deta = 0.5 * math.pi / half
    Ex = np.exp(1j * 2.0 * math.pi * np.outer(np.arange(-4, 5), xs) / w.lx)   # (9, Nx)
    Gz = np.exp(1j * 2.0 * math.pi * np.outer(np.arange(-4, 5), zs) / w.lz)   # (9, Nz)

    def quantity(comp, deriv):
        C = np.zeros((9, 9, 4), dtype=np.complex128)
        Cy = np.zeros((9, 9, 4), dtype=np.complex128)
        for t, (m, n, l) in enumerate(modes):
            c = a[comp, t] * np.exp(1j * ph[comp, t])
            if deriv == "x":
                c = c * 1j * 2.0 * math.pi * m / w.lx
            elif deriv == "z":
                c = c * 1j * 2.0 * math.pi * n / w.lz
            if deriv == "y":
                Cy[m + 4, n + 4, l - 1] += c
            else:
                C[m + 4, n + 4, l - 1] += c
        ls = np.arange(1, 5)
        if deriv == "y":
            Y = (dW[:, None] * np.sin(np.outer(eta, ls)) +
                 W[:, None] * ls[None, :] * deta * np.cos(np.outer(eta, ls)))
            T = np.einsum("mnl,yl->ymn", Cy, Y)
        else:
            Y = W[:, None] * np.sin(np.outer(eta, ls))
            T = np.einsum("mnl,yl->ymn", C, Y)
        U = np.einsum("ymn,nz->zym", T, Gz)
        return np.real(np.einsum("zym,mx->zyx", U, Ex))

    ux = quantity(2, "y") - quantity(1, "z")
    uy = quantity(0, "z") - quantity(2, "x")
    uz = quantity(1, "x") - quantity(0, "y")
    return np.stack([ux, uy, uz])


def velocity_field(nodes: np.ndarray, n_e: int, w: Workload, n_layers: int = 1,
                   amplitude: float = 0.1, nef: int = 8) -> np.ndarray:
    """Velocity DoF vector [cell][3][(k+1)^3] followed by [enriched cell][3][nef] for a channel
    workload: mean profile + perturbation in non-wall cells, perturbation only in wall cells
    plus enrichment coefficients u_tau e_x (nef = 8 trilinear weights, 1 a constant weight).
    Perturbation scaled to amplitude * U_bulk."""
    nx, ny, nz, k = w.nx, w.ny, w.nz, w.k
    n1 = k + 1
    xs, ys, zs = _unique_axes(nodes, nx, ny, nz, k)
    half = 0.5 * w.ly
    ydist = half - np.abs(ys)
    U = w.u_tau * _reichardt(ydist * w.u_tau / w.nu)               # (Ny,)
    # bulk velocity: mean of U over the channel height (trapezoid on a fine grid)
    yf = np.linspace(0.0, half, 20001)
    uf = w.u_tau * _reichardt(yf * w.u_tau / w.nu)
    ubulk = float(np.sum(0.5 * (uf[1:] + uf[:-1]) * np.diff(yf)) / half)
    up = _perturbation_grid(xs, ys, zs, w)                         # (3, Nz, Ny, Nx)
    scale = amplitude * ubulk / max(np.sqrt((up ** 2).sum(axis=0)).max(), 1e-300)
    up *= scale
    # grid -> canonical layout [cz][cy][cx][comp][lz][ly][lx]
    g = up.reshape(3, nz, n1, ny, n1, nx, n1)                      # comp, cz, lz, cy, ly, cx, lx
    std = np.transpose(g, (1, 3, 5, 0, 2, 4, 6)).copy()            # cz, cy, cx, comp, lz, ly, lx
    Ucell = U.reshape(ny, n1)                                       # cy, ly
    wall_row = np.zeros(ny, dtype=bool)
    if n_layers > 0:
        wall_row[:n_layers] = True
        wall_row[ny - n_layers:] = True
    mean = np.where(wall_row[:, None], 0.0, Ucell)                 # cy, ly
    std[:, :, :, 0, :, :, :] += mean[None, :, None, None, :, None]
    u = np.zeros(3 * nx * ny * nz * n1 ** 3 + 3 * nef * n_e)
    u[: std.size] = std.reshape(-1)
    enr = np.zeros((n_e, 3, nef))
    enr[:, 0, :] = w.u_tau
    u[std.size:] = enr.reshape(-1)
    return u


def _bump_wall(x: np.ndarray, lx: float) -> np.ndarray:
    s = x - 0.5 * lx
    return np.where(np.abs(s) < 1.0, 0.3 * np.cos(0.5 * math.pi * s) ** 2, 0.0)


def bump_velocity_field(nodes: np.ndarray, n_e: int, w: Workload, n_layers: int = 1,
                        amplitude: float = 0.1, nef: int = 8) -> np.ndarray:
    """Velocity DoF vector for a bump workload: the mean profile along x in the vertical distance to
    the nearer wall, plus a seeded perturbation uniform in [-1, 1] * amplitude * U_c (U_c the
    largest mean nodal value) in every component of every node; wall cells carry the perturbation
    only, with enrichment coefficients u_tau e_x."""
    nx, ny, nz, k = w.nx, w.ny, w.nz, w.k
    n3 = (k + 1) ** 3
    X = nodes.reshape(nz, ny, nx, n3, 3)
    yd = np.maximum(np.minimum(X[..., 1] - _bump_wall(X[..., 0], w.lx), w.ly - X[..., 1]), 0.0)
    U = w.u_tau * _reichardt(yd * w.u_tau / w.nu)                 # (nz, ny, nx, n3)
    wall_row = np.zeros(ny, dtype=bool)
    if n_layers > 0:
        wall_row[:n_layers] = True
        wall_row[ny - n_layers:] = True
    U = np.where(wall_row[None, :, None, None], 0.0, U)
    uc = max(float(U.max()), w.u_tau)
    pert = uniform(w.seed, 3 * U.size, -1.0, 1.0, stream=31).reshape(nz, ny, nx, 3, n3) * amplitude * uc
    std = pert.copy()
    std[:, :, :, 0, :] += U
    u = np.zeros(std.size + 3 * nef * n_e)
    u[: std.size] = std.reshape(-1)
    enr = np.zeros((n_e, 3, nef))
    enr[:, 0, :] = w.u_tau
    u[std.size:] = enr.reshape(-1)
    return u


def workload_velocity(nodes: np.ndarray, n_e: int, w: Workload, n_layers: int = 1, nef: int = 8) -> np.ndarray:
    """Velocity input of a workload of either geometry (nef enrichment coefficients per component)."""
    if w.geometry == 1:
        return bump_velocity_field(nodes, n_e, w, n_layers=n_layers, nef=nef)
    return velocity_field(nodes, n_e, w, n_layers=n_layers, nef=nef)


def pressure_rhs(n_p: int, seed: int) -> np.ndarray:
    """Seeded right-hand side uniform in [-1, 1] per DoF, minus its mean."""
    b = uniform(seed, n_p, -1.0, 1.0, stream=21)
    return b - b.mean()


def pressure_field(n_p: int, seed: int) -> np.ndarray:
    """Seeded DoF vector uniform in [-1, 1] (input of a single Laplace apply)."""
    return uniform(seed, n_p, -1.0, 1.0, stream=22)
