"""Three-dimensional problem descriptions for the D3Q19 variant of the scheme.

Same equation and coefficient families as :mod:`workloads.problems` (Eq. 1):

    B(phi) = u phi + b2 (phi^q / q) d,   C(phi) = phi + c3 phi^3,
    A(phi) = (1 + a2 phi^2) A0,  A0 symmetric positive definite (xx, xy, xz, yy, yz, zz)
    S = 0 | const | exp(lam t) F(x) | rate phi (1 - phi^exp)

on an nx x ny x nz box of cell-centred nodes; sides x-, x+, y-, y+, z-, z+
are periodic or half-way bounce-back walls with a constant value each (times
exp(wall_lam t)).  Arrays are [nz][ny][nx] (x fastest).  Problem data only:
no lattice Boltzmann arithmetic lives here.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from .problems import HBB, PERIODIC, Source


@dataclass
class Problem3:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dt: float
    x0: float = 0.0
    y0: float = 0.0
    z0: float = 0.0
    bc: tuple = (PERIODIC,) * 6
    u: tuple = (0.0, 0.0, 0.0)
    b2: float = 0.0
    b_dir: tuple = (1.0, 1.0, 1.0)
    b_q: float = 2.0
    c3: float = 0.0
    A0: tuple = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)   # xx, xy, xz, yy, yz, zz
    a2: float = 0.0
    k0: float = 1.0
    k2_mode: str = "hbb"
    k2: float = 1.0
    source: Source = field(default_factory=Source)   # kinds none, const, field, reaction
    src_field: Optional[np.ndarray] = None           # [nz][ny][nx]
    wall: tuple = (0.0,) * 6
    wall_lam: float = 0.0
    t0: float = 0.0
    nsteps: int = 0
    phi0_fn: Optional[Callable] = None               # phi0(X, Y, Z)
    phi_ref: float = 0.0
    meta: dict = field(default_factory=dict)

    def coords(self):
        xs = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
        ys = self.y0 + (np.arange(self.ny) + 0.5) * self.dx
        zs = self.z0 + (np.arange(self.nz) + 0.5) * self.dx
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        return X, Y, Z

    @property
    def c(self):
        return self.dx / self.dt

    def phi0(self) -> np.ndarray:
        X, Y, Z = self.coords()
        return np.ascontiguousarray(self.phi0_fn(X, Y, Z), dtype=np.float64)

    def replace(self, **kw) -> "Problem3":
        return dataclasses.replace(self, **kw)


def rot_tensor3(eig, angles) -> tuple:
    """R diag(eig) R^T with R = Rz(a) Ry(b) Rx(c), as (xx, xy, xz, yy, yz, zz)."""
    a, b, c = angles
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(c), -math.sin(c)], [0, math.sin(c), math.cos(c)]])
    R = Rz @ Ry @ Rx
    M = R @ np.diag(eig) @ R.T
    return (M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2])


def gaussian_hill3(n: int = 32, sigma0: float = 3.0, u=(0.1, 0.05, -0.04),
                   A0=(0.02, 0.004, 0.0, 0.015, -0.003, 0.01), nsteps: int = 100,
                   dx: float = 1.0, dt: float = 1.0, k2_mode: str = "hbb", k2: float = 1.0,
                   k0: float = 1.0) -> Problem3:
    """Advected, anisotropically spreading Gaussian hill on a periodic cube (the
    three-dimensional form of Sec. 4.2.1): exact solution with covariance
    sigma0^2 I + 2 A t centred at x_c + u t."""
    L = n * dx
    xc = (0.5 * L,) * 3

    def phi0(X, Y, Z):
        return np.exp(-((X - xc[0]) ** 2 + (Y - xc[1]) ** 2 + (Z - xc[2]) ** 2) / (2.0 * sigma0 ** 2))

    return Problem3(name=f"gaussian_hill3_{n}", nx=n, ny=n, nz=n, dx=dx, dt=dt, u=tuple(u), A0=tuple(A0),
                    k0=k0, k2_mode=k2_mode, k2=k2, nsteps=nsteps, phi0_fn=phi0,
                    meta=dict(sigma0=sigma0, centre=xc, L=L))


def steady_diffusion3(n: int = 5, k1: float = 1.25, alpha: float = 0.1, u=(0.1, 0.0, 0.05),
                      phi_bottom: float = 0.0, phi_top: float = 1.0, L: float = 1.0,
                      k2_mode: str = "hbb", k2: float = 1.0, nsteps: int = 20000) -> Problem3:
    """Steady diffusion between bounce-back walls at y = 0 and y = L, periodic in
    x and z, constant source 2 alpha dphi / L^2: exact phi = phi_0 + dphi y (2 - y)
    for L = 1 (the three-dimensional form of Sec. 4.1.1)."""
    dx = L / n
    dt = dx * dx * (1.0 / k1 - 0.5) / (3.0 * alpha)
    dphi = phi_top - phi_bottom
    return Problem3(name=f"steady_diffusion3_{n}", nx=n, ny=n, nz=n, dx=dx, dt=dt,
                    bc=(PERIODIC, PERIODIC, HBB, HBB, PERIODIC, PERIODIC), u=tuple(u),
                    A0=(alpha, 0.0, 0.0, alpha, 0.0, alpha), k2_mode=k2_mode, k2=k2,
                    source=Source(kind="const", const=2.0 * alpha * dphi / (L * L)),
                    wall=(0.0, 0.0, phi_bottom, phi_top, 0.0, 0.0), nsteps=nsteps,
                    phi0_fn=lambda X, Y, Z: np.full_like(X, phi_bottom),
                    meta=dict(k1=k1, alpha=alpha, dphi=dphi, phi_bottom=phi_bottom, L=L))


def random_state_problem3(nx: int, ny: int, nz: int, seed: int = 0, bc=(PERIODIC,) * 6,
                          nonlinear: bool = True, source: str = "const", flux_q: float = 2.0) -> Problem3:
    """Seeded problem for parity tests: random stable coefficients, a smooth random
    initial field, random constant wall values, a constant, field or reaction source."""
    rng = np.random.default_rng(seed)
    eig = rng.uniform(0.01, 0.06, size=3)
    A0 = rot_tensor3(eig, rng.uniform(0.0, math.pi, size=3))
    u = tuple(rng.uniform(-0.06, 0.06, size=3))
    nm = 4
    k = rng.integers(1, 3, size=(nm, 3))
    amp = rng.uniform(-0.25, 0.25, size=nm)
    ph = rng.uniform(0, 2 * math.pi, size=nm)
    base = rng.uniform(0.5, 1.0)

    def phi0(X, Y, Z):
        out = np.full_like(X, base)
        for m in range(nm):
            out += amp[m] * np.cos(2 * math.pi * (k[m, 0] * X / nx + k[m, 1] * Y / ny + k[m, 2] * Z / nz) + ph[m])
        return out

    kw = {}
    if source == "const":
        src = Source(kind="const", const=float(rng.uniform(-1e-3, 1e-3)))
    elif source == "reaction":
        src = Source(kind="reaction", const=float(rng.uniform(0.01, 0.05)), exp=float(rng.uniform(1.0, 2.0)))
    elif source == "field":
        src = Source(kind="field", lam=-0.02)
        kw["src_field"] = rng.uniform(-1e-3, 1e-3, size=(nz, ny, nx))
    else:
        src = Source()
    wall = tuple(float(v) for v in rng.uniform(0.2, 1.2, size=6))
    return Problem3(name=f"random3_{nx}x{ny}x{nz}_s{seed}", nx=nx, ny=ny, nz=nz, dx=1.0, dt=1.0,
                    bc=tuple(bc), u=u, b2=(0.04 if nonlinear else 0.0), c3=(0.02 if nonlinear else 0.0),
                    b_q=float(flux_q), b_dir=((1.0, 1.0, 1.0) if flux_q == 2.0 else (1.0, -0.5, 0.25)),
                    A0=A0, a2=(0.3 if nonlinear else 0.0), k0=float(rng.uniform(0.8, 1.2)), source=src,
                    wall=wall, nsteps=8, phi0_fn=phi0, phi_ref=base, **kw)


def gaussian_hill3_exact(p: Problem3, t: float, images: int = 1) -> np.ndarray:
    """sigma0^3 / sqrt(det S_t) exp(-r^T S_t^{-1} r / 2), S_t = sigma0^2 I + 2 A t,
    r = x - x_c - u t, summed over the periodic images."""
    s0 = p.meta["sigma0"]
    xc = p.meta["centre"]
    L = p.nx * p.dx
    a = p.A0
    A = np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])
    S = s0 * s0 * np.eye(3) + 2.0 * A * t
    Si = np.linalg.inv(S)
    X, Y, Z = p.coords()
    out = np.zeros_like(X)
    rng = range(-images, images + 1)
    for kx in rng:
        for ky in rng:
            for kz in rng:
                r = (X - xc[0] - p.u[0] * t + kx * L, Y - xc[1] - p.u[1] * t + ky * L,
                     Z - xc[2] - p.u[2] * t + kz * L)
                q = sum(Si[i, j] * r[i] * r[j] for i in range(3) for j in range(3))
                out += np.exp(-0.5 * q)
    return out * (s0 ** 3 / math.sqrt(np.linalg.det(S)))


def steady_diffusion3_exact(p: Problem3) -> np.ndarray:
    X, Y, Z = p.coords()
    y = Y / p.meta["L"]
    return p.meta["phi_bottom"] + p.meta["dphi"] * y * (2.0 - y)
