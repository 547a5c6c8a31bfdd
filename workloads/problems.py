"""Problem descriptions for the nonlinear anisotropic convection-diffusion equation

    d_t phi + div B(phi) = div( A(phi) grad C(phi) ) + S(x, t)          (Eq. 1 / Eq. 29)

with the coefficient families used by the paper's tests (Sec. 4) and by the
synthetic workloads of this project:

    B(phi) = u phi + b2 (phi^q / q) (d_x, d_y)   (q = 2, d = (1, 1) unless stated)
    C(phi) = phi + c3 phi^3                      (paper: D(x,phi,t) = C(phi) I)
    A(phi) = (1 + a2 phi^2) A0,  A0 symmetric positive definite
    S(x,t) = 0 | const | exp(lam t) sum_pq alpha_pq X_p(k x) Y_q(k y)   (X,Y in {sin, cos})
           | rate phi (1 - phi^exp)              (reaction term of Eq. 67)

All quantities are physical; nodes are cell-centred, x_i = x0 + (i + 1/2) dx
(the half-way bounce-back analysis places the wall half a cell outside the
first node, Sec. 3, Eq. 49).  Everything random is drawn from a seeded numpy
Generator here and passed to both implementations as plain numbers/arrays.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import numpy as np

PERIODIC = 0
HBB = 1
_SIDES = ("x-", "x+", "y-", "y+")


@dataclass
class Source:
    kind: str = "none"            # "none" | "const" | "trig" | "field" | "reaction"
    const: float = 0.0            # const: S; reaction: the rate
    exp: float = 1.0              # reaction: S = const phi (1 - phi^exp)
    lam: float = 0.0              # time factor exp(lam * t)
    k: float = math.pi            # spatial wavenumber of the trig tables
    alpha: tuple = (0.0, 0.0, 0.0, 0.0)   # (ss, sc, cs, cc): X_p(kx) Y_q(ky)

    def value(self, x, y, t):
        """Pointwise S(x, y, t) (numpy broadcasting)."""
        if self.kind == "none":
            return np.zeros(np.broadcast(x, y).shape)
        if self.kind == "const":
            return np.full(np.broadcast(x, y).shape, self.const)
        sx, cx = np.sin(self.k * x), np.cos(self.k * x)
        sy, cy = np.sin(self.k * y), np.cos(self.k * y)
        a_ss, a_sc, a_cs, a_cc = self.alpha
        return math.exp(self.lam * t) * (a_ss * sx * sy + a_sc * sx * cy
                                         + a_cs * cx * sy + a_cc * cx * cy)


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    dx: float
    dt: float
    x0: float = 0.0
    y0: float = 0.0
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)   # x-, x+, y-, y+
    u: tuple = (0.0, 0.0)
    b2: float = 0.0
    b_dir: tuple = (1.0, 1.0)            # direction of the power-law flux term
    b_q: float = 2.0                     # its exponent
    c3: float = 0.0
    A0: tuple = (0.0, 0.0, 0.0)          # (xx, xy, yy)
    a2: float = 0.0
    k0: float = 1.0
    k2_mode: str = "hbb"                 # "hbb": Eq. 62 from k1_eff ; "const": k2 below
    k2: float = 1.0
    source: Source = field(default_factory=Source)
    wall: tuple = (0.0, 0.0, 0.0, 0.0)   # constant wall value per side
    wall_arrays: Optional[Sequence[Optional[np.ndarray]]] = None   # per-node values along a side
    wall_lam: float = 0.0                # wall values carry the factor exp(wall_lam t)
    wall_fn: Optional[Callable] = None   # (x, y, t) -> wall value, re-evaluated every step
    src_field: Optional[np.ndarray] = None    # source kind "field": S = exp(lam t) src_field
    A_field: Optional[tuple] = None           # per-node diffusion tensor (xx, xy, yy) arrays
    t0: float = 0.0
    nsteps: int = 0
    phi0_fn: Optional[Callable] = None   # phi0(X, Y) -> array
    phi0_array: Optional[np.ndarray] = None
    phi_ref: float = 0.0                 # shift for reduced-precision storage
    meta: dict = field(default_factory=dict)

    # -- geometry -------------------------------------------------------
    def coords(self):
        """Cell-centred node coordinates as (X, Y), each of shape (ny, nx)."""
        xs = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
        ys = self.y0 + (np.arange(self.ny) + 0.5) * self.dy
        return np.meshgrid(xs, ys)

    @property
    def dy(self):
        return self.dx

    @property
    def c(self):
        return self.dx / self.dt

    def phi0(self) -> np.ndarray:
        if self.phi0_array is not None:
            a = np.ascontiguousarray(self.phi0_array, dtype=np.float64)
            assert a.shape == (self.ny, self.nx)
            return a
        X, Y = self.coords()
        return np.ascontiguousarray(self.phi0_fn(X, Y), dtype=np.float64)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def lattice_speed(self, phi_max: float) -> float:
        """max |B'(phi)| dt/dx over |phi| <= phi_max (advective Courant number)."""
        ux, uy = self.u
        slope = abs(self.b2) * max(abs(self.b_dir[0]), abs(self.b_dir[1])) * phi_max ** (self.b_q - 1.0)
        return (max(abs(ux), abs(uy)) + slope) * self.dt / self.dx

    def wall_arrays_at(self, t: float):
        """Wall values along the four sides at time t from wall_fn (x-, x+: one
        per row at the row centres; y-, y+: one per column)."""
        xs = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
        ys = self.y0 + (np.arange(self.ny) + 0.5) * self.dx
        x1, y1 = self.x0 + self.nx * self.dx, self.y0 + self.ny * self.dx
        f = self.wall_fn
        return [np.asarray(f(np.full_like(ys, self.x0), ys, t), dtype=np.float64),
                np.asarray(f(np.full_like(ys, x1), ys, t), dtype=np.float64),
                np.asarray(f(xs, np.full_like(xs, self.y0), t), dtype=np.float64),
                np.asarray(f(xs, np.full_like(xs, y1), t), dtype=np.float64)]


def _rot_tensor(l1: float, l2: float, theta: float) -> tuple:
    """R(theta) diag(l1, l2) R(theta)^T as (xx, xy, yy)."""
    c, s = math.cos(theta), math.sin(theta)
    xx = l1 * c * c + l2 * s * s
    yy = l1 * s * s + l2 * c * c
    xy = (l1 - l2) * c * s
    return (xx, xy, yy)


# ---------------------------------------------------------------------------
# Workload constructors
# ---------------------------------------------------------------------------
def gaussian_hill(n: int = 64, sigma0: float = 4.0, u=(0.1, 0.05), A0=(0.01, 0.0, 0.01),
                  nsteps: int = 500, dx: float = 1.0, dt: float = 1.0,
                  k2_mode: str = "hbb", k2: float = 1.0, k0: float = 1.0) -> Problem:
    """Advected, anisotropically spreading Gaussian hill on a periodic square
    (Sec. 4.2.1, Eqs. 70-71).  Default: the 64x64 lattice-unit case, dx = dt = 1,
    u = (0.1, 0.05), A = 0.01 I, sigma0 = 4 cells, centre at the domain middle."""
    L = n * dx
    xc, yc = 0.5 * L, 0.5 * L

    def phi0(X, Y):
        return np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2.0 * sigma0 ** 2))

    return Problem(name=f"gaussian_hill_{n}", nx=n, ny=n, dx=dx, dt=dt, u=tuple(u),
                   A0=tuple(A0), k0=k0, k2_mode=k2_mode, k2=k2, nsteps=nsteps, phi0_fn=phi0,
                   meta=dict(sigma0=sigma0, centre=(xc, yc), L=L))


def mms_sinsin(n: int = 64, kappa: float = 4.0, theta: float = math.pi / 6,
               eig=(0.05, 0.01), u=(0.05, 0.02), t_end: float = 0.1,
               nsteps: Optional[int] = None, k2_mode: str = "hbb", k2: float = 1.0) -> Problem:
    """Manufactured solution phi* = exp(-t) sin(pi x) sin(pi y) on the unit square
    with half-way bounce-back Dirichlet walls phi_w = 0 and the matching source.
    Diffusive scaling: dx = 1/n, dt = kappa dx^2 (so A dt/dx^2 = kappa A)."""
    A0 = _rot_tensor(eig[0], eig[1], theta)
    dx = 1.0 / n
    dt = kappa * dx * dx
    ux, uy = u
    axx, axy, ayy = A0
    pi = math.pi
    # S = phi_t + div(u phi) - div(A grad phi) for the manufactured phi*
    src = Source(kind="trig", lam=-1.0, k=pi,
                 alpha=(-1.0 + pi * pi * (axx + ayy),  # sin x sin y
                        pi * uy,                       # sin x cos y
                        pi * ux,                       # cos x sin y
                        -2.0 * pi * pi * axy))         # cos x cos y
    if nsteps is None:
        nsteps = int(round(t_end / dt))

    def phi0(X, Y):
        return np.sin(pi * X) * np.sin(pi * Y)

    return Problem(name=f"mms_sinsin_{n}", nx=n, ny=n, dx=dx, dt=dt,
                   bc=(HBB, HBB, HBB, HBB), u=tuple(u), A0=A0, k2_mode=k2_mode, k2=k2,
                   source=src, wall=(0.0, 0.0, 0.0, 0.0), nsteps=nsteps, phi0_fn=phi0,
                   meta=dict(kappa=kappa, t_end=nsteps * dt))


def nonlinear_modes(n: int = 8192, seed: int = 0, nmodes: int = 16, kmax: int = 8,
                    u=(0.1, 0.05), eig=(0.04, 0.008), theta: float = math.pi / 4,
                    b2: float = 1.0, a2: float = 1.0, nsteps: int = 1000,
                    courant: float = 0.25) -> Problem:
    """Nonlinear anisotropic CDE on a periodic n x n lattice (dx = 1):
    B = u phi + (phi^2/2)(1,1), C = phi, A = (1 + phi^2) A0 with A0 of eigenvalues
    (0.04, 0.008) at angle pi/4; phi0 = a sum of `nmodes` seeded Fourier modes with
    integer wavenumbers in 1..kmax and amplitudes U(-0.5, 0.5).  The time step keeps
    the advective Courant number max|B'(phi0)| dt/dx at `courant` (or dt = 1)."""
    rng = np.random.default_rng(seed)
    kx = rng.integers(1, kmax + 1, size=nmodes) * rng.choice([-1, 1], size=nmodes)
    ky = rng.integers(1, kmax + 1, size=nmodes) * rng.choice([-1, 1], size=nmodes)
    amp = rng.uniform(-0.5, 0.5, size=nmodes)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=nmodes)
    L = float(n)

    def phi0(X, Y):
        out = np.zeros_like(X)
        for m in range(nmodes):
            out += amp[m] * np.cos(2.0 * math.pi * (kx[m] * X + ky[m] * Y) / L + phase[m])
        return out

    phi_bound = float(np.abs(amp).sum())
    speed = max(abs(u[0]), abs(u[1])) + abs(b2) * phi_bound
    dt = min(1.0, courant / speed)
    A0 = _rot_tensor(eig[0], eig[1], theta)
    return Problem(name=f"nonlinear_modes_{n}", nx=n, ny=n, dx=1.0, dt=dt, u=tuple(u), b2=b2,
                   A0=A0, a2=a2, nsteps=nsteps, phi0_fn=phi0,
                   meta=dict(seed=seed, kx=kx, ky=ky, amp=amp, phase=phase, phi_bound=phi_bound))


def steady_diffusion(n: int = 5, k1: float = 1.25, alpha: float = 0.1, ux: float = 0.1,
                     phi_bottom: float = 0.0, phi_top: float = 1.0, L: float = 1.0,
                     k2_mode: str = "hbb", k2: float = 1.0, k0: float = 1.0,
                     nsteps: int = 20000) -> Problem:
    """Unidirectional steady diffusion with HBB walls at y = 0 and y = L, periodic
    in x (Sec. 3, Eqs. 31-36; Sec. 4.1.1): u = (ux, 0), constant source
    S = 2 alpha dphi / L^2, exact phi = phi_0 + dphi y (2 - y) for L = 1.
    dt follows from alpha = cs^2 (1/k1 - 1/2) dt (Eq. 30) with c = dx/dt."""
    dx = L / n
    # alpha = (dx^2 / (3 dt)) (1/k1 - 1/2)  ->  dt = dx^2 (1/k1 - 1/2) / (3 alpha)
    dt = dx * dx * (1.0 / k1 - 0.5) / (3.0 * alpha)
    dphi = phi_top - phi_bottom
    src = Source(kind="const", const=2.0 * alpha * dphi / (L * L))
    return Problem(name=f"steady_diffusion_{n}", nx=n, ny=n, dx=dx, dt=dt,
                   bc=(PERIODIC, PERIODIC, HBB, HBB), u=(ux, 0.0), A0=(alpha, 0.0, alpha),
                   k0=k0, k2_mode=k2_mode, k2=k2, source=src,
                   wall=(0.0, 0.0, phi_bottom, phi_top), nsteps=nsteps,
                   phi0_fn=lambda X, Y: np.full_like(X, phi_bottom),
                   meta=dict(k1=k1, alpha=alpha, dphi=dphi, phi_bottom=phi_bottom, L=L))


def linear_cde(n: int = 200, alpha: float = 0.01, u=(0.1, 0.1), c: float = 1.0,
               t_end: float = 3.0, L: float = 2.0, k2_mode: str = "hbb", k2: float = 1.0,
               walls: bool = False) -> Problem:
    """Linear isotropic CDE with a constant velocity on the square [0, L]^2
    (Sec. 4.1.2, Eqs. 65-66): phi* = exp((1 - 2 pi^2 alpha) t) sin(pi (x + y)),
    S = exp(lam t) [sin(pi(x+y)) + pi (ux + uy) cos(pi(x+y))].  Periodic, or with
    bounce-back walls that carry the exact solution (wall arrays x exp(lam t))."""
    dx = L / n
    dt = dx / c
    lam = 1.0 - 2.0 * math.pi ** 2 * alpha
    pu = math.pi * (u[0] + u[1])
    # sin(a+b) = sa cb + ca sb ; cos(a+b) = ca cb - sa sb
    src = Source(kind="trig", lam=lam, k=math.pi, alpha=(-pu, 1.0, 1.0, pu))
    kw = {}
    if walls:
        s = (np.arange(n) + 0.5) * dx
        kw = dict(bc=(HBB, HBB, HBB, HBB), wall_lam=lam,
                  wall_arrays=[np.sin(math.pi * (0.0 + s)), np.sin(math.pi * (L + s)),
                               np.sin(math.pi * (s + 0.0)), np.sin(math.pi * (s + L))])
    return Problem(name=f"linear_cde_{n}" + ("_walls" if walls else ""), nx=n, ny=n, dx=dx,
                   dt=dt, u=tuple(u), A0=(alpha, 0.0, alpha), k2_mode=k2_mode, k2=k2,
                   source=src, nsteps=int(round(t_end / dt)),
                   phi0_fn=lambda X, Y: np.sin(math.pi * (X + Y)),
                   meta=dict(alpha=alpha, lam=lam), **kw)


def burgers_fisher_solution(x, y, t, a: float, alpha: float, b: float, delta: float):
    """Travelling-wave solution of the Burgers-Fisher equation (Eq. 67, convection
    along x only, diffusion alpha in both directions):
        phi = [1/2 + 1/2 tanh(A (x + y - omega t))]^(1/delta),
        A = -a delta / (4 alpha (delta + 1)),
        omega = a / (delta + 1) + 2 b alpha (delta + 1) / a.
    Eq. 69 prints omega = (a^2 + 2 b alpha (delta + 1)) / (a (delta + 1)); the
    wave satisfies Eq. 67 only with (delta + 1)^2 in that numerator (checked by
    substitution), which is the omega above."""
    A = -a * delta / (4.0 * alpha * (delta + 1.0))
    om = a / (delta + 1.0) + 2.0 * b * alpha * (delta + 1.0) / a
    return (0.5 + 0.5 * np.tanh(A * (x + y - om * t))) ** (1.0 / delta)


def burgers_fisher(n: int = 120, a: float = 2.0, alpha: float = 0.05, b: float = 0.05,
                   delta: float = 1.5, c: float = 5.0, t_end: float = 1.0, k2_mode: str = "hbb",
                   k2: float = 1.0) -> Problem:
    """Burgers-Fisher equation (Sec. 4.1.3, Eq. 67) on [-1, 2]^2 with n x n nodes:
    B = a phi^(delta+1)/(delta+1) (1, 0) (the conservative form of a phi^delta d_x phi),
    A = alpha I, S = b phi (1 - phi^delta); bounce-back walls carrying the exact
    solution, re-evaluated at every step (wall_fn); phi0 the exact solution at t = 0."""
    dx = 3.0 / n
    dt = dx / c
    sol = lambda X, Y, t: burgers_fisher_solution(X, Y, t, a, alpha, b, delta)  # noqa: E731
    return Problem(name=f"burgers_fisher_{n}", nx=n, ny=n, dx=dx, dt=dt, x0=-1.0, y0=-1.0,
                   bc=(HBB, HBB, HBB, HBB), u=(0.0, 0.0), b2=a, b_dir=(1.0, 0.0), b_q=delta + 1.0,
                   A0=(alpha, 0.0, alpha), k2_mode=k2_mode, k2=k2,
                   source=Source(kind="reaction", const=b, exp=delta),
                   wall_fn=sol, nsteps=int(round(t_end / dt)),
                   phi0_fn=lambda X, Y: sol(X, Y, 0.0),
                   meta=dict(a=a, alpha=alpha, b=b, delta=delta))


def variable_tensor(n: int = 100, alpha: float = 1e-2, u=(0.1, 0.1), c: float = 1.0,
                    t_end: float = 3.0, walls: bool = True) -> Problem:
    """Anisotropic CDE with a variable diffusion tensor (Sec. 4.2.2, Eqs. 73-76) on
    the unit square: A = diag(2 - sin(2 pi x) sin(2 pi y), 1) alpha,
    phi* = exp((1 - 12 pi^2 alpha) t) sin(2 pi x) sin(2 pi y) and the source of
    Eq. 75 as a per-node field times exp(lam t).  Bounce-back walls with
    phi_w = 0 (the solution vanishes there), or periodic."""
    dx = 1.0 / n
    dt = dx / c
    lam = 1.0 - 12.0 * math.pi ** 2 * alpha
    xs = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xs, xs)
    s2x, s2y = np.sin(2 * math.pi * X), np.sin(2 * math.pi * Y)
    c2x, c2y = np.cos(2 * math.pi * X), np.cos(2 * math.pi * Y)
    field = (s2x * s2y + 4.0 * alpha * math.pi ** 2 * np.cos(4 * math.pi * X) * s2y ** 2
             + 2.0 * math.pi * (u[0] * c2x * s2y + u[1] * s2x * c2y))
    A_field = (alpha * (2.0 - s2x * s2y), np.zeros_like(X), np.full_like(X, alpha))
    bc = (HBB, HBB, HBB, HBB) if walls else (PERIODIC,) * 4
    return Problem(name=f"variable_tensor_{n}", nx=n, ny=n, dx=dx, dt=dt, bc=bc, u=tuple(u),
                   A0=(2.0 * alpha, 0.0, alpha), source=Source(kind="field", lam=lam),
                   src_field=field, A_field=A_field, nsteps=int(round(t_end / dt)),
                   phi0_fn=lambda X_, Y_: np.sin(2 * math.pi * X_) * np.sin(2 * math.pi * Y_),
                   meta=dict(alpha=alpha, lam=lam))


def batched_instances(count: int = 512, seed: int = 0, nmin: int = 32, nmax: int = 1024,
                      nsteps: int = 2000):
    """Independent instances of uneven size: side log-uniform in [nmin, nmax],
    A0 eigenvalues U(0.005, 0.1) at angle U(0, pi), |u| = U(0, 0.1) in a random
    direction (lattice units).  Even-indexed instances are periodic Gaussian hills
    (sigma0 = n/16, no source); odd ones are HBB-walled manufactured solutions with
    dt = dx^2 (so the lattice diffusion tensor equals A0)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        l1, l2 = rng.uniform(0.005, 0.1, size=2)
        th = rng.uniform(0.0, math.pi)
        speed = rng.uniform(0.0, 0.1)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        ul = (speed * math.cos(ang), speed * math.sin(ang))
        A_lat = _rot_tensor(l1, l2, th)
        if k % 2 == 0:
            p = gaussian_hill(n=n, sigma0=n / 16.0, u=ul, A0=A_lat, nsteps=nsteps)
        else:
            # physical units on the unit square: dx = 1/n, dt = dx^2, A = A_lat,
            # u = u_lat dx/dt = u_lat n
            p = mms_sinsin(n=n, kappa=1.0, theta=th, eig=(l1, l2),
                           u=(ul[0] * n, ul[1] * n), nsteps=nsteps)
        p.name = f"inst{k}_{p.name}"
        p.meta["index"] = k
        out.append(p)
    return out


def random_state_problem(nx: int, ny: int, seed: int = 0, bc=(PERIODIC,) * 4,
                         nonlinear: bool = True, source: str = "trig", flux_q: float = 2.0) -> Problem:
    """A generic seeded problem for parity tests: random coefficients within the
    stable range, a smooth random initial field, optional walls with random
    constant values and a trig, constant or reaction source; flux_q != 2 gives
    the power-law flux b2 (phi^q / q)(1, -1/2)."""
    rng = np.random.default_rng(seed)
    l1, l2 = rng.uniform(0.01, 0.08, size=2)
    th = rng.uniform(0.0, math.pi)
    A0 = _rot_tensor(l1, l2, th)
    u = tuple(rng.uniform(-0.08, 0.08, size=2))
    nm = 4
    kx = rng.integers(1, 3, size=nm)
    ky = rng.integers(1, 3, size=nm)
    amp = rng.uniform(-0.3, 0.3, size=nm)
    ph = rng.uniform(0, 2 * math.pi, size=nm)
    base = rng.uniform(0.5, 1.0)

    def phi0(X, Y):
        out = np.full_like(X, base)
        for m in range(nm):
            out += amp[m] * np.cos(2 * math.pi * (kx[m] * X / nx + ky[m] * Y / ny) + ph[m])
        return out

    if source == "trig":
        src = Source(kind="trig", lam=-0.01, k=2 * math.pi / max(nx, ny),
                     alpha=tuple(rng.uniform(-1e-3, 1e-3, size=4)))
    elif source == "const":
        src = Source(kind="const", const=float(rng.uniform(-1e-3, 1e-3)))
    elif source == "reaction":
        src = Source(kind="reaction", const=float(rng.uniform(0.01, 0.05)), exp=float(rng.uniform(1.0, 2.0)))
    else:
        src = Source()
    wall = tuple(float(v) for v in rng.uniform(0.2, 1.2, size=4))
    return Problem(name=f"random_{nx}x{ny}_s{seed}", nx=nx, ny=ny, dx=1.0, dt=1.0,
                   bc=tuple(bc), u=u, b2=(0.05 if nonlinear else 0.0),
                   c3=(0.02 if nonlinear else 0.0), A0=A0, a2=(0.3 if nonlinear else 0.0),
                   k0=float(rng.uniform(0.8, 1.2)), source=src, wall=wall,
                   b_q=float(flux_q), b_dir=((1.0, 1.0) if flux_q == 2.0 else (1.0, -0.5)),
                   nsteps=8, phi0_fn=phi0, phi_ref=base)
