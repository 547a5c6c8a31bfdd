"""Closed-form solutions of the PDE (not of the lattice scheme) used as references.

Each function evaluates the analytic phi*(x, t) at the cell-centred nodes of a
:class:`~workloads.problems.Problem`.
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_hill_exact(p, t: float, images: int = 1) -> np.ndarray:
    """Advected anisotropic Gaussian hill (Eq. 71) normalised to peak 1 at t = 0:
    phi* = sigma0^2 / sqrt(det S_t) exp(-r^T S_t^{-1} r / 2), S_t = sigma0^2 I + 2 A t,
    r = x - x_c - u t, summed over periodic images of the domain."""
    s0 = p.meta["sigma0"]
    xc, yc = p.meta["centre"]
    L = p.nx * p.dx
    axx, axy, ayy = p.A0
    sxx = s0 * s0 + 2.0 * axx * t
    syy = s0 * s0 + 2.0 * ayy * t
    sxy = 2.0 * axy * t
    det = sxx * syy - sxy * sxy
    ixx, iyy, ixy = syy / det, sxx / det, -sxy / det
    X, Y = p.coords()
    out = np.zeros_like(X)
    for kx in range(-images, images + 1):
        for ky in range(-images, images + 1):
            rx = X - xc - p.u[0] * t + kx * L
            ry = Y - yc - p.u[1] * t + ky * L
            out += np.exp(-0.5 * (ixx * rx * rx + 2.0 * ixy * rx * ry + iyy * ry * ry))
    return out * (s0 * s0 / math.sqrt(det))


def mms_sinsin_exact(p, t: float) -> np.ndarray:
    """phi* = exp(-t) sin(pi x) sin(pi y)."""
    X, Y = p.coords()
    return math.exp(-t) * np.sin(math.pi * X) * np.sin(math.pi * Y)


def linear_cde_exact(p, t: float) -> np.ndarray:
    """phi* = exp((1 - 2 pi^2 alpha) t) sin(pi (x + y))  (Eq. 66 with the exponent
    that the source term of Eq. 65 implies)."""
    X, Y = p.coords()
    return math.exp(p.meta["lam"] * t) * np.sin(math.pi * (X + Y))


def steady_diffusion_exact(p) -> np.ndarray:
    """phi = phi_0 + dphi y (2 - y) with y measured in units of L (Eq. 36)."""
    X, Y = p.coords()
    y = (Y - p.y0) / p.meta["L"]
    return p.meta["phi_bottom"] + p.meta["dphi"] * y * (2.0 - y)


def variable_tensor_exact(p, t: float) -> np.ndarray:
    """phi* = exp((1 - 12 pi^2 alpha) t) sin(2 pi x) sin(2 pi y) (Eq. 76)."""
    X, Y = p.coords()
    return math.exp(p.meta["lam"] * t) * np.sin(2 * math.pi * X) * np.sin(2 * math.pi * Y)


def burgers_fisher_exact(p, t: float) -> np.ndarray:
    """Eq. 68 (with the corrected wave speed, see burgers_fisher_solution)."""
    from .problems import burgers_fisher_solution
    X, Y = p.coords()
    m = p.meta
    return burgers_fisher_solution(X, Y, t, m["a"], m["alpha"], m["b"], m["delta"])
