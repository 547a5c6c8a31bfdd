"""Relaxation-parameter presets (Table 1): the LBGK, MLBM and RLBM models and the
optimal B-TriRT (OB-TriRT) choice as special cases of the three-block collision.

The first-order block always follows from the diffusion tensor (Eq. 30); the
presets fix k0 and k2 relative to it.  For an anisotropic tensor the relaxation
time tau is taken from the mean lattice diffusivity, tr(A dt/dx^2)/2.
"""
from __future__ import annotations


def lattice_tau(A0, dx: float, dt: float) -> float:
    """tau with (tau - 1/2)/3 = tr(A)/2 dt/dx^2 (Eq. 30 with K1 = I/tau)."""
    alpha = 0.5 * (A0[0] + A0[2]) * dt / (dx * dx)
    return 3.0 * alpha + 0.5


def relaxation_preset(model: str, A0, dx: float, dt: float, Z: float = 1e-4) -> dict:
    """Return {k0, k2_mode, k2} for model in {"lbgk", "mlbm", "rlbm", "ob-trirt"}.

    LBGK:     k0 = k1 = k2 = 1/tau
    MLBM:     k0 = k2 = 1/tau, k1 = 1/tau_Z with tau_Z = tau - Z; the diffusion
              tensor fixes k1, so tau = tau_Z + Z here
    RLBM:     k0 = 1, k1 = 1/tau, k2 = 1
    OB-TriRT: k0 = 1, k2 from the half-way bounce-back relation (Eq. 62)
    """
    m = model.lower()
    tau = lattice_tau(A0, dx, dt)
    if m == "lbgk":
        return dict(k0=1.0 / tau, k2_mode="const", k2=1.0 / tau)
    if m == "mlbm":
        t = tau + Z
        return dict(k0=1.0 / t, k2_mode="const", k2=1.0 / t)
    if m == "rlbm":
        return dict(k0=1.0, k2_mode="const", k2=1.0)
    if m in ("ob-trirt", "obtrirt", "btrirt"):
        return dict(k0=1.0, k2_mode="hbb", k2=1.0)
    raise ValueError(f"unknown model {model!r}")
