"""Burgers-Fisher equation (Sec. 4.1.3, Eqs. 67-69): the closed form, and the
oracle's power-law flux and phi-dependent reaction source pinned to the
printed errors of Tables 4 and 5 and to second-order convergence (Fig. 8).

Readings (also listed with the design notes):
- Eq. 67 convects along x only, with diffusion alpha in x and y; the travelling
  wave of Eq. 68 in x + y then needs omega = a/(delta+1) + 2 b alpha (delta+1)/a,
  i.e. (delta+1)^2 where Eq. 69 prints (delta+1) (checked below by substitution).
- "Proper" boundary conditions: bounce-back walls carrying the exact solution at
  every step; the tables are at t = 1 (as Fig. 8).
- Powers with non-integer exponents are taken of max(phi, 0).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads, paper_value
from paper_1902_09813_gb300.presets import relaxation_preset


def _residual(a, alpha, b, delta, omega_fn):
    """max |Eq. 67 residual| of the travelling wave by central differences."""
    A = -a * delta / (4.0 * alpha * (delta + 1.0))
    om = omega_fn(a, alpha, b, delta)

    def phi(x, y, t):
        return (0.5 + 0.5 * np.tanh(A * (x + y - om * t))) ** (1.0 / delta)

    rng = np.random.default_rng(0)
    x, y, t = rng.uniform(-0.5, 0.5, 50), rng.uniform(-0.5, 0.5, 50), rng.uniform(0.0, 0.5, 50)
    # keep the points on the front (values away from 0 and 1)
    s = x + y - om * t
    x = x - s + rng.uniform(-0.5, 0.5, 50) / abs(A)
    h = 1e-4 / max(1.0, abs(A))
    f = phi(x, y, t)
    ft = (phi(x, y, t + h) - phi(x, y, t - h)) / (2 * h)
    fx = (phi(x + h, y, t) - phi(x - h, y, t)) / (2 * h)
    fxx = (phi(x + h, y, t) - 2 * f + phi(x - h, y, t)) / (h * h)
    fyy = (phi(x, y + h, t) - 2 * f + phi(x, y - h, t)) / (h * h)
    r = ft + a * f ** delta * fx - alpha * (fxx + fyy) - b * f * (1 - f ** delta)
    scale = np.abs(ft).max()
    return float(np.abs(r).max() / scale)


def test_closed_form_solves_eq67_with_corrected_speed():
    corrected = lambda a, al, b, d: a / (d + 1) + 2 * b * al * (d + 1) / a  # noqa: E731
    printed = lambda a, al, b, d: (a * a + 2 * b * al * (d + 1)) / (a * (d + 1))  # noqa: E731
    for a, al, b, d in ((2.0, 0.01, 0.05, 1.5), (1.0, 0.05, 0.3, 2.0), (3.0, 0.1, 1.0, 1.0)):
        rc, rp = _residual(a, al, b, d, corrected), _residual(a, al, b, d, printed)
        assert rc < 1e-5 and rp > 30 * rc, (rc, rp)
    # the workloads closed form is that wave
    p = w.burgers_fisher(n=30, a=2.0, alpha=0.01)
    X, Y = p.coords()
    A = -2.0 * 1.5 / (4 * 0.01 * 2.5)
    om = corrected(2.0, 0.01, 0.05, 1.5)
    ref = (0.5 + 0.5 * np.tanh(A * (X + Y - om * 0.3))) ** (1 / 1.5)
    assert np.allclose(w.burgers_fisher_exact(p, 0.3), ref, rtol=1e-14, atol=0)


def test_power_law_flux_and_reaction_terms():
    p = w.burgers_fisher(n=10, a=2.0, alpha=0.05)
    for phi in (0.0, 0.3, 0.9, 1.0):
        B = oracle.B(p, phi)
        assert B[0] == pytest.approx(2.0 * phi ** 2.5 / 2.5, rel=1e-14, abs=1e-300)
        assert B[1] == 0.0
        assert oracle.source(p, 0.1, 0.2, 0.5, phi) == pytest.approx(0.05 * phi * (1 - phi ** 1.5), abs=1e-16)
    # a small undershoot below zero stays finite
    assert math.isfinite(oracle.source(p, 0.0, 0.0, 0.0, -1e-6))
    assert all(math.isfinite(v) for v in oracle.B(p, -1e-6))


def _gre(p):
    lat = oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(p.nsteps)
    return w.gre(lat.phi(), w.burgers_fisher_exact(p, p.nsteps * p.dt))


TABLES = [
    # (model, a, alpha, key, rel tol)
    ("ob-trirt", 1.0, 0.05, "gre_table4_obtrirt_a1", 0.06),
    ("ob-trirt", 2.0, 0.05, "gre_table4_obtrirt_a2", 0.06),
    ("ob-trirt", 3.0, 0.05, "gre_table4_obtrirt_a3", 0.06),
    ("lbgk", 1.0, 0.05, "gre_table4_lbgk_a1", 0.06),
    ("lbgk", 2.0, 0.05, "gre_table4_lbgk_a2", 0.06),
    ("lbgk", 3.0, 0.05, "gre_table4_lbgk_a3", 0.06),
    ("mlbm", 1.0, 0.05, "gre_table4_mlbm_a1", 0.06),
    ("mlbm", 2.0, 0.05, "gre_table4_mlbm_a2", 0.06),
    ("rlbm", 1.0, 0.05, "gre_table4_rlbm_a1", 0.06),
    ("rlbm", 2.0, 0.05, "gre_table4_rlbm_a2", 0.06),
    ("rlbm", 3.0, 0.05, "gre_table4_rlbm_a3", 0.07),
    ("ob-trirt", 2.0, 0.005, "gre_table5_obtrirt_al0.005", 0.06),
    ("ob-trirt", 2.0, 0.1, "gre_table5_obtrirt_al0.1", 0.06),
    ("ob-trirt", 2.0, 0.5, "gre_table5_obtrirt_al0.5", 0.06),
    ("lbgk", 2.0, 0.1, "gre_table5_lbgk_al0.1", 0.06),
    ("mlbm", 2.0, 0.1, "gre_table5_mlbm_al0.1", 0.06),
    ("rlbm", 2.0, 0.005, "gre_table5_rlbm_al0.005", 0.06),
    ("rlbm", 2.0, 0.1, "gre_table5_rlbm_al0.1", 0.06),
    ("rlbm", 2.0, 0.5, "gre_table5_rlbm_al0.5", 0.06),
]


@pytest.mark.parametrize("model,a,alpha,key,tol", TABLES, ids=[t[3] for t in TABLES])
def test_tables_4_5(model, a, alpha, key, tol):
    """dx = 1/40 on [-1, 2]^2 (120^2 nodes), c = 5, b = 0.05, delta = 1.5, t = 1."""
    p = w.burgers_fisher(n=120, a=a, alpha=alpha, t_end=1.0)
    p = p.replace(**relaxation_preset(model, p.A0, p.dx, p.dt))
    assert _gre(p) == pytest.approx(paper_value(key), rel=tol)


def test_second_order_convergence():
    """Fig. 8 setting (a = 2, alpha = 0.01, t = 1), dx = 1/20, 1/40, 1/80."""
    errs = [_gre(w.burgers_fisher(n=n, a=2.0, alpha=0.01, t_end=1.0)) for n in (60, 120, 240)]
    for coarse, fine in zip(errs, errs[1:]):
        assert 3.5 < coarse / fine < 6.0, errs
