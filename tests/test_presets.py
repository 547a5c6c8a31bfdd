"""Table 1 presets: LBGK through the preset equals a textbook BGK scheme; RLBM and
MLBM parameters follow the table."""
import numpy as np
import pytest

import oracle
import workloads as w
from paper_1902_09813_gb300.presets import lattice_tau, relaxation_preset
from test_oracle_pins import _textbook_bgk_diffusion


def test_lbgk_preset_is_textbook_bgk():
    tau = 0.8
    a = (tau - 0.5) / 3.0
    base = w.gaussian_hill(n=20, sigma0=3.0, u=(0.0, 0.0), A0=(a, 0.0, a), nsteps=40)
    pre = relaxation_preset("lbgk", base.A0, base.dx, base.dt)
    p = base.replace(**pre)
    assert lattice_tau(p.A0, p.dx, p.dt) == pytest.approx(tau)
    lat = oracle.run(p)
    assert np.allclose(lat.phi(), _textbook_bgk_diffusion(p.phi0(), tau, p.nsteps), atol=1e-13, rtol=0)


def test_table1_values():
    A0, dx, dt = (0.1, 0.0, 0.1), 1.0, 1.0      # tau = 0.8
    assert relaxation_preset("rlbm", A0, dx, dt) == dict(k0=1.0, k2_mode="const", k2=1.0)
    m = relaxation_preset("mlbm", A0, dx, dt, Z=1e-4)
    assert m["k0"] == pytest.approx(1.0 / 0.8001) and m["k2"] == pytest.approx(1.0 / 0.8001)
    assert relaxation_preset("ob-trirt", A0, dx, dt)["k2_mode"] == "hbb"
    with pytest.raises(ValueError):
        relaxation_preset("mrt", A0, dx, dt)


@pytest.mark.parametrize("model,u0,key,tol", [
    ("lbgk", 0.01, "gre_table3_lbgk_u0.01", 0.08), ("lbgk", 0.1, "gre_table3_lbgk_u0.1", 0.08),
    ("lbgk", 1.0, "gre_table3_lbgk_u1.0", 0.08),
    ("rlbm", 0.01, "gre_table3_rlbm_u0.01", 0.05), ("rlbm", 0.1, "gre_table3_rlbm_u0.1", 0.05)])
def test_table3_comparison_models(model, u0, key, tol):
    """The comparison models of Table 3 through the Table 1 presets (same walled
    linear CDE as the OB-TriRT pins): GRE within a few percent of the print."""
    from conftest import cpu_threads, paper_value
    p = w.linear_cde(n=100, alpha=0.01, u=(u0, u0), c=5.0, t_end=1.0, walls=True)
    p = p.replace(**relaxation_preset(model, p.A0, p.dx, p.dt))
    lat = oracle.run(p, nthreads=cpu_threads())
    err = w.gre(lat.phi(), w.linear_cde_exact(p, p.nsteps * p.dt))
    assert err == pytest.approx(paper_value(key), rel=tol)
