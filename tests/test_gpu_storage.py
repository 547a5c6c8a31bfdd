"""Reduced-precision population storage under FP32 compute.

Two stored forms: deviations from w_i phi_ref (one reference per lattice) and
deviations from w_i phi(x) of the node that wrote the population (local shift).
Checked here: FP32 storage with the local shift against the FP64 oracle within
the FP32 tolerance; the discretisation error against the closed-form solutions
(Gaussian hill, manufactured solution) within 1 % of the oracle's own, except
BF16 on the 128^2 manufactured solution, whose measured miss is pinned; the
local shift never less accurate than the reference shift; TMA-staged and plain
kernels, and checkpoint/resume, bitwise equal."""
import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _lattice(p, storage, shift, **kw):
    from paper_1902_09813_gb300 import Lattice
    return Lattice.from_problem(p, compute="f32", storage=storage, shift=shift, **kw)


def _oracle_phi(p, nsteps):
    return oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(nsteps).phi()


@pytest.mark.parametrize("case", [(37, 29, (0, 0, 0, 0), True, "trig"), (37, 29, (1, 1, 1, 1), True, "trig"),
                                  (70, 65, (0, 0, 1, 1), True, "const"), (96, 40, (1, 1, 1, 1), False, "trig"),
                                  (3, 3, (1, 1, 1, 1), True, "const"), (5, 97, (1, 1, 0, 0), True, "trig")],
                         ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_local_shift_fp32_storage_matches_oracle(case):
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=11 * nx + ny, bc=bc, nonlinear=nonlin, source=src)
    steps = 10
    lat = _lattice(p, "f32", "local")
    lat.init(p.phi0(), t0=p.t0).step(steps)
    o = oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(steps)
    assert _rel(lat.phi_host(), o.phi()) <= TOL32
    # post-collision populations (the oracle's of its next step; read_f undoes the local shift)
    o.step(1)
    assert _rel(lat.read_f(), o.fpost) <= TOL32
    assert lat.check() == 0


CLOSED = {
    "hill64": (lambda: w.gaussian_hill(), lambda p: w.gaussian_hill_exact(p, p.nsteps * p.dt)),
    "mms64": (lambda: w.mms_sinsin(n=64), lambda p: w.mms_sinsin_exact(p, p.t0 + p.nsteps * p.dt)),
    "mms128": (lambda: w.mms_sinsin(n=128), lambda p: w.mms_sinsin_exact(p, p.t0 + p.nsteps * p.dt)),
}
# The reduced-precision bar: the local shift's GRE against the closed form within
# 1 % of the oracle's.  BF16 (8 significant bits) misses it on the 128^2
# manufactured solution (measured +22.7 %); that case is pinned separately below
# as a regression of the measured miss, not as a bar.
BAR = 0.01
MISSED = {("mms128", "bf16")}


def _gre_pair(name, storage):
    make, exact = CLOSED[name]
    p = make()
    ex = exact(p)
    phi_o = _oracle_phi(p, p.nsteps)
    g0 = w.gre(phi_o, ex)
    phi_ref = float(p.phi0().mean())
    res = {}
    for shift in ("ref", "local"):
        lat = _lattice(p, storage, shift, phi_ref=phi_ref)
        lat.init(p.phi0(), t0=p.t0).step(p.nsteps)
        got = lat.phi_host()
        res[shift] = (w.gre(got, ex), _rel(got, phi_o))
    return g0, res


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("name", list(CLOSED))
def test_storage_discretisation_error_vs_closed_form(name, storage):
    g0, res = _gre_pair(name, storage)
    g_loc, e_loc = res["local"]
    if (name, storage) not in MISSED:
        assert abs(g_loc - g0) <= BAR * g0, (g0, res)
    # the local shift is never the less accurate form (up to FP32 arithmetic noise)
    assert e_loc <= res["ref"][1] * 1.05 + 1e-6, res


def test_bf16_local_shift_misses_bar_on_mms128_regression():
    """BF16 storage with the local shift on the 128^2 manufactured solution: the
    GRE is 22.7 % above the oracle's, outside the 1 % bar.  Pinned as measured."""
    g0, res = _gre_pair("mms128", "bf16")
    rel = res["local"][0] / g0 - 1.0
    assert rel > BAR
    assert 0.18 <= rel <= 0.28, rel


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", [(100, 37, (0, 0, 0, 0), True, "trig"), (100, 37, (1, 1, 1, 1), True, "trig"),
                                  (65, 17, (0, 0, 1, 1), False, "const"), (3, 3, (0, 0, 0, 0), True, "trig")],
                         ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_local_shift_tma_bitwise_equals_plain(case, storage):
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=5 * nx + ny, bc=bc, nonlinear=nonlin, source=src)
    a = _lattice(p, storage, "local").set_sweep_variant("tma")
    b = _lattice(p, storage, "local").set_sweep_variant("plain")
    a.init(p.phi0()).step(9)
    b.init(p.phi0()).step(9)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    assert a.check() == 0


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_local_shift_checkpoint_resume_bitwise(storage):
    p = w.random_state_problem(45, 33, seed=4, bc=(1, 1, 0, 0), nonlinear=True)
    a = _lattice(p, storage, "local")
    a.init(p.phi0()).step(7)
    state = a.save()
    a.step(6)
    b = _lattice(p, storage, "local")
    b.load(state)
    b.step(6)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    # a state of the other stored form is refused
    c = _lattice(p, storage, "ref")
    with pytest.raises(Exception):
        c.load(state)
