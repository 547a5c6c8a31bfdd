"""The vector-access sweeps: one step per launch (BTRT_SWEEP_VEC), each thread
owning four x-consecutive nodes and moving every population plane with one
vector load and one vector store, and two steps per launch (BTRT_SWEEP_TB2V)
with the same access in both steps.  Their per-node arithmetic is the plain
sweep's, so the results must be bitwise identical for every storage format and
shift, both coefficient modes, every source kind, periodic and bounce-back
sides, and widths that are not multiples of four (ragged last groups, groups
that fall back to the per-node path next to the domain edges)."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

CASES = [
    # (nx, ny, bc, nonlinear, source)
    (100, 37, (0, 0, 0, 0), True, "trig"),
    (100, 37, (1, 1, 1, 1), True, "trig"),
    (65, 17, (0, 0, 1, 1), False, "const"),
    (130, 50, (1, 1, 0, 0), False, "none"),
    (131, 9, (0, 0, 0, 0), False, "trig"),
    (3, 3, (0, 0, 0, 0), True, "trig"),
    (4, 4, (1, 1, 1, 1), True, "const"),
    (9, 5, (0, 0, 1, 1), True, "trig"),
    (10, 6, (1, 1, 1, 1), False, "none"),
    (5, 97, (1, 1, 0, 0), True, "reaction"),
    (33, 17, (0, 0, 0, 0), True, "reaction"),
    (258, 3, (1, 1, 0, 0), True, "trig"),
]
FORMATS = [("f32", "ref"), ("f32", "local"), ("f16", "ref"), ("f16", "local"), ("bf16", "ref"), ("bf16", "local")]


def _lattice(p, storage, shift, variant):
    from paper_1902_09813_gb300 import Lattice
    return Lattice.from_problem(p, compute="f32", storage=storage, shift=shift).set_sweep_variant(variant)


def _against_plain(p, storage, shift, steps, form="vec"):
    a = _lattice(p, storage, shift, form)
    b = _lattice(p, storage, shift, "plain")
    a.init(p.phi0(), t0=p.t0).step(steps)
    b.init(p.phi0(), t0=p.t0).step(steps)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    assert a.time() == b.time()
    assert a.check() == 0
    return a, b


@pytest.mark.parametrize("fmt", FORMATS, ids=lambda f: "-".join(f))
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_vec_sweep_bitwise_equals_plain(case, fmt):
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=7 * nx + ny, bc=bc, nonlinear=nonlin, source=src,
                               flux_q=2.5 if src == "reaction" else 2.0)
    _against_plain(p, fmt[0], fmt[1], 9)


TB2V_CASES = CASES + [
    (37, 70, (0, 0, 0, 0), True, "trig"),     # tiles ragged in x and y, periodic ring wraps
    (64, 64, (1, 1, 1, 1), False, "trig"),    # whole tiles, walls on every side
    (70, 33, (1, 1, 0, 0), True, "const"),
]


@pytest.mark.parametrize("steps", [9, 10])
@pytest.mark.parametrize("fmt", FORMATS, ids=lambda f: "-".join(f))
@pytest.mark.parametrize("case", TB2V_CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_tb2v_sweep_bitwise_equals_plain(case, fmt, steps):
    """Two steps per launch with vector access (the intermediate step in shared
    memory in the storage format): bitwise equal to one plain step per launch,
    for odd step counts too (the last step runs in the plain form)."""
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=5 * nx + 3 * ny, bc=bc, nonlinear=nonlin, source=src,
                               flux_q=2.5 if src == "reaction" else 2.0)
    _against_plain(p, fmt[0], fmt[1], steps, form="tb2v")


def test_vec_sweep_fields_residual_and_large_ragged_grid():
    """Per-node tensor and source fields (the variable-tensor problem), the
    residual step after vector-form steps, and a 4099 x 4093 grid with FP16
    storage and the local shift and FP32 storage with the reference shift."""
    p = w.variable_tensor(n=70, alpha=1e-2, walls=True, t_end=0.2)
    p = p.replace(dt=20.0 * p.dx ** 2, nsteps=11, phi_ref=0.0)
    for form in ("vec", "tb2v"):
        for storage, shift in (("f32", "ref"), ("f16", "local")):
            a, b = _against_plain(p, storage, shift, p.nsteps, form=form)
            assert a.step_residual(5) == b.step_residual(5)
    q = w.nonlinear_modes(n=4096, nsteps=4).replace(nx=4099, ny=4093)
    for storage, shift in (("f32", "ref"), ("f16", "local"), ("bf16", "local")):
        b = _lattice(q, storage, shift, "plain")
        b.init(q.phi0()).step(4)
        pb = b.phi_host()
        del b
        for form in ("vec", "tb2v"):
            a = _lattice(q, storage, shift, form)
            a.init(q.phi0()).step(4)
            assert np.array_equal(a.phi_host(), pb), form
            del a


def test_vec_sweep_mms_8192_matches_plain():
    """The benchmark's 8192^2 manufactured-solution lattice, FP16 local shift,
    both vector forms."""
    q = w.mms_sinsin(n=8192, nsteps=4)
    b = _lattice(q, "f16", "local", "plain")
    b.init(q.phi0(), t0=q.t0).step(4)
    pb = b.phi_host()
    del b
    for form in ("vec", "tb2v"):
        a = _lattice(q, "f16", "local", form)
        a.init(q.phi0(), t0=q.t0).step(4)
        assert np.array_equal(a.phi_host(), pb), form
        del a


def test_vec_rejects_other_compute():
    from paper_1902_09813_gb300 import Lattice, _capi as C
    p = w.random_state_problem(20, 20, seed=2)
    for c in ("f64", "df64"):
        for form in ("vec", "tb2v"):
            with pytest.raises(C.BtrtError):
                Lattice.from_problem(p, compute=c).set_sweep_variant(form)
