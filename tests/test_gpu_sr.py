"""Stochastically rounded FP16/BF16 storage (BTRT_SHIFT_LOCAL_SR and, with phi as
a double-word pair, BTRT_SHIFT_LOCAL_DW_SR).

Checked here: against the FP64 oracle about as close as round-to-nearest storage
(stochastic rounding has twice the error variance of round-to-nearest per value,
but no repeated bias); the plain and vector forms store the same values bitwise,
since the random bits depend only on the node, the step index and the population;
the stored values are not those of round-to-nearest; the steps are reproducible
(same steps, same values) and survive checkpoint/resume bitwise; the kernel forms,
storage formats and batch forms that do not take it refuse it; in the batch forms
that take it every member stores what it stores alone."""
import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _lattice(p, storage, shift, **kw):
    from paper_1902_09813_gb300 import Lattice
    return Lattice.from_problem(p, compute="f32", storage=storage, shift=shift, **kw)


CASES = [(37, 29, (0, 0, 0, 0), True, "trig"), (37, 29, (1, 1, 1, 1), True, "trig"),
         (70, 65, (0, 0, 1, 1), True, "const"), (96, 40, (1, 1, 1, 1), False, "trig"),
         (3, 3, (1, 1, 1, 1), True, "const"), (5, 97, (1, 1, 0, 0), True, "reaction")]


RN_OF = {"local_sr": "local", "local_dw_sr": "local_dw", "moment_sr": "local"}


@pytest.mark.parametrize("shift", ["local_sr", "local_dw_sr", "moment_sr"])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_sr_matches_oracle_like_round_to_nearest(case, storage, shift):
    """phi after 10 steps, and the post-collision populations as read back (the
    first-moment form adds its stored j), against the FP64 oracle: at most twice
    the error of round-to-nearest storage with the local shift."""
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=17 * nx + ny, bc=bc, nonlinear=nonlin, source=src,
                               flux_q=2.5 if src == "reaction" else 2.0)
    steps = 10
    o = oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(steps)
    ref = o.phi()
    o.step(1)
    got, gotf = {}, {}
    for sh in (shift, RN_OF[shift]):
        lat = _lattice(p, storage, sh)
        lat.init(p.phi0(), t0=p.t0).step(steps)
        assert lat.check() == 0
        got[sh] = _rel(lat.phi_host(), ref)
        gotf[sh] = _rel(lat.read_f(), o.fpost)
    rn = got[RN_OF[shift]]
    assert got[shift] <= 2.0 * rn + 1e-6, got
    assert gotf[shift] <= 2.0 * gotf[RN_OF[shift]] + 1e-6, gotf


@pytest.mark.parametrize("shift", ["local_sr", "moment_sr"])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("workload", ["mms", "nonlinear"])
def test_sr_plain_and_vector_forms_bitwise(storage, workload, shift):
    """Interior groups on the vector path, edges on the per-node path: every node
    stores the same stochastically rounded values as in the plain form."""
    if workload == "mms":
        p = w.mms_sinsin(n=130)
    else:
        p = w.random_state_problem(134, 70, seed=5, bc=(0, 0, 1, 1), nonlinear=True)
    out = {}
    for form in ("plain", "vec"):
        lat = _lattice(p, storage, shift)
        lat.set_sweep_variant(form)
        lat.init(p.phi0(), t0=p.t0).step(9)
        out[form] = (lat.phi_host(), lat.read_f())
    assert np.array_equal(out["plain"][0], out["vec"][0])
    assert np.array_equal(out["plain"][1], out["vec"][1])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_sr_differs_from_round_to_nearest_and_repeats(storage):
    p = w.random_state_problem(66, 41, seed=9, bc=(1, 1, 0, 0), nonlinear=True)
    runs = []
    for shift in ("local_sr", "local_sr", "local"):
        lat = _lattice(p, storage, shift).init(p.phi0(), t0=p.t0).step(6)
        runs.append(lat.read_f())
    assert np.array_equal(runs[0], runs[1])          # same steps, same random bits
    assert not np.array_equal(runs[0], runs[2])      # not the round-to-nearest values
    # the two roundings differ by at most one last place of the stored deviation
    assert _rel(runs[0], runs[2]) < 1e-2


@pytest.mark.parametrize("shift", ["local_sr", "local_dw_sr", "moment_sr"])
def test_sr_checkpoint_resume_bitwise(shift):
    p = w.random_state_problem(45, 33, seed=4, bc=(1, 1, 0, 0), nonlinear=True)
    a = _lattice(p, "bf16", shift)
    a.init(p.phi0()).step(7)
    state = a.save()
    a.step(6)
    b = _lattice(p, "bf16", shift)
    b.load(state)
    b.step(6)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())


def test_sr_refusals():
    from paper_1902_09813_gb300 import Batch, Lattice, _capi as C
    p = w.random_state_problem(40, 30, seed=6)
    lat = _lattice(p, "f16", "local_sr").init(p.phi0())
    for form in ("tb2", "tb2v", "tma"):
        with pytest.raises(C.BtrtError):
            lat.set_sweep_variant(form)
    lat.set_sweep_variant("vec")
    lat.set_sweep_variant("plain")
    dw = _lattice(p, "f16", "local_dw_sr").init(p.phi0())
    with pytest.raises(C.BtrtError):
        dw.set_sweep_variant("vec")
    with pytest.raises(C.BtrtError):
        Batch([dw])
    mo = _lattice(p, "bf16", "moment_sr").init(p.phi0())
    for form in ("tb2", "tb2v", "tma"):
        with pytest.raises(C.BtrtError):
            mo.set_sweep_variant(form)
    mo.set_sweep_variant("vec")
    with pytest.raises(C.BtrtError):
        Batch([mo])
    b = Batch([lat])                     # stochastic rounding in batches: not in the two-step form
    with pytest.raises(C.BtrtError):
        b.set_tiles(32, 8, 2, 2)
    b.close()
    with pytest.raises(C.BtrtError):
        Lattice.from_problem(p, compute="f32", storage="f32", shift="local_sr")
    with pytest.raises(C.BtrtError):
        Lattice.from_problem(p, compute="f64", storage="f64", shift="local_sr")


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_sr_unbiased_on_a_uniform_state(storage):
    """A uniform field: every node computes the same post-collision deviations, so
    round-to-nearest stores the same rounded value everywhere (a bias of up to half
    a last place), while stochastic rounding stores the two neighbouring values in
    proportions whose mean is the unrounded deviation (FP32 storage of the same
    lattice gives that value).  Over 65536 nodes the stochastic mean is within four
    standard errors of it and far closer than round-to-nearest."""
    n = 256
    p = w.random_state_problem(n, n, seed=2, nonlinear=False, source="const")
    p = p.replace(phi0_fn=None, phi0_array=np.full((n, n), 0.7))
    wts = np.array([4, 1, 1, 1, 1, 0.25, 0.25, 0.25, 0.25]) / 9.0
    f = {}
    for st, sh in ((storage, "local_sr"), (storage, "local"), ("f32", "local")):
        # the initialising collision's stores (f = f_eq(phi0), the same deviation at every
        # node), as stored: the populations read back less w_i phi of the node (the
        # stochastically rounded phi plane may differ from node to node by one place)
        lat = _lattice(p, st, sh).init(p.phi0(), t0=p.t0)
        f[(st, sh)] = lat.read_f() - wts[:, None, None] * lat.phi_host()[None]
    ref = f[("f32", "local")]
    sr = f[(storage, "local_sr")] - ref
    rn = f[(storage, "local")] - ref
    checked = 0
    for i in range(1, 9):
        assert np.ptp(rn[i]) == 0.0                  # one rounded value everywhere
        bias = abs(float(rn[i].mean()))
        if bias == 0.0:
            continue                                 # exactly representable: nothing to test
        vals = np.unique(sr[i])
        assert 1 <= len(vals) <= 2                    # the two neighbours of the exact value
        mean, se = float(sr[i].mean()), float(sr[i].std()) / n
        assert abs(mean) <= 4.0 * se + 1e-12, (i, mean, se, bias)
        assert abs(mean) < 0.2 * bias, (i, mean, bias)
        checked += 1
    assert checked >= 4


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("form", [0, 1, 3])
def test_sr_batch_members_equal_alone(storage, form):
    """The random bits depend on the member's own node, step and population, so a
    member stores in a batch exactly what it stores alone (persistent, one step per
    launch and vector batch forms; autotuning skips the two-step form)."""
    from paper_1902_09813_gb300 import Batch
    probs = w.batched_instances(count=6, seed=7, nmin=20, nmax=140, nsteps=0)
    probs.append(w.random_state_problem(45, 31, seed=8, bc=(1, 1, 0, 0), nonlinear=True))
    alone = [_lattice(p, storage, "local_sr").init(p.phi0(), t0=p.t0).step(9) for p in probs]
    mixed = [_lattice(p, storage, "local_sr").init(p.phi0(), t0=p.t0) for p in probs]
    b = Batch(mixed).set_tiles(32, 4, 2, form)
    b.step(4).step(5, residual=True)
    for a, m in zip(alone, mixed):
        assert np.array_equal(a.phi_host(), m.phi_host())
        assert np.array_equal(a.read_f(), m.read_f())
    shape = b.autotune(steps_per_trial=1)
    assert shape[3] != 2
    b.close()
