"""Batched persistent launch: every member's result is bitwise the same alone and
in the mix, for every tile shape; FP64 batches match the oracle; residuals match
the definition; a barrier wait that cannot complete ends with BTRT_ETIMEOUT."""
import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads

pytestmark = pytest.mark.gpu


def _mix(compute="f32", storage="f16", count=10, seed=3):
    probs = w.batched_instances(count=count, seed=seed, nmin=20, nmax=150, nsteps=30)
    for k, p in enumerate(probs):
        p.phi_ref = float(p.phi0().mean()) if storage != "f64" else 0.0
    # add a nonlinear member and ragged/wall variety
    probs.append(w.random_state_problem(45, 31, seed=8, bc=(1, 1, 0, 0), nonlinear=True))
    probs.append(w.random_state_problem(33, 70, seed=9, bc=(0, 0, 1, 1), nonlinear=False, source="const"))
    return probs


def _make(p, compute, storage, shift="ref"):
    import torch
    from paper_1902_09813_gb300 import Lattice
    lat = Lattice.from_problem(p, compute=compute, storage=storage, stream=torch.cuda.current_stream(),
                               shift=shift)
    lat.init(p.phi0(), t0=p.t0)
    return lat


@pytest.mark.parametrize("compute,storage,shift", [("f32", "f16", "ref"), ("f32", "f32", "ref"),
                                                  ("f32", "bf16", "ref"), ("f64", "f64", "ref"),
                                                  ("f32", "f16", "local"), ("f32", "bf16", "local")])
def test_alone_equals_in_mix_bitwise(compute, storage, shift):
    from paper_1902_09813_gb300 import Batch
    probs = _mix(compute, storage)
    steps = 17
    alone = [_make(p, compute, storage, shift).step(steps) for p in probs]
    mixed = [_make(p, compute, storage, shift) for p in probs]
    b = Batch(mixed)
    b.step(5).step(12)
    b.set_tiles(32, 8, 2, 2 if compute == "f32" else 1).step(3)
    alone = [a.step(3) for a in alone]
    for a, m in zip(alone, mixed):
        assert np.array_equal(a.phi_host(), m.phi_host())
        assert np.array_equal(a.read_f(), m.read_f())
        assert a.time() == m.time()
    b.close()


@pytest.mark.parametrize("compute,storage,shift,shape", [("f32", "f16", "local", (32, 8, 4, 1)),
                                                        ("f32", "f16", "local", (32, 8, 4, 2)),
                                                        ("f32", "f16", "local", (16, 16, 1, 3)),
                                                        ("f32", "f32", "ref", (32, 8, 2, 3)),
                                                        ("f32", "bf16", "ref", (32, 8, 1, 2)),
                                                        ("f32", "f32", "ref", (32, 8, 2, 0)),
                                                        ("f64", "f64", "ref", (32, 8, 4, 1))])
def test_constant_coefficient_batch_form_bitwise(compute, storage, shift, shape):
    """A batch whose members all take the constant-coefficient collision and no
    reaction source runs the form compiled for that case; a member switched to
    nonlinear coefficients between slices makes the next slice run the form that
    takes any member.  Both stay bitwise equal to the members stepped alone."""
    from paper_1902_09813_gb300 import Batch
    probs = w.batched_instances(count=8, seed=21, nmin=20, nmax=150, nsteps=30)
    for p in probs:
        p.phi_ref = float(p.phi0().mean()) if storage != "f64" else 0.0
    alone = [_make(p, compute, storage, shift).step(10) for p in probs]
    mixed = [_make(p, compute, storage, shift) for p in probs]
    b = Batch(mixed).set_tiles(*shape)
    b.step(10)
    for a, m in zip(alone, mixed):
        assert np.array_equal(a.phi_host(), m.phi_host())
    for lat in (alone[3], mixed[3]):
        c = lat.coef
        c.a2 = 0.5
        c.b2 = 0.01
        lat.set_coeffs(c)
    b.step(7)
    alone = [a.step(7) for a in alone]
    for a, m in zip(alone, mixed):
        assert np.array_equal(a.phi_host(), m.phi_host())
        assert np.array_equal(a.read_f(), m.read_f())
    assert b.check() == 0
    b.close()


@pytest.mark.parametrize("shape", [(32, 8, 1, 0), (32, 8, 4, 0), (64, 4, 2, 0), (32, 4, 2, 0),
                                   (32, 8, 1, 1), (64, 4, 2, 1), (32, 8, 4, 2), (64, 4, 1, 2),
                                   (16, 16, 1, 1), (8, 32, 1, 0), (32, 8, 1, 3), (32, 8, 4, 3),
                                   (64, 4, 2, 3), (16, 16, 1, 3), (8, 32, 1, 3), (32, 4, 4, 3), (16, 8, 2, 3),
                                   (32, 4, 4, 1)])
def test_tile_shapes_bitwise(shape):
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f32", "f16", count=6, seed=5)
    ref = [_make(p, "f32", "f16").step(9) for p in probs]
    mixed = [_make(p, "f32", "f16") for p in probs]
    b = Batch(mixed).set_tiles(*shape)
    b.step(9)
    for a, m in zip(ref, mixed):
        assert np.array_equal(a.phi_host(), m.phi_host())
    b.close()


def test_fp64_batch_matches_oracle():
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f64", "f64", count=6, seed=7)
    lats = [_make(p, "f64", "f64") for p in probs]
    b = Batch(lats)
    b.step(11)
    for p, lat in zip(probs, lats):
        o = oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(11)
        ref = o.phi()
        got = lat.phi_host()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-11
    b.close()


def test_residuals_match_definition():
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f64", "f64", count=5, seed=11)
    lats = [_make(p, "f64", "f64") for p in probs]
    b = Batch(lats)
    b.step(6)
    before = [l.phi_host() for l in lats]
    b.step(4, residual=True)
    # the residual is of the last step only: redo the comparison from step 9 to 10
    lats2 = [_make(p, "f64", "f64").step(9) for p in probs]
    r = b.residuals()
    for k, l2 in enumerate(lats2):
        a = l2.phi_host()
        l2.step(1)
        expect = np.linalg.norm(l2.phi_host() - a)
        assert r[k] == pytest.approx(expect, rel=1e-9, abs=1e-300)
    del before
    b.close()


def test_two_step_form_residual_and_odd_steps():
    """The two-step batch form with an odd slice and a residual slice: results
    bitwise equal to the members alone, residuals equal to the definition."""
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f32", "f32", count=5, seed=19)
    alone = [_make(p, "f32", "f32") for p in probs]
    mixed = [_make(p, "f32", "f32") for p in probs]
    b = Batch(mixed).set_tiles(32, 8, 2, 2)
    b.step(7)
    b.step(6, residual=True)
    r = b.residuals()
    for a in alone:
        a.step(12)
    before = [a.phi_host() for a in alone]
    for a in alone:
        a.step(1)
    for k, (a, m) in enumerate(zip(alone, mixed)):
        assert np.array_equal(a.phi_host(), m.phi_host())
        assert np.array_equal(a.read_f(), m.read_f())
        assert a.time() == m.time()
        expect = np.linalg.norm(a.phi_host() - before[k])
        assert r[k] == pytest.approx(expect, rel=1e-5, abs=1e-30)
    b.close()


def test_vector_form_residual_slice():
    """The vector batch form with a residual slice (its last step in the
    step-per-launch form): results bitwise equal to the members alone, residuals
    equal to the definition."""
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f32", "f16", count=5, seed=23)
    alone = [_make(p, "f32", "f16", "local") for p in probs]
    mixed = [_make(p, "f32", "f16", "local") for p in probs]
    b = Batch(mixed).set_tiles(16, 16, 1, 3)
    b.step(7)
    b.step(6, residual=True)
    r = b.residuals()
    for a in alone:
        a.step(12)
    before = [a.phi_host() for a in alone]
    for a in alone:
        a.step(1)
    for k, (a, m) in enumerate(zip(alone, mixed)):
        assert np.array_equal(a.phi_host(), m.phi_host())
        assert np.array_equal(a.read_f(), m.read_f())
        expect = np.linalg.norm(a.phi_host() - before[k])
        assert r[k] == pytest.approx(expect, rel=1e-5, abs=1e-30)
    b.close()


def test_autotune_keeps_results():
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f32", "f16", count=6, seed=13)
    mixed = [_make(p, "f32", "f16") for p in probs]
    b = Batch(mixed)
    shape = b.autotune(steps_per_trial=2)
    assert shape[:3] in [(32, 8, 1), (32, 8, 2), (32, 8, 4), (64, 4, 1), (64, 4, 2), (32, 4, 2), (16, 16, 1),
                         (8, 32, 1), (32, 4, 4), (16, 8, 2)]
    assert shape[3] in (0, 1, 2, 3)
    n_done = mixed[0].time()[0]
    assert n_done == 10 * 4 * 3   # ten shapes, four forms (FP32), 1 + 2 steps each
    ref = [_make(p, "f32", "f16").step(n_done + 5) for p in probs]
    b.step(5)
    for a, m in zip(ref, mixed):
        assert np.array_equal(a.phi_host(), m.phi_host())
    b.close()


def test_step_tol_flags_match_residuals_and_nonfinite():
    """btrt_batch_step_tol: bit 0 exactly where the member's residual of the last
    step is below tol, bit 1 for the member whose initial field holds a NaN (a
    failure made on the host); flags in pinned host memory and in device memory
    agree, and the members advance as with btrt_batch_step."""
    import torch
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f32", "f16", count=6, seed=29)
    mixed = [_make(p, "f32", "f16", "local") for p in probs]
    bad = w.random_state_problem(24, 20, seed=4, bc=(1, 1, 0, 0))
    arr = bad.phi0()
    arr[3, 4] = float("nan")
    lat_bad = _make(bad.replace(phi0_array=arr), "f32", "f16", "local")
    b = Batch(mixed + [lat_bad])
    flags = b.step_tol(10, tol=1e30)
    torch.cuda.synchronize()
    f = flags.numpy()
    assert list(f[:-1] & 2) == [0] * len(mixed) and f[-1] & 2 == 2
    r = b.residuals()
    tol = float(np.median(r[:-1]))
    flags = b.step_tol(4, tol=tol)
    dev = torch.empty(len(mixed) + 1, dtype=torch.int32, device="cuda")
    r = b.residuals()            # synchronises: the pinned flags are ready
    f = flags.numpy().copy()
    assert list(f[:-1] & 1) == [1 if v < tol else 0 for v in r[:-1]]
    b.step_tol(1, tol=tol, out=dev)
    r1 = b.residuals()
    assert list(dev.cpu().numpy()[:-1] & 1) == [1 if v < tol else 0 for v in r1[:-1]]
    assert mixed[0].time()[0] == 15
    b.close()


@pytest.mark.parametrize("own_stream", [False, True])
def test_slice_graphs_captured_and_prepare_advances_nothing(own_stream):
    """The slice graphs are captured on the default stream as on a stream of the
    caller's; btrt_batch_prepare captures without running (no member moves), and
    the replayed graphs give the members' plain results bitwise, in every form."""
    import torch
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f32", "f16", count=5, seed=31)
    stream = torch.cuda.Stream() if own_stream else torch.cuda.current_stream()
    with torch.cuda.stream(stream):
        mixed = [_make(p, "f32", "f16", "local") for p in probs]
        ref = [_make(p, "f32", "f16", "local") for p in probs]
        b = Batch(mixed, stream=stream)
        for form in (1, 2, 3, 0):
            b.set_tiles(32, 4, 2, form)
            assert b.graphs() == 0
            b.prepare(6)
            # the cooperative persistent form (0) may not be capturable: it then launches directly
            captured = b.graphs()
            assert captured == 1 or (form == 0 and captured == -1)
            assert mixed[0].time()[0] == ref[0].time()[0]      # nothing ran
            b.step_tol(6, tol=0.0)
            b.step(6, residual=True)
            assert b.graphs() == captured                      # replayed, not captured again
            for a in ref:
                a.step(12)
        stream.synchronize()
        for a, m in zip(ref, mixed):
            assert np.array_equal(a.phi_host(), m.phi_host())
        b.close()


@pytest.mark.parametrize("form", [1, 2, 3, 0])
def test_freeze_keeps_flagged_members_and_settle_rewinds(form):
    """Freezing on: the members a step_tol call flags are left unchanged by later
    launches of this batch and of a new one (bit 2 and a NaN residual from then
    on), settle() sets their step counts back to the flagged step, and a cleared
    member steps on alone as if never batched; the others stay bitwise equal to
    their solves alone."""
    import torch
    from paper_1902_09813_gb300 import Batch
    probs = _mix("f32", "f16", count=6, seed=41)
    mixed = [_make(p, "f32", "f16", "local") for p in probs]
    b = Batch(mixed).set_tiles(32, 4, 2, form).set_freeze(True)
    n = len(mixed)
    f = torch.empty(n, dtype=torch.int32, pin_memory=True)
    r = torch.empty(n, dtype=torch.float64, pin_memory=True)
    b.step_tol(10, tol=0.0, out=f, resid_out=r)
    torch.cuda.synchronize()
    assert not f.numpy().any()
    tol = float(np.median(r.numpy()))
    b.step_tol(5, tol=tol, out=f, resid_out=r)
    torch.cuda.synchronize()
    frozen = (f.numpy() & 1).astype(bool)
    assert 0 < frozen.sum() < n
    b.step_tol(7, tol=0.0, out=f, resid_out=r)
    torch.cuda.synchronize()
    assert list(f.numpy() & 4) == [4 if z else 0 for z in frozen]
    assert np.all(np.isnan(r.numpy()[frozen])) and not np.any(np.isnan(r.numpy()[~frozen]))
    b.close()
    b2 = Batch(mixed).set_tiles(32, 8, 1, 1)
    b2.step(4)
    torch.cuda.synchronize()
    b2.close()
    for k, (p, lat) in enumerate(zip(probs, mixed)):
        s = lat.settle()
        assert s == (15 if frozen[k] else -1)
        steps = 15 if frozen[k] else 26
        assert lat.time()[0] == steps
        ref = _make(p, "f32", "f16", "local").step(steps)
        assert np.array_equal(lat.phi_host(), ref.phi_host())
        if frozen[k]:
            assert lat.settle(clear=True) == 15
            assert lat.settle() == -1
            lat.step(3)
            assert np.array_equal(lat.phi_host(), ref.step(3).phi_host())


def test_barrier_timeout_reported():
    """A barrier that can never be released ends the launch after the wait limit
    with BTRT_ETIMEOUT (no hang, no device fault); the device stays usable."""
    from paper_1902_09813_gb300 import Batch, _capi as C
    probs = _mix("f32", "f16", count=4, seed=17)
    lats = [_make(p, "f32", "f16") for p in probs]
    b = Batch(lats).set_wait_limit(2000, never_release=True)
    b.step(3)
    with pytest.raises(C.BtrtError) as ei:
        b.check()
    assert ei.value.code == C.ETIMEOUT
    b.close()
    fresh = _make(probs[0], "f32", "f16").step(2)
    assert fresh.check() == 0
