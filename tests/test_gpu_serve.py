"""Continuous-batching server: requests that arrive while others run are admitted
at slice boundaries and share the device; each result is bitwise the same as the
same problem solved alone for the same number of steps; the plain sequential
baseline gives the same answers; memory admission respects the budget."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def _problems(count=9, seed=21):
    probs = w.batched_instances(count=count, seed=seed, nmin=24, nmax=96, nsteps=0)
    for p in probs:
        p.phi_ref = float(p.phi0().mean())
    return probs


def _alone(p, steps, compute="f32", storage="f16", shift="auto"):
    from paper_1902_09813_gb300 import Lattice
    lat = Lattice.from_problem(p, compute=compute, storage=storage, shift=shift)
    lat.init(p.phi0(), t0=p.t0).step(steps)
    return lat.phi_host()


@pytest.mark.parametrize("shift", ["auto", "local_sr"])
def test_serve_results_equal_alone(shift):
    from paper_1902_09813_gb300.serve import Server, poisson_trace
    probs = _problems()
    trace = poisson_trace(probs, rate=400.0, seed=1)
    srv = Server(slice_steps=20, max_steps=120, tol=1e-30, shift=shift)
    res = srv.run(trace)
    assert len(res) == len(probs)
    assert srv.stats["peak_active"] >= 2          # work overlapped on the device
    for r, p in zip(res, probs):
        assert r.steps == 120
        assert r.finished >= r.arrival
        assert np.array_equal(r.phi, _alone(p, r.steps, shift=shift))


def test_serve_convergence_stop_and_sequential_baseline():
    from paper_1902_09813_gb300.serve import Server, poisson_trace, serve_sequential
    probs = _problems(count=5, seed=4)
    trace = poisson_trace(probs, rate=1000.0, seed=2)
    tol = 1e-3   # loose: members stop at different slices
    srv = Server(slice_steps=10, max_steps=400, tol=tol)
    res = srv.run(trace)
    seq = serve_sequential(trace, slice_steps=10, max_steps=400, tol=tol)
    for a, b, p in zip(res, seq, probs):
        assert a.steps == b.steps
        assert a.residual < tol or a.steps == 400
        assert np.array_equal(a.phi, b.phi)
        assert a.residual == pytest.approx(b.residual, rel=1e-12, abs=1e-300)


def test_serve_budget_limits_admission():
    from paper_1902_09813_gb300.serve import Server, _bytes_needed, poisson_trace
    probs = _problems(count=6, seed=9)
    need = max(_bytes_needed(p, "f32", "f16") for p in probs)
    trace = poisson_trace(probs, rate=1e6, seed=3)      # all arrive at once
    srv = Server(budget_bytes=2.5 * need, slice_steps=10, max_steps=30, tol=1e-30)
    res = srv.run(trace)
    assert len(res) == 6
    assert srv.stats["peak_bytes"] <= 2.5 * need
    assert srv.stats["peak_active"] < len(probs)      # the budget held some requests back


def test_unstable_request_is_retired_alone():
    """A request whose initial field holds a NaN (a failure made on the host) is
    reported as unstable after its first slice; the others complete and equal
    their solves alone, in the server and in the sequential baseline."""
    from paper_1902_09813_gb300.serve import Server, poisson_trace, serve_sequential
    probs = _problems(count=5, seed=13)
    bad = probs[2]
    arr = bad.phi0()
    arr[3, 4] = float("nan")
    probs[2] = bad.replace(phi0_fn=None, phi0_array=arr)
    trace = poisson_trace(probs, rate=1e6, seed=4)
    srv = Server(slice_steps=10, max_steps=40, tol=1e-30)
    res = srv.run(trace)
    seq = serve_sequential(trace, slice_steps=10, max_steps=40, tol=1e-30)
    for out in (res, seq):
        assert [r.status for r in out] == ["done", "done", "unstable", "done", "done"]
        assert out[2].steps == 10
        for k in (0, 1, 3, 4):
            assert out[k].steps == 40
            assert np.array_equal(out[k].phi, _alone(probs[k], 40))
