"""Host logic of the continuous-batching server without a GPU: admission by the
memory budget, retirement at the residual tolerance or the step cap, a member
with a non-finite flag retired alone, results in request order, the queue-depth
series.  The lattice and batch classes are replaced by fakes that keep only a step
count; the workspace sizes come from the real library (no device needed)."""
import numpy as np
import pytest

import workloads as w
from paper_1902_09813_gb300 import serve


class _FakeLattice:
    """Keeps a step count.  A frozen lattice (flagged by a batch with freezing on)
    no longer moves on the device, while its host count goes on with its batch;
    settle() sets the count back, as the library does."""
    closed = 0

    def __init__(self, p):
        self.p = p
        self.steps = 0          # device state
        self.host_steps = 0     # the step count the host believes
        self.frozen_at = None

    @classmethod
    def from_problem(cls, p, compute="f32", storage="f16", stream=None, shift="auto"):
        return cls(p)

    def init(self, phi0, t0=0.0):
        return self

    def settle(self, clear=False):
        if self.frozen_at is None:
            return -1
        self.host_steps = self.frozen_at
        return self.frozen_at

    def phi_host(self):
        assert self.host_steps == self.steps
        return np.full((self.p.ny, self.p.nx), float(self.steps))

    def close(self):
        _FakeLattice.closed += 1


class _FakeBatch:
    """Residual of a member after s steps: rate ** s (rate in the problem's meta);
    a member whose meta has `bad_at` raises flag bit 1 once it passes that step."""
    created = 0
    open_ = 0

    def __init__(self, lats, stream=None):
        self.lats = lats
        self.freeze = False
        _FakeBatch.created += 1
        _FakeBatch.open_ += 1

    def set_tiles(self, *shape):
        return self

    def set_freeze(self, on=True):
        self.freeze = on
        return self

    def prepare(self, n, residual=True):
        return self

    def step(self, n, residual=False):
        for lat in self.lats:
            lat.host_steps += n
            if lat.frozen_at is None:
                lat.steps += n
        return self

    def step_tol(self, n, tol, out=None, resid_out=None):
        self.step(n, residual=True)
        for k, lat in enumerate(self.lats):
            if lat.frozen_at is not None:
                out[k], resid_out[k] = 4, float("nan")
                continue
            r = lat.p.meta["rate"] ** lat.steps
            f = (1 if r < tol else 0) | (2 if lat.steps >= lat.p.meta.get("bad_at", 1 << 30) else 0)
            out[k], resid_out[k] = f, r
            if self.freeze and f:
                lat.frozen_at = lat.steps
        return out

    def close(self):
        _FakeBatch.open_ -= 1


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(serve, "Lattice", _FakeLattice)
    monkeypatch.setattr(serve, "Batch", _FakeBatch)
    _FakeBatch.created = 0
    _FakeBatch.open_ = 0
    _FakeLattice.closed = 0


def _problems(rates, n=32):
    out = []
    for k, r in enumerate(rates):
        p = w.random_state_problem(n, n, seed=k)
        p.meta = dict(p.meta, rate=r)
        out.append(p)
    return out


def test_budget_admission_and_retirement(fakes):
    probs = _problems([0.5, 0.9, 0.99, 0.5])
    need = serve._bytes_needed(probs[0], "f32", "f16")
    budget = 2.5 * need + serve._batch_bytes(probs[:2], "f32", "f16")   # two lattices and their tables
    srv = serve.Server(budget_bytes=budget, slice_steps=10, max_steps=200, tol=1e-6, stream=object())
    res = srv.run([(0.0, p) for p in probs])
    assert [r.rid for r in res] == [0, 1, 2, 3]
    assert srv.stats["peak_active"] == 2
    # first slice whose end passes the tolerance, else the cap
    expect = []
    for r in (0.5, 0.9, 0.99, 0.5):
        s = 10
        while r ** s >= 1e-6 and s < 200:
            s += 10
        expect.append(s)
    assert [r.steps for r in res] == expect
    assert all(r.status == "done" for r in res)
    assert all(np.all(r.phi == r.steps) for r in res)
    assert res[2].residual > 1e-6 and res[2].steps == 200   # the cap, not the tolerance
    # waiting requests are admitted as members retire: every request ran, never more than two at once
    assert max(d[1] for d in srv.depth) == 2 and srv.depth[0][2] == 2


def test_oversized_request_rejected_and_budget_kept(fakes):
    """A request whose workspace and batch tables alone exceed the budget is
    rejected (status "rejected", no phi) instead of being admitted past the budget;
    the others run, and the peak of lattice workspaces plus batch tables never
    exceeds the budget."""
    probs = _problems([0.5, 0.5, 0.5])
    big = w.random_state_problem(400, 300, seed=5)
    big.meta = dict(big.meta, rate=0.5)
    small = serve._bytes_needed(probs[0], "f32", "f16")
    budget = 2 * small + serve._batch_bytes(probs[:2], "f32", "f16")
    assert serve._bytes_needed(big, "f32", "f16") > budget
    srv = serve.Server(budget_bytes=budget, slice_steps=10, max_steps=100, tol=1e-6, stream=object())
    res = srv.run([(0.0, probs[0]), (0.0, big), (0.0, probs[1]), (0.0, probs[2])])
    assert [r.status for r in res] == ["done", "rejected", "done", "done"]
    assert res[1].phi is None and srv.stats["rejected"] == 1
    assert srv.stats["peak_bytes"] <= budget
    assert srv.stats["peak_active"] == 2


def test_batch_tables_counted_in_admission(fakes):
    """Two lattices fit the budget only without their batch tables: the second
    waits for the first to retire."""
    probs = _problems([0.5, 0.5])
    need = serve._bytes_needed(probs[0], "f32", "f16")
    budget = 2 * need + serve._batch_bytes(probs[:1], "f32", "f16")   # less than the two-member tables
    assert 2 * need + serve._batch_bytes(probs, "f32", "f16") > budget
    srv = serve.Server(budget_bytes=budget, slice_steps=10, max_steps=100, tol=1e-6, stream=object())
    res = srv.run([(0.0, p) for p in probs])
    assert [r.status for r in res] == ["done", "done"]
    assert srv.stats["peak_active"] == 1 and srv.stats["peak_bytes"] <= budget


def test_stop_reasons_counted(fakes):
    probs = _problems([0.5, 0.999])
    srv = serve.Server(budget_bytes=1e12, slice_steps=10, max_steps=50, tol=1e-6, stream=object())
    srv.run([(0.0, p) for p in probs])
    assert srv.stats["tol_hits"] == 1 and srv.stats["cap_hits"] == 1


def test_unstable_member_retired_alone(fakes):
    probs = _problems([0.9, 0.9, 0.9])
    probs[1].meta["bad_at"] = 30
    srv = serve.Server(budget_bytes=1e12, slice_steps=10, max_steps=100, tol=1e-30, stream=object())
    res = srv.run([(0.0, p) for p in probs])
    assert [r.status for r in res] == ["done", "unstable", "done"]
    assert res[1].steps == 30 and res[0].steps == 100 and res[2].steps == 100


def test_depth_series_thinning():
    depth = [(0.1 * k, k % 5, 10 - k % 10) for k in range(100)]
    out = serve.depth_series(depth, points=16)
    assert out[0] == list(depth[0]) and out[-1] == list(depth[-1])
    assert 16 <= len(out) <= 18
    assert serve.depth_series([]) == []


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_queued_slices_give_the_same_results(fakes, depth):
    """With one, two or three slices queued ahead of the flags being read, every
    request stops at the same step with the same phi (a flagged member stays
    frozen in the slices queued after it: the fake checks that the host's step
    count was set back before phi is read); every lattice and every batch is
    closed at the end and the budget is returned."""
    probs = _problems([0.5, 0.9, 0.99, 0.5, 0.7, 0.95])
    probs[4].meta["bad_at"] = 20
    srv = serve.Server(budget_bytes=1e12, slice_steps=10, max_steps=120, tol=1e-6, stream=object(),
                       depth=depth)
    res = srv.run([(0.0, p) for p in probs])
    assert [r.status for r in res] == ["done", "done", "done", "done", "unstable", "done"]
    expect = []
    for r in (0.5, 0.9, 0.99, 0.5, None, 0.95):
        s = 10
        while r is not None and r ** s >= 1e-6 and s < 120:
            s += 10
        expect.append(s if r is not None else 20)
    assert [r.steps for r in res] == expect
    assert all(np.all(r.phi == r.steps) for r in res)
    assert _FakeLattice.closed == len(probs) and _FakeBatch.open_ == 0
    assert srv._used == 0
    caps = sum(1 for r in res if r.status == "done" and r.steps == 120)
    assert caps == 3 and srv.stats["cap_hits"] == caps
    assert srv.stats["tol_hits"] == 2 and srv.stats["unstable"] == 1


def test_first_burst_starts_the_device_early(fakes):
    """With nothing running, only `first_burst` requests are admitted before the
    first slice is queued; the others join later slices, and every request still
    stops where it would alone."""
    probs = _problems([0.5, 0.9, 0.7, 0.5, 0.95, 0.6])
    srv = serve.Server(budget_bytes=1e12, slice_steps=10, max_steps=60, tol=1e-6, stream=object(), first_burst=2)
    res = srv.run([(0.0, p) for p in probs])
    assert srv.depth[0][1] == 2                       # the first slice ran two members
    assert srv.stats["peak_active"] > 2               # the rest joined while it ran
    for r, p in zip(res, probs):
        s = 10
        while p.meta["rate"] ** s >= 1e-6 and s < 60:
            s += 10
        assert r.steps == s and np.all(r.phi == r.steps)
    assert _FakeLattice.closed == len(probs) and _FakeBatch.open_ == 0
