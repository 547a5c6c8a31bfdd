"""Continuous-batching solve server for B-TriRT lattices.

Requests (lattice problems) arrive over time.  The server admits them while the
device-memory budget allows, keeps every admitted lattice resident, and
advances all active lattices together in slices of ``slice_steps`` steps with
one batched launch (a CUDA graph) per slice (:class:`~.lattice.Batch`).  The
device computes each member's steady-state residual ||phi^{n+1} - phi^n||_2 in
the slice's last step, compares it with the tolerance and freezes the members
it flags.  Two slices stay queued: when slice k has finished, the server reads
its flags (slice k + 1 already runs, leaving the flagged members as they
were), retires the members that converged (residual < tol), went non-finite or
reached ``max_steps``, copies their phi to the host and frees their memory.
Admission of arriving requests, the phi copies and the next batch's graph
capture happen while slices run, so requests join the next slice queued and
share the device with the others.

:func:`serve_sequential` is the plain baseline: the same requests, first come
first served, one lattice at a time with plain per-step launches and the same
stopping rule.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import List, Optional

import numpy as np
import torch

from .lattice import Batch, Lattice, batch_workspace_bytes, grid_desc, workspace_bytes


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float          # seconds since the start of the trace
    admitted: float
    finished: float
    steps: int
    residual: float
    phi: Optional[np.ndarray]
    status: str = "done"     # "unstable": a non-finite phi appeared; the request was retired alone;
                             # "rejected": it needs more device memory than the whole budget (no phi)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _desc(p, compute, storage):
    # the workspace size does not depend on the stored form
    return grid_desc(p.nx, p.ny, p.dx, p.dt, p.bc, compute, storage, p.x0, p.y0, p.phi_ref)


def _bytes_needed(p, compute, storage) -> int:
    return workspace_bytes(_desc(p, compute, storage))


def _batch_bytes(problems, compute, storage) -> int:
    """Device bytes of the batch tables (descriptors, tiles, step table, reduction
    scratch) for a batch of these problems."""
    return batch_workspace_bytes([_desc(p, compute, storage) for p in problems]) if problems else 0


class _Member:
    """A request admitted to the device."""
    __slots__ = ("rid", "arrival", "admitted", "lat", "need", "steps", "p", "retired", "last_batch")

    def __init__(self, rid, arrival, admitted, lat, need, p):
        self.rid, self.arrival, self.admitted, self.lat, self.need, self.p = rid, arrival, admitted, lat, need, p
        self.steps = 0            # steps queued so far (slices in flight included)
        self.retired = False
        self.last_batch = None    # the batch of the last slice that included it


class _Slice:
    __slots__ = ("batch", "members", "steps_after", "ev0", "ev1", "flags", "resid")


class Server:
    """Continuous batching with the host work taken off the device's critical path.

    Two slices are kept queued: slice k + 1 is launched before slice k's flags are
    read.  The batches run with freezing on, so a member that slice k flags
    (converged or non-finite) is left unchanged by slice k + 1 on the device and is
    retired exactly as it was at the end of slice k; members that reach the step
    cap are left out of the next slice when it is queued.  While slices run, the
    server admits arriving requests (their lattices are created and initialised on
    a separate stream) and collects the phi copies of retired members; a new
    membership's batch is built and its slice graph captured before its first
    slice is queued, also while the device works on the queued slices."""

    def __init__(self, budget_bytes: float = 150e9, slice_steps: int = 100, max_steps: int = 20000,
                 tol: float = 1e-8, compute: str = "f32", storage: str = "f16",
                 max_active: int = 4096, stream=None, tiles=None, shift: str = "auto", depth: int = 2,
                 first_burst: int = 16):
        self.budget = float(budget_bytes)
        self.slice_steps = int(slice_steps)
        self.max_steps = int(max_steps)
        self.tol = float(tol)
        self.compute, self.storage, self.shift = compute, storage, shift
        self.max_active = max_active
        self.depth_limit = max(1, int(depth))   # slices queued at once
        self.first_burst = max(1, int(first_burst))   # admissions before the first slice of a busy period
        self.cuda = torch.cuda.is_available()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        # admissions and retirement copies run here, beside the slices
        self.side = torch.cuda.Stream() if self.cuda else None
        self.tiles = tiles
        self.stats = dict(slices=0, rebuilds=0, peak_active=0, peak_bytes=0, rejected=0, tol_hits=0,
                          cap_hits=0, unstable=0, gpu_busy_s=0.0, admit_s=0.0, rebuild_s=0.0, span_s=0.0,
                          wait_s=0.0)
        self.depth = []        # (t, members of the slice, waiting) at every slice read
        self._bufs = []        # free (flags, residuals) result buffers

    def run(self, trace) -> List[Result]:
        """trace: list of (arrival_seconds, problem), arrival-sorted.  Runs in real
        time: a request becomes visible once the wall clock passes its arrival.

        Admission counts every resident lattice's workspace and the batch tables of
        the membership it would join; a request that needs more than the whole
        budget on its own is rejected (status "rejected").  A request admitted while
        slices run joins the next slice queued.  The stats record the device's busy
        time (CUDA events around every slice), the host time spent admitting,
        rebuilding batches (with the graph capture) and waiting on the device with
        nothing else to do, and how many requests stopped at the tolerance or at
        the step cap."""
        self._t0 = time.perf_counter()
        self._pending = deque((i, a, p) for i, (a, p) in enumerate(trace))
        self._waiting = deque()
        self._active: List[_Member] = []     # resident, not retired
        self._staged: List[_Member] = []     # admitted, joining at the next slice queued
        self._draining = []                  # (Result, pinned phi, event, member): phi copy in flight
        self._zombies: List[_Member] = []    # retired, phi taken, waiting for their batches to close
        self._used = 0.0
        self._results: List[Result] = []
        inflight = deque()
        batch, batch_members = None, []
        old_batches = []                     # replaced batches, closed once their slices are read
        st = self.stats
        while (self._pending or self._waiting or self._active or self._staged or inflight
               or self._draining or self._zombies):
            # with nothing running, admit a first group only and start the device on it;
            # the rest are admitted while its slices run
            self._admit(None if inflight else self.first_burst)
            # keep depth_limit slices queued
            while len(inflight) < self.depth_limit:
                if self._staged:
                    if self.side is not None:
                        self.side.synchronize()      # the new lattices are initialised
                    self._active.extend(self._staged)
                    self._staged = []
                runnable = [m for m in self._active if m.steps < self.max_steps]
                if not runnable:
                    break
                if batch is None or runnable != batch_members:
                    tr = time.perf_counter()
                    if batch is not None:
                        old_batches.append(batch)
                    batch = Batch([m.lat for m in runnable], stream=self.stream)
                    batch_members = runnable
                    if self.tiles:
                        batch.set_tiles(*self.tiles)
                    batch.set_freeze(True)
                    batch.prepare(self.slice_steps)  # the graph capture, before the slice's events
                    st["rebuilds"] += 1
                    st["rebuild_s"] += time.perf_counter() - tr
                inflight.append(self._queue(batch, runnable))
                st["peak_active"] = max(st["peak_active"], len(runnable))
            if not inflight:
                self._drain(block=True)
                self._bury(old_batches, batch)
                if self._pending and not self._waiting:   # idle until the next arrival
                    time.sleep(max(0.0, min(0.002, self._pending[0][1] - self._now())))
                continue
            sl = inflight.popleft()
            # host work while the oldest slice runs
            tw = time.perf_counter()
            while not _done(sl.ev1):
                busy = self._drain(block=False)
                busy = self._admit() or busy
                if not busy:
                    time.sleep(0.0002)
            st["wait_s"] += time.perf_counter() - tw
            self._read(sl)
            if batch is not None and not any(not m.retired for m in batch_members):
                old_batches.append(batch)
                batch, batch_members = None, []
            self._bury(old_batches, batch, inflight)
        self._bury(old_batches + ([batch] if batch is not None else []), None)
        st["span_s"] = self._now()
        self._results.sort(key=lambda r: r.rid)
        return self._results

    _t0 = 0.0

    def _now(self) -> float:
        return time.perf_counter() - self._t0

    def _buffers(self, n: int):
        """A free (flags, residuals) pair of at least n entries: pinned host memory
        on a GPU, numpy otherwise."""
        for k, (f, r) in enumerate(self._bufs):
            if len(f) >= n:
                return self._bufs.pop(k)
        m = max(n, 256)
        if self.cuda:
            return (torch.empty(m, dtype=torch.int32, pin_memory=True),
                    torch.empty(m, dtype=torch.float64, pin_memory=True))
        return np.zeros(m, dtype=np.int32), np.zeros(m, dtype=np.float64)

    def _queue(self, batch, members) -> _Slice:
        sl = _Slice()
        sl.batch, sl.members = batch, members
        sl.flags, sl.resid = self._buffers(len(members))
        n = len(members)
        sl.ev0, sl.ev1 = _event(), _event()
        _record(sl.ev0, self.stream)
        # the slice, then the tolerance test and non-finite check on the device
        batch.step_tol(self.slice_steps, self.tol, out=sl.flags[:n], resid_out=sl.resid[:n])
        _record(sl.ev1, self.stream)
        for m in members:
            m.steps += self.slice_steps
            m.last_batch = batch
        sl.steps_after = [m.steps for m in members]
        return sl

    def _read(self, sl: _Slice):
        """The slice has finished: retire the members it flagged (frozen since on the
        device) and those at the step cap (left out of the slices queued since)."""
        st = self.stats
        n = len(sl.members)
        flags = _host(sl.flags)[:n].copy()
        res = _host(sl.resid)[:n].copy()
        self._bufs.append((sl.flags, sl.resid))
        st["gpu_busy_s"] += _elapsed_s(sl.ev0, sl.ev1)
        st["slices"] += 1
        self.depth.append((round(self._now(), 4), n, len(self._waiting) + len(self._pending)))
        for i, m in enumerate(sl.members):
            f = int(flags[i])
            if m.retired or f & 4:
                continue
            steps = sl.steps_after[i]
            if f & 3 or steps >= self.max_steps:
                status = "unstable" if f & 2 else "done"
                if status == "unstable":
                    st["unstable"] += 1
                elif f & 1:
                    st["tol_hits"] += 1
                else:
                    st["cap_hits"] += 1
                if f & 3:
                    m.lat.settle()   # its step count back to the end of this slice
                m.retired = True
                m.steps = steps
                self._active.remove(m)
                self._retire(m, float(res[i]), status)

    def _admit(self, limit: Optional[int] = None) -> bool:
        """Moves arrived requests to the waiting queue and admits them (at most
        `limit` of them) while the budget allows; their lattices are created and
        initialised on the side stream.  Returns whether it admitted or rejected any."""
        now = self._now()
        while self._pending and self._pending[0][1] <= now:
            self._waiting.append(self._pending.popleft())
        if not self._waiting:
            return False
        st = self.stats
        ta = time.perf_counter()
        resident = [m.p for m in self._active] + [m.p for m in self._staged]
        acted = False
        admitted = 0
        while self._waiting and len(resident) < self.max_active and (limit is None or admitted < limit):
            rid, arr, p = self._waiting[0]
            need = _bytes_needed(p, self.compute, self.storage)
            if need + _batch_bytes([p], self.compute, self.storage) > self.budget:
                self._waiting.popleft()      # can never fit: reject rather than break the budget
                self._results.append(Result(rid, arr, now, self._now(), 0, float("nan"), None, "rejected"))
                st["rejected"] += 1
                acted = True
                continue
            tables = _batch_bytes(resident + [p], self.compute, self.storage)
            if self._used + need + tables > self.budget:
                break
            self._waiting.popleft()
            self._staged.append(_Member(rid, arr, self._now(), self._create(p), need, p))
            self._used += need
            admitted += 1
            resident.append(p)
            st["peak_bytes"] = max(st["peak_bytes"], self._used + tables)
            acted = True
        st["admit_s"] += time.perf_counter() - ta
        return acted

    def _create(self, p):
        if self.side is None:
            lat = Lattice.from_problem(p, compute=self.compute, storage=self.storage,
                                       stream=self.stream, shift=self.shift)
            return lat.init(p.phi0(), t0=p.t0)
        with torch.cuda.stream(self.side):
            lat = Lattice.from_problem(p, compute=self.compute, storage=self.storage,
                                       stream=self.side, shift=self.shift)
            phi0 = torch.from_numpy(np.ascontiguousarray(p.phi0(), dtype=np.float64)).pin_memory()
            lat.init(phi0.to(lat.device, non_blocking=True), t0=p.t0)
        return lat

    def _retire(self, m: _Member, residual: float, status: str):
        """Queues the member's phi copy on the side stream (the slice that last
        changed it has finished; later slices leave it frozen); the result is
        recorded once the copy has landed."""
        r = Result(m.rid, m.arrival, m.admitted, 0.0, m.steps, residual, None, status)
        if self.side is None:
            r.phi = m.lat.phi_host()
            r.finished = self._now()
            self._results.append(r)
            self._zombies.append(m)
            return
        with torch.cuda.stream(self.side):
            d = m.lat.phi(dtype=torch.float64)
            h = torch.empty(d.shape, dtype=torch.float64, pin_memory=True)
            h.copy_(d, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.side)
        self._draining.append((r, h, ev, m))

    def _drain(self, block: bool) -> bool:
        """Records the results whose phi copies have landed; True if any did."""
        keep, done = [], False
        for r, h, ev, m in self._draining:
            if block or ev.query():
                ev.synchronize()
                r.phi = h.numpy().copy()
                r.finished = self._now()
                self._results.append(r)
                self._zombies.append(m)
                done = True
            else:
                keep.append((r, h, ev, m))
        self._draining = keep
        return done

    def _bury(self, old_batches, current, inflight=()):
        """Closes replaced batches that no queued slice uses, then the retired
        lattices whose batches are all closed (their memory leaves the budget)."""
        live = {id(s.batch) for s in inflight}
        for b in list(old_batches):
            if b is not current and id(b) not in live:
                b.close()
                b.server_closed = True
                old_batches.remove(b)
        keep = []
        for m in self._zombies:
            if m.last_batch is None or getattr(m.last_batch, "server_closed", False):
                m.lat.close()
                self._used -= m.need
            else:
                keep.append(m)
        self._zombies = keep

    def idle_fraction(self) -> float:
        """Share of the run's wall time in which no slice was running on the device."""
        span = self.stats["span_s"]
        return 0.0 if span <= 0 else max(0.0, 1.0 - self.stats["gpu_busy_s"] / span)


def _host(buf):
    return buf.numpy() if isinstance(buf, torch.Tensor) else np.asarray(buf)


def _done(ev) -> bool:
    return ev is None or ev.query()


def _event():
    return torch.cuda.Event(enable_timing=True) if torch.cuda.is_available() else None


def _record(ev, stream):
    if ev is not None:
        ev.record(stream)


def _elapsed_s(e0, e1) -> float:
    return 0.0 if e0 is None else e0.elapsed_time(e1) * 1e-3


def serve_sequential(trace, slice_steps: int = 100, max_steps: int = 20000, tol: float = 1e-8,
                     compute: str = "f32", storage: str = "f16", stream=None,
                     shift: str = "auto") -> List[Result]:
    """Plain baseline: one request at a time in arrival order, plain per-step
    launches, the same residual check every slice_steps steps."""
    stream = stream if stream is not None else torch.cuda.current_stream()
    t0 = time.perf_counter()
    results = []
    for rid, (arr, p) in enumerate(trace):
        now = time.perf_counter() - t0
        if now < arr:
            time.sleep(arr - now)
        adm = time.perf_counter() - t0
        lat = Lattice.from_problem(p, compute=compute, storage=storage, stream=stream, shift=shift)
        lat.init(p.phi0(), t0=p.t0)
        steps, r, status = 0, float("inf"), "done"
        while True:
            r = lat.step_residual(slice_steps)
            steps += slice_steps
            if lat.flags() & 1:
                status = "unstable"
                break
            if r < tol or steps >= max_steps:
                break
        phi = lat.phi_host()
        results.append(Result(rid, arr, adm, time.perf_counter() - t0, steps, r, phi, status))
        del lat
    return results


def poisson_trace(problems, rate: float, seed: int = 0):
    """Arrival times of a Poisson process of the given rate (requests/s)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(problems)))
    return [(float(a), p) for a, p in zip(t, problems)]


def depth_series(depth, points: int = 16) -> list:
    """Queue depth over time, thinned to about `points` samples: [t, active, waiting]."""
    if not depth:
        return []
    stride = max(1, len(depth) // points)
    out = [list(d) for d in depth[::stride]]
    if out[-1] != list(depth[-1]):
        out.append(list(depth[-1]))
    return out


def summarize(results: List[Result]) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    return {"requests": len(results), "solves_per_s": round(len(results) / span, 3),
            "p50_s": round(float(np.percentile(lat, 50)), 4),
            "p99_s": round(float(np.percentile(lat, 99)), 4),
            "mean_steps": round(float(np.mean([r.steps for r in results])), 1),
            "span_s": round(span, 3)}
