"""Continuous-batching solve server for B-TriRT lattices.

Requests (lattice problems) arrive over time.  The server admits them while the
device-memory budget allows, keeps every admitted lattice resident, and
advances all active lattices together in slices of ``slice_steps`` steps with
one batched launch (a CUDA graph) per slice (:class:`~.lattice.Batch`).  The
device computes each member's steady-state residual ||phi^{n+1} - phi^n||_2 in
the slice's last step and compares it with the tolerance; at every slice
boundary the server reads those flags, retires the members that converged
(residual < tol), went non-finite or reached ``max_steps``,
copies their phi to the host, frees their memory and admits waiting requests.
Requests that arrive while others run therefore join at the next boundary and
share the device with them.

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


class Server:
    def __init__(self, budget_bytes: float = 150e9, slice_steps: int = 100, max_steps: int = 20000,
                 tol: float = 1e-8, compute: str = "f32", storage: str = "f16",
                 max_active: int = 4096, stream=None, tiles=None, shift: str = "auto"):
        self.budget = float(budget_bytes)
        self.slice_steps = int(slice_steps)
        self.max_steps = int(max_steps)
        self.tol = float(tol)
        self.compute, self.storage, self.shift = compute, storage, shift
        self.max_active = max_active
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.tiles = tiles
        self.stats = dict(slices=0, rebuilds=0, peak_active=0, peak_bytes=0, rejected=0, tol_hits=0,
                          cap_hits=0, unstable=0, gpu_busy_s=0.0, admit_s=0.0, rebuild_s=0.0, span_s=0.0)
        self.depth = []        # (t, active, waiting) at every slice
        self._flags = None     # pinned stop flags, see _flag_buffer

    def run(self, trace) -> List[Result]:
        """trace: list of (arrival_seconds, problem), arrival-sorted.  Runs in real
        time: a request becomes visible once the wall clock passes its arrival.

        Admission counts every active lattice's workspace and the batch tables of
        the membership it would join; a request that needs more than the whole
        budget on its own is rejected (status "rejected").  The stats record the
        device's busy time (CUDA events around every slice), the host time spent
        admitting and rebuilding batches, and how many requests stopped at the
        tolerance or at the step cap."""
        t0 = time.perf_counter()
        pending = deque((i, a, p) for i, (a, p) in enumerate(trace))
        waiting = deque()
        active = []            # [rid, arrival, admitted, lattice, bytes, steps, problem]
        used = 0.0
        results: List[Result] = []
        batch: Optional[Batch] = None
        dirty = True
        st = self.stats
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0][1] <= now:
                waiting.append(pending.popleft())
            # admission by memory budget (and a cap on members)
            ta = time.perf_counter()
            while waiting and len(active) < self.max_active:
                rid, arr, p = waiting[0]
                need = _bytes_needed(p, self.compute, self.storage)
                if need + _batch_bytes([p], self.compute, self.storage) > self.budget:
                    waiting.popleft()      # can never fit: reject rather than break the budget
                    results.append(Result(rid, arr, now, time.perf_counter() - t0, 0, float("nan"), None,
                                          "rejected"))
                    st["rejected"] += 1
                    continue
                tables = _batch_bytes([a[6] for a in active] + [p], self.compute, self.storage)
                if used + need + tables > self.budget:
                    break
                waiting.popleft()
                lat = Lattice.from_problem(p, compute=self.compute, storage=self.storage,
                                           stream=self.stream, shift=self.shift)
                lat.init(p.phi0(), t0=p.t0)
                used += need
                active.append([rid, arr, time.perf_counter() - t0, lat, need, 0, p])
                dirty = True
            st["admit_s"] += time.perf_counter() - ta
            st["peak_active"] = max(st["peak_active"], len(active))
            tables = _batch_bytes([a[6] for a in active], self.compute, self.storage)
            st["peak_bytes"] = max(st["peak_bytes"], used + tables)
            if not active:
                if pending:   # idle until the next arrival
                    time.sleep(max(0.0, min(0.002, pending[0][1] - (time.perf_counter() - t0))))
                continue
            if dirty:
                tr = time.perf_counter()
                if batch is not None:
                    batch.close()
                batch = Batch([a[3] for a in active], stream=self.stream)
                if self.tiles:
                    batch.set_tiles(*self.tiles)
                st["rebuilds"] += 1
                st["rebuild_s"] += time.perf_counter() - tr
                dirty = False
            ev0, ev1 = _event(), _event()
            _record(ev0, self.stream)
            # the slice, then the tolerance test and non-finite check on the device
            ft = batch.step_tol(self.slice_steps, self.tol, out=self._flag_buffer(len(active)))
            _record(ev1, self.stream)
            res = batch.residuals()          # synchronises: the flags have landed too
            flags = ft.numpy().copy() if isinstance(ft, torch.Tensor) else np.asarray(ft)
            st["gpu_busy_s"] += _elapsed_s(ev0, ev1)
            bad = flags & 2                  # non-finite phi in that member only
            st["slices"] += 1
            self.depth.append((round(time.perf_counter() - t0, 4), len(active), len(waiting) + len(pending)))
            done_idx = []
            for k, a in enumerate(active):
                a[5] += self.slice_steps
                if bad[k] or (flags[k] & 1) or a[5] >= self.max_steps:
                    done_idx.append(k)
            if done_idx:
                for k in reversed(done_idx):
                    rid, arr, adm, lat, need, steps, _ = active[k]
                    phi = lat.phi_host()
                    status = "unstable" if bad[k] else "done"
                    if status == "unstable":
                        st["unstable"] += 1
                    elif flags[k] & 1:
                        st["tol_hits"] += 1
                    else:
                        st["cap_hits"] += 1
                    results.append(Result(rid, arr, adm, time.perf_counter() - t0, steps,
                                          float(res[k]), phi, status))
                    used -= need
                    del active[k]
                batch.close()
                batch = None
                dirty = True
        if batch is not None:
            batch.close()
        st["span_s"] = time.perf_counter() - t0
        results.sort(key=lambda r: r.rid)
        return results

    def _flag_buffer(self, n: int):
        """Pinned host memory for the per-member stop flags of a slice (reused)."""
        if not torch.cuda.is_available():
            return None
        if self._flags is None or self._flags.numel() < n:
            self._flags = torch.empty(max(n, 256), dtype=torch.int32, pin_memory=True)
        return self._flags[:n]

    def idle_fraction(self) -> float:
        """Share of the run's wall time in which no slice was running on the device."""
        span = self.stats["span_s"]
        return 0.0 if span <= 0 else max(0.0, 1.0 - self.stats["gpu_busy_s"] / span)


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
