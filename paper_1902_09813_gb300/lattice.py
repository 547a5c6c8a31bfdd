"""Python binding of one lattice: argument marshalling around the C ABI.

PyTorch provides the device workspace and the CUDA stream; every step of the
sweep runs in libbtrt's kernels.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _capi as C

_K2 = {"hbb": C.K2_HBB, "const": C.K2_CONST}
_SRC = {"none": C.SRC_NONE, "const": C.SRC_CONST, "trig": C.SRC_TRIG, "field": C.SRC_FIELD,
        "reaction": C.SRC_REACTION}


def grid_desc(nx, ny, dx, dt, bc=(0, 0, 0, 0), compute="f64", storage="f64",
              x0=0.0, y0=0.0, phi_ref=0.0, fields=0, shift="ref") -> C.GridDesc:
    g = C.GridDesc()
    g.nx, g.ny = int(nx), int(ny)
    for k in range(4):
        g.bc[k] = int(bc[k])
    g.compute, g.storage = C.FORMATS[compute], C.FORMATS[storage]
    g.dx, g.dt, g.x0, g.y0, g.phi_ref = float(dx), float(dt), float(x0), float(y0), float(phi_ref)
    g.fields = int(fields)
    g.shift = C.SHIFTS[shift]
    return g


def coeffs(u=(0.0, 0.0), b2=0.0, c3=0.0, A0=(0.0, 0.0, 0.0), a2=0.0, k0=1.0, k2_mode="hbb",
           k2=1.0, source=None, wall_lam=0.0, b_dir=(1.0, 1.0), b_q=2.0) -> C.Coeffs:
    c = C.Coeffs()
    c.u[0], c.u[1] = float(u[0]), float(u[1])
    c.b2, c.c3, c.a2, c.k0 = float(b2), float(c3), float(a2), float(k0)
    for k in range(3):
        c.A0[k] = float(A0[k])
    c.k2_mode = _K2[k2_mode]
    c.k2 = float(k2)
    if source is not None:
        c.src_kind = _SRC[source.kind]
        c.src_const, c.src_lam, c.src_k = float(source.const), float(source.lam), float(source.k)
        for k in range(4):
            c.src_alpha[k] = float(source.alpha[k])
        if source.kind == "reaction":
            c.react_rate, c.react_exp = float(source.const), float(source.exp)
    c.wall_lam = float(wall_lam)
    c.b_dir[0], c.b_dir[1] = float(b_dir[0]), float(b_dir[1])
    c.b_q = float(b_q)
    return c


def workspace_bytes(desc: C.GridDesc) -> int:
    n = C.load().btrt_workspace_bytes(ctypes.byref(desc))
    if n == 0:
        raise C.BtrtError(C.EINVAL, C.load().btrt_last_error().decode())
    return int(n)


def batch_workspace_bytes(descs) -> int:
    """Device bytes of the batch tables for lattices with these grid descriptions."""
    arr = (C.GridDesc * len(descs))(*descs)
    n = C.load().btrt_batch_workspace_bytes_desc(arr, len(descs))
    if n == 0:
        raise C.BtrtError(C.EINVAL, C.load().btrt_last_error().decode())
    return int(n)


class Lattice:
    """One B-TriRT D2Q9 lattice resident on the GPU.

    Build it with :meth:`from_problem` (any object with the attributes of
    ``workloads.Problem``) or from a :class:`GridDesc` and :class:`Coeffs`.
    """

    def __init__(self, desc: C.GridDesc, coef: C.Coeffs, device=None, stream=None,
                 workspace: Optional[torch.Tensor] = None, defer_coeffs: bool = False):
        self.lib = C.load()
        self.desc = desc
        self.coef = coef
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = workspace_bytes(desc)
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        elif workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError("workspace too small")
        self.workspace = workspace
        h = ctypes.c_void_p()
        C.check(self.lib.btrt_create(ctypes.byref(desc), ctypes.c_void_p(workspace.data_ptr()),
                                     nbytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.handle = h
        if not defer_coeffs:
            C.check(self.lib.btrt_set_coeffs(self.handle, ctypes.byref(coef)))

    # ------------------------------------------------------------ construction
    @classmethod
    def from_problem(cls, p, compute="f64", storage=None, device=None, stream=None,
                     phi_ref=None, shift="auto") -> "Lattice":
        """shift: stored form of F32/F16/BF16 populations -- "ref" (f - w_i phi_ref),
        "local" (f^+ - w_i phi of the writing node), "local_dw" (local, with phi kept
        as a double-word pair so that it is never rounded to FP32; plain kernel form),
        "local_sr" (local, F16/BF16 storage rounded stochastically; plain and vector
        forms), "local_dw_sr" (both; plain form), "moment_sr" (F16/BF16: the writer's
        first-moment term subtracted as well, j kept in two more planes, stochastic
        rounding; plain and vector forms) or "auto" (local for the 16-bit
        formats, whose rounding it keeps well below the discretisation error; ref for
        FP32 storage)."""
        storage = storage or compute
        if shift == "auto":
            shift = "local" if storage in ("f16", "bf16") else "ref"
        src_field = getattr(p, "src_field", None)
        A_field = getattr(p, "A_field", None)
        fields = (C.FIELD_SOURCE if src_field is not None else 0) | \
                 (C.FIELD_DIFFUSION if A_field is not None else 0)
        desc = grid_desc(p.nx, p.ny, p.dx, p.dt, p.bc, compute, storage, p.x0, p.y0,
                         p.phi_ref if phi_ref is None else phi_ref, fields, shift)
        coef = coeffs(p.u, p.b2, p.c3, p.A0, p.a2, p.k0, p.k2_mode, p.k2, p.source,
                      getattr(p, "wall_lam", 0.0), getattr(p, "b_dir", (1.0, 1.0)), getattr(p, "b_q", 2.0))
        lat = cls(desc, coef, device=device, stream=stream, defer_coeffs=True)
        if src_field is not None:
            lat.set_source_field(src_field)
        if A_field is not None:
            lat.set_diffusion_field(*A_field)
        C.check(lat.lib.btrt_set_coeffs(lat.handle, ctypes.byref(coef)))
        wall_fn_arrs = p.wall_arrays_at(p.t0 + p.dt) if getattr(p, "wall_fn", None) is not None else None
        for side in range(4):
            arrs = getattr(p, "wall_arrays", None)
            if wall_fn_arrs is not None:
                lat.set_boundary(side, wall_fn_arrs[side])
            elif arrs is not None and arrs[side] is not None:
                lat.set_boundary(side, arrs[side])
            else:
                lat.set_boundary(side, [p.wall[side]])
        return lat

    def step_walls(self, p, nsteps: int = 1):
        """Advance nsteps with wall values re-evaluated from p.wall_fn before every
        step (at the step's end time, as the bounce-back rule takes them)."""
        for _ in range(nsteps):
            _, t = self.time()
            for side, v in enumerate(p.wall_arrays_at(t + p.dt)):
                self.set_boundary(side, v)
            self.step(1)
        return self

    @property
    def nx(self):
        return self.desc.nx

    @property
    def ny(self):
        return self.desc.ny

    @property
    def real_dtype(self):
        return torch.float32 if self.desc.compute == C.F32 else torch.float64

    def set_boundary(self, side: int, values):
        v = np.ascontiguousarray(np.atleast_1d(np.asarray(values, dtype=np.float64)))
        C.check(self.lib.btrt_set_boundary(self.handle, side,
                                           v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), v.size))

    def set_source_field(self, F):
        a = np.ascontiguousarray(F, dtype=np.float64)
        assert a.shape == (self.ny, self.nx)
        C.check(self.lib.btrt_set_source_field(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return self

    def set_diffusion_field(self, Axx, Axy, Ayy):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (Axx, Axy, Ayy)]
        for a in arrs:
            assert a.shape == (self.ny, self.nx)
        ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs]
        C.check(self.lib.btrt_set_diffusion_field(self.handle, *ptrs))
        return self

    def set_sweep_variant(self, variant: str):
        """Kernel form of an FP32-compute lattice: 'auto', 'plain', 'tma' (TMA-staged
        tiles), 'tb2' (two steps per launch), 'vec' (one step per launch with
        vector loads and stores of four x-consecutive nodes per thread) or 'tb2v'
        (two steps per launch with the vector access in both)."""
        code = {"auto": C.SWEEP_AUTO, "plain": C.SWEEP_PLAIN, "tma": C.SWEEP_TMA, "tb2": C.SWEEP_TB2,
                "vec": C.SWEEP_VEC, "tb2v": C.SWEEP_TB2V}[variant]
        C.check(self.lib.btrt_set_sweep_variant(self.handle, code))
        return self

    def set_coeffs(self, coef: C.Coeffs):
        self.coef = coef
        C.check(self.lib.btrt_set_coeffs(self.handle, ctypes.byref(coef)))

    # ------------------------------------------------------------ state
    def init(self, phi0, t0: float = 0.0):
        """f = f_eq(phi0).  phi0: numpy array (host) or torch tensor (host or device),
        float64 or float32, shape (ny, nx)."""
        if isinstance(phi0, np.ndarray):
            a = np.ascontiguousarray(phi0)
            if a.dtype not in (np.float64, np.float32):
                a = a.astype(np.float64)
            assert a.shape == (self.ny, self.nx)
            dt = C.F64 if a.dtype == np.float64 else C.F32
            C.check(self.lib.btrt_init_phi(self.handle, ctypes.c_void_p(a.ctypes.data), dt, 0, float(t0)))
            return self
        t = phi0.contiguous()
        if t.dtype not in (torch.float64, torch.float32):
            t = t.double()
        assert tuple(t.shape) == (self.ny, self.nx)
        dt = C.F64 if t.dtype == torch.float64 else C.F32
        C.check(self.lib.btrt_init_phi(self.handle, ctypes.c_void_p(t.data_ptr()), dt,
                                       1 if t.is_cuda else 0, float(t0)))
        if t.is_cuda:
            self._keep = t   # the copy is asynchronous on the stream
        return self

    def step(self, nsteps: int = 1):
        C.check(self.lib.btrt_step(self.handle, int(nsteps)))
        return self

    def step_residual(self, nsteps: int = 1) -> float:
        """Advance nsteps and return ||phi^n - phi^{n-1}||_2 of the last step."""
        r = ctypes.c_double()
        C.check(self.lib.btrt_step_residual(self.handle, int(nsteps), ctypes.byref(r)))
        return r.value

    def phi(self, out: Optional[torch.Tensor] = None, dtype=None) -> torch.Tensor:
        """phi as a device tensor (asynchronous on the lattice stream)."""
        dtype = dtype or self.real_dtype
        if out is None:
            out = torch.empty((self.ny, self.nx), dtype=dtype, device=self.device)
        code = C.F64 if out.dtype == torch.float64 else C.F32
        C.check(self.lib.btrt_read_phi(self.handle, ctypes.c_void_p(out.data_ptr()), code,
                                       1 if out.is_cuda else 0))
        return out

    def phi_host(self, dtype=np.float64) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=dtype)
        code = C.F64 if out.dtype == np.float64 else C.F32
        C.check(self.lib.btrt_read_phi(self.handle, ctypes.c_void_p(out.ctypes.data), code, 0))
        return out

    def read_f(self, x0=0, y0=0, w=None, h=None) -> np.ndarray:
        """Post-collision populations of a window, FP64, shape (9, h, w)."""
        w = self.nx - x0 if w is None else w
        h = self.ny - y0 if h is None else h
        out = np.empty((9, h, w), dtype=np.float64)
        C.check(self.lib.btrt_read_f(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     x0, y0, w, h))
        return out

    def mass(self) -> float:
        v = ctypes.c_double()
        C.check(self.lib.btrt_mass(self.handle, ctypes.byref(v)))
        return v.value

    def settle(self, clear: bool = False) -> int:
        """The step at which a batch froze this lattice (its step count is set back
        to it), or -1 if it is not frozen.  clear: also remove the mark (only when
        no queued batch launch still includes the lattice)."""
        s = ctypes.c_int64()
        C.check(self.lib.btrt_settle(self.handle, 1 if clear else 0, ctypes.byref(s)))
        return s.value

    def check(self) -> int:
        """Raises BtrtError(EUNSTABLE) if the sweep has produced a non-finite phi."""
        flags = ctypes.c_int32()
        C.check(self.lib.btrt_check(self.handle, ctypes.byref(flags)))
        return flags.value

    def flags(self) -> int:
        """The device flags without raising (bit 0: non-finite phi, bit 2: a tile-copy wait gave up)."""
        flags = ctypes.c_int32()
        self.lib.btrt_check(self.handle, ctypes.byref(flags))
        return flags.value

    def time(self):
        s = ctypes.c_int64()
        t = ctypes.c_double()
        C.check(self.lib.btrt_get_time(self.handle, ctypes.byref(s), ctypes.byref(t)))
        return s.value, t.value

    def save(self) -> bytes:
        n = self.lib.btrt_state_bytes(self.handle)
        buf = ctypes.create_string_buffer(n)
        C.check(self.lib.btrt_save(self.handle, buf, n))
        return buf.raw

    def load(self, state: bytes):
        buf = ctypes.create_string_buffer(state, len(state))
        C.check(self.lib.btrt_load(self.handle, buf, len(state)))
        return self

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.btrt_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent lattices advanced together: one batched launch form over all
    members (persistent, one launch per step, two steps per launch or the vector
    form; set_tiles / autotune pick it), each call's launches replayed from a CUDA
    graph (see btrt_batch_* in include/btrt.h)."""

    def __init__(self, lattices, stream=None, device=None):
        self.lib = C.load()
        self.members = list(lattices)
        n = len(self.members)
        self._handles = (ctypes.c_void_p * n)(*[m.handle.value for m in self.members])
        self.device = torch.device(device if device is not None else self.members[0].device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = self.lib.btrt_batch_workspace_bytes(self._handles, n)
        if nbytes == 0:
            raise C.BtrtError(C.EINVAL, self.lib.btrt_last_error().decode())
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        C.check(self.lib.btrt_batch_create(self._handles, n, ctypes.c_void_p(self.workspace.data_ptr()),
                                           int(nbytes), ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(h)))
        self.handle = h

    def __len__(self):
        return len(self.members)

    def step(self, nsteps: int, residual: bool = False):
        C.check(self.lib.btrt_batch_step(self.handle, int(nsteps), 1 if residual else 0))
        return self

    def prepare(self, nsteps: int, residual: bool = True):
        """Capture the CUDA graphs of an nsteps-step call (step with residual, or
        step_tol) without running them; no member advances."""
        C.check(self.lib.btrt_batch_prepare(self.handle, int(nsteps), 1 if residual else 0))
        return self

    def graphs(self) -> int:
        """Slice graphs held (-1: capture failed, launches go directly)."""
        n = ctypes.c_int32()
        C.check(self.lib.btrt_batch_graphs(self.handle, ctypes.byref(n)))
        return n.value

    def step_tol(self, nsteps: int, tol: float, out: Optional[torch.Tensor] = None,
                 resid_out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Advance nsteps steps and flag, on the device, each member whose residual
        of the last step is below tol (bit 0), whose phi went non-finite (bit 1) or
        that was frozen before the call (bit 2).  The flags land in `out` (pinned
        host int32 by default) and, if given, the residuals in `resid_out` (float64,
        same memory kind) in stream order: synchronise the batch stream, or an event
        recorded after the call, before reading them."""
        if out is None:
            out = torch.empty(len(self.members), dtype=torch.int32, pin_memory=True)
        if resid_out is not None and resid_out.is_cuda != out.is_cuda:
            raise ValueError("out and resid_out must both be host or both be device tensors")
        C.check(self.lib.btrt_batch_step_tol(self.handle, int(nsteps), float(tol),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(resid_out.data_ptr() if resid_out is not None else 0),
                                             1 if out.is_cuda else 0))
        return out

    def set_freeze(self, enable: bool = True):
        """step_tol freezes the members it flags: later batch launches leave them
        unchanged (Lattice.settle restores their step counts)."""
        C.check(self.lib.btrt_batch_set_freeze(self.handle, 1 if enable else 0))
        return self

    def member_flags(self) -> np.ndarray:
        """Each member's device flags (bit 0: non-finite phi)."""
        out = np.zeros(len(self.members), dtype=np.int32)
        C.check(self.lib.btrt_batch_member_flags(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def residuals(self) -> np.ndarray:
        out = np.empty(len(self.members), dtype=np.float64)
        C.check(self.lib.btrt_batch_residuals(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def set_tiles(self, block_x: int, block_y: int, rows: int, per_step: int = 0):
        """Tile shape and launch form: per_step 0 = persistent launch per call, 1 = one
        launch per step, 2 = two steps per launch (FP32 compute), 3 = one launch per
        step in the vector form (FP32 compute)."""
        C.check(self.lib.btrt_batch_set_tiles(self.handle, block_x, block_y, rows, per_step))
        return self

    def autotune(self, steps_per_trial: int = 4):
        """Returns (block_x, block_y, rows, per_step_launch) of the fastest candidate."""
        bx, by, r, ps = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        C.check(self.lib.btrt_batch_autotune(self.handle, steps_per_trial, ctypes.byref(bx),
                                             ctypes.byref(by), ctypes.byref(r), ctypes.byref(ps)))
        return bx.value, by.value, r.value, ps.value

    def check(self) -> int:
        flags = ctypes.c_int32()
        C.check(self.lib.btrt_batch_check(self.handle, ctypes.byref(flags)))
        return flags.value

    def set_wait_limit(self, polls: int, never_release: bool = False):
        C.check(self.lib.btrt_batch_set_wait_limit(self.handle, int(polls), 1 if never_release else 0))
        return self

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.btrt_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
