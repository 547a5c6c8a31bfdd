"""Python binding of one D3Q19 lattice: argument marshalling around the C ABI of
include/btrt3.h.  PyTorch provides the device workspace and the stream; every
step runs in libbtrt's kernels."""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _capi as C

_K2 = {"hbb": C.K2_HBB, "const": C.K2_CONST}
_SRC = {"none": C.SRC_NONE, "const": C.SRC_CONST, "field": C.SRC_FIELD, "reaction": C.SRC_REACTION}


def grid_desc3(nx, ny, nz, dx, dt, bc=(0,) * 6, compute="f64", storage="f64", x0=0.0, y0=0.0, z0=0.0,
               phi_ref=0.0, fields=0, shift="ref") -> C.GridDesc3:
    g = C.GridDesc3()
    g.nx, g.ny, g.nz = int(nx), int(ny), int(nz)
    for k in range(6):
        g.bc[k] = int(bc[k])
    g.compute, g.storage = C.FORMATS[compute], C.FORMATS[storage]
    g.shift = C.SHIFTS[shift]
    g.fields = int(fields)
    g.dx, g.dt, g.x0, g.y0, g.z0, g.phi_ref = float(dx), float(dt), float(x0), float(y0), float(z0), float(phi_ref)
    return g


def coeffs3(p) -> C.Coeffs3:
    """Coefficients of a workloads.Problem3-like object."""
    c = C.Coeffs3()
    for k in range(3):
        c.u[k] = float(p.u[k])
        c.b_dir[k] = float(p.b_dir[k])
    c.b2, c.b_q, c.c3, c.a2, c.k0 = float(p.b2), float(p.b_q), float(p.c3), float(p.a2), float(p.k0)
    for k in range(6):
        c.A0[k] = float(p.A0[k])
        c.wall[k] = float(p.wall[k])
    c.k2_mode = _K2[p.k2_mode]
    c.k2 = float(p.k2)
    src = p.source
    c.src_kind = _SRC[src.kind]
    if src.kind == "const":
        c.src_const = float(src.const)
    elif src.kind == "field":
        c.src_lam = float(src.lam)
    elif src.kind == "reaction":
        c.react_rate, c.react_exp = float(src.const), float(src.exp)
    c.wall_lam = float(p.wall_lam)
    return c


class Lattice3:
    """One B-TriRT D3Q19 lattice resident on the GPU."""

    def __init__(self, desc: C.GridDesc3, coef: C.Coeffs3, device=None, stream=None,
                 workspace: Optional[torch.Tensor] = None, src_field=None):
        self.lib = C.load()
        self.desc, self.coef = desc, coef
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = self.lib.btrt3_workspace_bytes(ctypes.byref(desc))
        if nbytes == 0:
            raise C.BtrtError(C.EINVAL, self.lib.btrt_last_error().decode())
        if workspace is None:
            workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        self.workspace = workspace
        h = ctypes.c_void_p()
        C.check(self.lib.btrt3_create(ctypes.byref(desc), ctypes.c_void_p(workspace.data_ptr()), int(nbytes),
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.handle = h
        if src_field is not None:
            a = np.ascontiguousarray(src_field, dtype=np.float64)
            assert a.shape == (desc.nz, desc.ny, desc.nx)
            C.check(self.lib.btrt3_set_source_field(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        C.check(self.lib.btrt3_set_coeffs(self.handle, ctypes.byref(coef)))

    @classmethod
    def from_problem(cls, p, compute="f64", storage=None, device=None, stream=None, shift="auto") -> "Lattice3":
        storage = storage or compute
        if shift == "auto":
            shift = "local" if storage in ("f16", "bf16") else "ref"
        fields = C.FIELD_SOURCE if p.src_field is not None else 0
        desc = grid_desc3(p.nx, p.ny, p.nz, p.dx, p.dt, p.bc, compute, storage, p.x0, p.y0, p.z0, p.phi_ref,
                          fields, shift)
        return cls(desc, coeffs3(p), device=device, stream=stream, src_field=p.src_field)

    @property
    def shape(self):
        return (self.desc.nz, self.desc.ny, self.desc.nx)

    @property
    def real_dtype(self):
        return torch.float32 if self.desc.compute == C.F32 else torch.float64

    def init(self, phi0, t0: float = 0.0):
        if isinstance(phi0, np.ndarray):
            a = np.ascontiguousarray(phi0, dtype=np.float64)
            assert a.shape == self.shape
            C.check(self.lib.btrt3_init_phi(self.handle, ctypes.c_void_p(a.ctypes.data), C.F64, 0, float(t0)))
            return self
        t = phi0.contiguous()
        if t.dtype not in (torch.float64, torch.float32):
            t = t.double()
        assert tuple(t.shape) == self.shape
        code = C.F64 if t.dtype == torch.float64 else C.F32
        C.check(self.lib.btrt3_init_phi(self.handle, ctypes.c_void_p(t.data_ptr()), code,
                                        1 if t.is_cuda else 0, float(t0)))
        if t.is_cuda:
            self._keep = t
        return self

    def step(self, nsteps: int = 1):
        C.check(self.lib.btrt3_step(self.handle, int(nsteps)))
        return self

    def phi(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.shape, dtype=self.real_dtype, device=self.device)
        code = C.F64 if out.dtype == torch.float64 else C.F32
        C.check(self.lib.btrt3_read_phi(self.handle, ctypes.c_void_p(out.data_ptr()), code,
                                        1 if out.is_cuda else 0))
        return out

    def phi_host(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        C.check(self.lib.btrt3_read_phi(self.handle, ctypes.c_void_p(out.ctypes.data), C.F64, 0))
        return out

    def read_f(self, x0=0, y0=0, z0=0, w=None, h=None, d=None) -> np.ndarray:
        w = self.desc.nx - x0 if w is None else w
        h = self.desc.ny - y0 if h is None else h
        d = self.desc.nz - z0 if d is None else d
        out = np.empty((19, d, h, w), dtype=np.float64)
        C.check(self.lib.btrt3_read_f(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      x0, y0, z0, w, h, d))
        return out

    def mass(self) -> float:
        v = ctypes.c_double()
        C.check(self.lib.btrt3_mass(self.handle, ctypes.byref(v)))
        return v.value

    def flags(self) -> int:
        """Device flags without raising (bit 0: non-finite phi, bit 3: debug index check)."""
        f = ctypes.c_int32()
        self.lib.btrt3_check(self.handle, ctypes.byref(f))
        return f.value

    def check(self) -> int:
        f = ctypes.c_int32()
        C.check(self.lib.btrt3_check(self.handle, ctypes.byref(f)))
        return f.value

    def time(self):
        s, t = ctypes.c_int64(), ctypes.c_double()
        C.check(self.lib.btrt3_get_time(self.handle, ctypes.byref(s), ctypes.byref(t)))
        return s.value, t.value

    def save(self) -> bytes:
        n = self.lib.btrt3_state_bytes(self.handle)
        buf = ctypes.create_string_buffer(n)
        C.check(self.lib.btrt3_save(self.handle, buf, n))
        return buf.raw

    def load(self, state: bytes):
        buf = ctypes.create_string_buffer(state, len(state))
        C.check(self.lib.btrt3_load(self.handle, buf, len(state)))
        return self

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.btrt3_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
