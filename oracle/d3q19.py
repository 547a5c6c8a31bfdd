"""FP64 CPU oracle of the B-TriRT scheme on the D3Q19 lattice -- TEST
INFRASTRUCTURE ONLY (same rules as the package: tests, smoke and the benchmark's
CPU legs only).  ``btrt_oracle3.c`` is compiled with gcc into ``oracle/_build``
and called through ctypes; inputs come from :mod:`workloads.problems3`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "btrt_oracle3.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle3.so"
NQ = 19

_K2 = {"hbb": 0, "const": 1}
_SRC_KIND = {"none": 0, "const": 1, "field": 3, "reaction": 4}


def build(force: bool = False) -> Path:
    _BUILD.mkdir(exist_ok=True)
    if _LIB_PATH.exists() and not force and _LIB_PATH.stat().st_mtime > _SRC.stat().st_mtime:
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared",
            "-fPIC", str(_SRC), "-o", str(_LIB_PATH) + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(str(_LIB_PATH) + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Problem3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 6),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
        ("u", ctypes.c_double * 3), ("b2", ctypes.c_double), ("b_dir", ctypes.c_double * 3),
        ("b_q", ctypes.c_double), ("c3", ctypes.c_double),
        ("A0", ctypes.c_double * 6), ("a2", ctypes.c_double), ("k0", ctypes.c_double),
        ("k2_mode", ctypes.c_int32), ("src_kind", ctypes.c_int32),
        ("k2", ctypes.c_double),
        ("src_const", ctypes.c_double), ("src_lam", ctypes.c_double),
        ("react_rate", ctypes.c_double), ("react_exp", ctypes.c_double),
        ("wall", ctypes.c_double * 6), ("wall_lam", ctypes.c_double),
        ("src_field", ctypes.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        P = ctypes.POINTER(_Problem3)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        d = ctypes.c_double
        L.btrt3_oracle_B.argtypes = [P, d, dp]
        L.btrt3_oracle_C.argtypes = [P, d]
        L.btrt3_oracle_C.restype = d
        L.btrt3_oracle_K1.argtypes = [P, d, dp]
        L.btrt3_oracle_k2.argtypes = [P, dp]
        L.btrt3_oracle_k2.restype = d
        L.btrt3_oracle_feq.argtypes = [P, d, dp]
        L.btrt3_oracle_RP.argtypes = [d, dp, dp, d, dp, dp]
        L.btrt3_oracle_collide.argtypes = [P, dp, d, ctypes.c_long, d, d, dp]
        L.btrt3_oracle_init.argtypes = [P, dp, dp, dp]
        L.btrt3_oracle_phi.argtypes = [P, dp, dp]
        L.btrt3_oracle_run.argtypes = [P, dp, dp, dp, d, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        L.btrt3_oracle_lattice.argtypes = [ip, ip, ip, dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_problem(p) -> tuple:
    s = _Problem3()
    s.nx, s.ny, s.nz = p.nx, p.ny, p.nz
    for k in range(6):
        s.bc[k] = int(p.bc[k])
        s.wall[k] = p.wall[k]
    s.dx, s.dt, s.x0, s.y0, s.z0 = p.dx, p.dt, p.x0, p.y0, p.z0
    for k in range(3):
        s.u[k] = p.u[k]
        s.b_dir[k] = p.b_dir[k]
    s.b2, s.b_q, s.c3 = p.b2, p.b_q, p.c3
    for k in range(6):
        s.A0[k] = p.A0[k]
    s.a2, s.k0 = p.a2, p.k0
    s.k2_mode = _K2[p.k2_mode]
    s.k2 = p.k2
    src = p.source
    s.src_kind = _SRC_KIND[src.kind]
    s.src_const, s.src_lam = src.const, src.lam
    s.react_rate, s.react_exp = src.const, src.exp
    s.wall_lam = p.wall_lam
    keep = []
    if p.src_field is not None:
        a = np.ascontiguousarray(p.src_field, dtype=np.float64)
        assert a.shape == (p.nz, p.ny, p.nx)
        keep.append(a)
        s.src_field = a.ctypes.data
    return s, keep


class OracleLattice3:
    """State: pre-collision populations f at time t ([19, nz, ny, nx]), the last
    post-collision populations, phi_prev."""

    def __init__(self, problem, nthreads: int = 1):
        self.problem = problem
        self.s, self._keep = make_problem(problem)
        self.nthreads = nthreads
        shape = (NQ, problem.nz, problem.ny, problem.nx)
        self.f = np.zeros(shape)
        self.fpost = np.zeros(shape)
        self.phi_prev = np.zeros(shape[1:])
        self.step_index = 0
        self.t0 = problem.t0

    def init(self, phi0=None):
        phi0 = np.ascontiguousarray(self.problem.phi0() if phi0 is None else phi0, dtype=np.float64)
        lib().btrt3_oracle_init(ctypes.byref(self.s), _ptr(phi0), _ptr(self.f), _ptr(self.phi_prev))
        self.step_index = 0
        return self

    @property
    def t(self) -> float:
        return self.t0 + self.step_index * self.problem.dt

    def step(self, nsteps: int = 1):
        lib().btrt3_oracle_run(ctypes.byref(self.s), _ptr(self.f), _ptr(self.fpost), _ptr(self.phi_prev),
                               self.t0, self.step_index, nsteps, self.nthreads)
        self.step_index += nsteps
        return self

    def phi(self) -> np.ndarray:
        out = np.zeros(self.f.shape[1:])
        lib().btrt3_oracle_phi(ctypes.byref(self.s), _ptr(self.f), _ptr(out))
        return out


def lattice():
    """(c [19, 3] int array, w [19])."""
    cx, cy, cz = (ctypes.c_int * NQ)(), (ctypes.c_int * NQ)(), (ctypes.c_int * NQ)()
    w = np.zeros(NQ)
    lib().btrt3_oracle_lattice(cx, cy, cz, _ptr(w))
    return np.array([list(cx), list(cy), list(cz)]).T, w


def feq(problem, phi: float) -> np.ndarray:
    s, keep = make_problem(problem)
    out = np.zeros(NQ)
    lib().btrt3_oracle_feq(ctypes.byref(s), phi, _ptr(out))
    return out


def B(problem, phi: float) -> np.ndarray:
    s, keep = make_problem(problem)
    out = np.zeros(3)
    lib().btrt3_oracle_B(ctypes.byref(s), phi, _ptr(out))
    return out


def K1(problem, phi: float) -> np.ndarray:
    s, keep = make_problem(problem)
    out = np.zeros(9)
    lib().btrt3_oracle_K1(ctypes.byref(s), phi, _ptr(out))
    return out.reshape(3, 3)


def k2(problem, K1m) -> float:
    s, keep = make_problem(problem)
    a = np.ascontiguousarray(K1m, dtype=np.float64).reshape(9)
    return lib().btrt3_oracle_k2(ctypes.byref(s), _ptr(a))


def RP(k0: float, K1m, K2m, c: float, g) -> np.ndarray:
    """sum_j (R_ij + P_ij) g_j (Eq. 77) for general K1, K2."""
    out = np.zeros(NQ)
    k1a = np.ascontiguousarray(K1m, dtype=np.float64).reshape(9)
    k2a = np.ascontiguousarray(K2m, dtype=np.float64).reshape(9)
    ga = np.ascontiguousarray(g, dtype=np.float64)
    lib().btrt3_oracle_RP(k0, _ptr(k1a), _ptr(k2a), c, _ptr(ga), _ptr(out))
    return out


def collide(problem, f, phi_prev: float, node: int, t: float, t_prev: float) -> np.ndarray:
    s, keep = make_problem(problem)
    fa = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(NQ)
    lib().btrt3_oracle_collide(ctypes.byref(s), _ptr(fa), phi_prev, node, t, t_prev, _ptr(out))
    return out


def run(problem, nsteps=None, nthreads: int = 1) -> OracleLattice3:
    lat = OracleLattice3(problem, nthreads=nthreads).init()
    lat.step(problem.nsteps if nsteps is None else nsteps)
    return lat
