"""FP64 CPU oracle of the B-TriRT D2Q9 scheme -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA library: the C source
``btrt_oracle.c`` is compiled here with gcc into ``oracle/_build`` and called
through ctypes.  Inputs come from :mod:`workloads` (seeded problem data).

Pins (see ``tests/test_oracle_pins.py``): Eq. 9-10 moment identities, the
printed D2Q9 matrices R, P, C, H, T (Eqs. 78, 79, 85, 88, 90) and the block
diagonalisations (Eqs. 92, 95, 99), mass conservation, reduction to a textbook
BGK scheme, the exact steady state of the half-way bounce-back problem
(Eq. 36 with Eq. 62) and its numerical slip (Eq. 61), the Gaussian-hill and
manufactured-solution closed forms with second-order convergence, and the
paper's printed errors for the linear CDE (Sec. 4.1.2, Table 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "btrt_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle.so"
NQ = 9

_BC = {0: 0, 1: 1}
_K2 = {"hbb": 0, "const": 1}
_SRC_KIND = {"none": 0, "const": 1, "trig": 2, "field": 3, "reaction": 4}


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP if available).  No FMA contraction and
    no fast-math so that its arithmetic is the plain IEEE order of the source."""
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


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 4),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("u", ctypes.c_double * 2), ("b2", ctypes.c_double),
        ("c3", ctypes.c_double),
        ("A0", ctypes.c_double * 3), ("a2", ctypes.c_double),
        ("k0", ctypes.c_double),
        ("k2_mode", ctypes.c_int32), ("src_kind", ctypes.c_int32),
        ("k2", ctypes.c_double),
        ("src_const", ctypes.c_double), ("src_lam", ctypes.c_double), ("src_k", ctypes.c_double),
        ("src_alpha", ctypes.c_double * 4),
        ("wall", ctypes.c_double * 4),
        ("wall_lam", ctypes.c_double),
        ("wall_arr", ctypes.c_void_p * 4),
        ("src_field", ctypes.c_void_p),
        ("A_field", ctypes.c_void_p * 3),
        ("b_dir", ctypes.c_double * 2), ("b_q", ctypes.c_double),
        ("react_rate", ctypes.c_double), ("react_exp", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # BTRT_ORACLE_LIB points the tests at a deliberately mutated build of this
        # oracle (tests/test_oracle_mutations.py); unset, the pinned source is used.
        path = os.environ.get("BTRT_ORACLE_LIB") or build()
        L = ctypes.CDLL(str(path))
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        d = ctypes.c_double
        L.btrt_oracle_B.argtypes = [P, d, dp]
        L.btrt_oracle_C.argtypes = [P, d]
        L.btrt_oracle_C.restype = d
        L.btrt_oracle_A.argtypes = [P, d, dp]
        L.btrt_oracle_K1.argtypes = [P, d, dp]
        L.btrt_oracle_k2_from_k1.argtypes = [d]
        L.btrt_oracle_k2_from_k1.restype = d
        L.btrt_oracle_k2.argtypes = [P, dp]
        L.btrt_oracle_k2.restype = d
        L.btrt_oracle_source.argtypes = [P, d, d, d, d]
        L.btrt_oracle_source.restype = d
        L.btrt_oracle_feq.argtypes = [P, d, dp]
        L.btrt_oracle_relax.argtypes = [d, dp, dp, d, dp, dp]
        L.btrt_oracle_collide.argtypes = [P, dp, d, d, d, d, d, dp]
        L.btrt_oracle_init.argtypes = [P, dp, dp, dp]
        L.btrt_oracle_phi.argtypes = [P, dp, dp]
        L.btrt_oracle_step.argtypes = [P, dp, dp, dp, d, ctypes.c_int, ctypes.c_int]
        L.btrt_oracle_run.argtypes = [P, dp, dp, dp, d, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        L.btrt_oracle_node_step.argtypes = [P, dp, ctypes.c_int, ctypes.c_int, d, d, dp, dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_problem(p) -> tuple:
    """Translate a workloads.Problem into the oracle's C struct.  Returns the
    struct and the list of numpy arrays it points to (kept alive by the caller)."""
    s = _Problem()
    s.nx, s.ny = p.nx, p.ny
    for k in range(4):
        s.bc[k] = int(p.bc[k])
    s.dx, s.dt, s.x0, s.y0 = p.dx, p.dt, p.x0, p.y0
    s.u[0], s.u[1] = p.u
    s.b2, s.c3 = p.b2, p.c3
    for k in range(3):
        s.A0[k] = p.A0[k]
    s.a2, s.k0 = p.a2, p.k0
    s.k2_mode = _K2[p.k2_mode]
    s.k2 = p.k2
    src = p.source
    s.src_kind = _SRC_KIND[src.kind]
    s.src_const, s.src_lam, s.src_k = src.const, src.lam, src.k
    s.react_rate, s.react_exp = src.const, getattr(src, "exp", 1.0)
    s.b_dir[0], s.b_dir[1] = getattr(p, "b_dir", (1.0, 1.0))
    s.b_q = getattr(p, "b_q", 2.0)
    for k in range(4):
        s.src_alpha[k] = src.alpha[k]
        s.wall[k] = p.wall[k]
    s.wall_lam = p.wall_lam
    keep = []
    if p.wall_arrays is not None:
        for k, arr in enumerate(p.wall_arrays):
            if arr is not None:
                a = np.ascontiguousarray(arr, dtype=np.float64)
                keep.append(a)
                s.wall_arr[k] = a.ctypes.data
    if getattr(p, "src_field", None) is not None:
        a = np.ascontiguousarray(p.src_field, dtype=np.float64)
        assert a.shape == (p.ny, p.nx)
        keep.append(a)
        s.src_field = a.ctypes.data
    if getattr(p, "A_field", None) is not None:
        for k in range(3):
            a = np.ascontiguousarray(p.A_field[k], dtype=np.float64)
            assert a.shape == (p.ny, p.nx)
            keep.append(a)
            s.A_field[k] = a.ctypes.data
    return s, keep


class OracleLattice:
    """A lattice advanced by the oracle.  State: pre-collision populations f at
    time t (planes [9, ny, nx]), the last post-collision populations, phi_prev."""

    def __init__(self, problem, nthreads: int = 1):
        self.problem = problem
        self.s, self._keep = make_problem(problem)
        self.nthreads = nthreads
        n = problem.nx * problem.ny
        self.f = np.zeros((NQ, problem.ny, problem.nx))
        self.fpost = np.zeros_like(self.f)
        self.phi_prev = np.zeros((problem.ny, problem.nx))
        self.step_index = 0
        self.t0 = problem.t0
        del n
        # walls re-evaluated every step (time-dependent Dirichlet data): the C
        # struct points at these arrays, refilled before each step
        self._walls = None
        if getattr(problem, "wall_fn", None) is not None:
            self._walls = [np.array(a, dtype=np.float64) for a in problem.wall_arrays_at(problem.t0)]
            for k, a in enumerate(self._walls):
                self.s.wall_arr[k] = a.ctypes.data
            self.s.wall_lam = 0.0

    def init(self, phi0=None):
        if phi0 is None:
            phi0 = self.problem.phi0()
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        lib().btrt_oracle_init(ctypes.byref(self.s), _ptr(phi0), _ptr(self.f), _ptr(self.phi_prev))
        self.step_index = 0
        return self

    @property
    def t(self) -> float:
        return self.t0 + self.step_index * self.problem.dt

    def step(self, nsteps: int = 1):
        if self._walls is None:
            lib().btrt_oracle_run(ctypes.byref(self.s), _ptr(self.f), _ptr(self.fpost),
                                  _ptr(self.phi_prev), self.t0, self.step_index, nsteps, self.nthreads)
            self.step_index += nsteps
            return self
        for _ in range(nsteps):
            # the wall value of the step from t_n to t_{n+1} is taken at t_{n+1}
            for a, v in zip(self._walls, self.problem.wall_arrays_at(self.t + self.problem.dt)):
                a[:] = v
            lib().btrt_oracle_run(ctypes.byref(self.s), _ptr(self.f), _ptr(self.fpost),
                                  _ptr(self.phi_prev), self.t0, self.step_index, 1, self.nthreads)
            self.step_index += 1
        return self

    def phi(self) -> np.ndarray:
        out = np.zeros((self.problem.ny, self.problem.nx))
        lib().btrt_oracle_phi(ctypes.byref(self.s), _ptr(self.f), _ptr(out))
        return out

    def mass(self) -> float:
        return float(self.phi().sum())


# -- per-node helpers -------------------------------------------------------
def feq(problem, phi: float) -> np.ndarray:
    s, keep = make_problem(problem)
    out = np.zeros(NQ)
    lib().btrt_oracle_feq(ctypes.byref(s), phi, _ptr(out))
    return out


def relax(k0: float, K1, K2, c: float, fneq) -> np.ndarray:
    K1 = np.ascontiguousarray(K1, dtype=np.float64).reshape(4)
    K2 = np.ascontiguousarray(K2, dtype=np.float64).reshape(4)
    fneq = np.ascontiguousarray(fneq, dtype=np.float64)
    out = np.zeros(NQ)
    lib().btrt_oracle_relax(k0, _ptr(K1), _ptr(K2), c, _ptr(fneq), _ptr(out))
    return out


def collide(problem, f, phi_prev: float, x: float, y: float, t: float, t_prev: float) -> np.ndarray:
    s, keep = make_problem(problem)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(NQ)
    lib().btrt_oracle_collide(ctypes.byref(s), _ptr(f), phi_prev, x, y, t, t_prev, _ptr(out))
    return out


def K1(problem, phi: float) -> np.ndarray:
    s, keep = make_problem(problem)
    out = np.zeros(4)
    lib().btrt_oracle_K1(ctypes.byref(s), phi, _ptr(out))
    return out.reshape(2, 2)


def k2_from_k1(k1: float) -> float:
    return lib().btrt_oracle_k2_from_k1(k1)


def B(problem, phi: float) -> np.ndarray:
    s, keep = make_problem(problem)
    out = np.zeros(2)
    lib().btrt_oracle_B(ctypes.byref(s), phi, _ptr(out))
    return out


def C(problem, phi: float) -> float:
    s, keep = make_problem(problem)
    return lib().btrt_oracle_C(ctypes.byref(s), phi)


def source(problem, x: float, y: float, t: float, phi: float = 0.0) -> float:
    s, keep = make_problem(problem)
    return lib().btrt_oracle_source(ctypes.byref(s), x, y, t, phi)


def node_step(problem, win, ix: int, iy: int, phi_prev: float, t_next: float):
    """Pull-form step of one node from a [3, 3, 9] window of post-collision
    populations (see btrt_oracle_node_step)."""
    s, keep = make_problem(problem)
    win = np.ascontiguousarray(win, dtype=np.float64).reshape(-1)
    out = np.zeros(NQ)
    phi = np.zeros(1)
    lib().btrt_oracle_node_step(ctypes.byref(s), _ptr(win), ix, iy, phi_prev, t_next,
                                _ptr(out), _ptr(phi))
    return out, float(phi[0])


def run(problem, nsteps=None, nthreads: int = 1) -> OracleLattice:
    lat = OracleLattice(problem, nthreads=nthreads).init()
    lat.step(problem.nsteps if nsteps is None else nsteps)
    return lat
