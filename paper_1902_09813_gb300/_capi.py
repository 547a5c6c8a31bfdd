"""ctypes declarations of the C ABI in include/*.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libbtrt.so"

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
BC_PERIODIC, BC_HBB = 0, 1
F64, F32, F16, BF16, DF64 = 0, 1, 2, 3, 4
K2_HBB, K2_CONST = 0, 1
SRC_NONE, SRC_CONST, SRC_TRIG, SRC_FIELD, SRC_REACTION = 0, 1, 2, 3, 4
FIELD_SOURCE, FIELD_DIFFUSION = 1, 2
SWEEP_AUTO, SWEEP_PLAIN, SWEEP_TMA, SWEEP_TB2, SWEEP_VEC, SWEEP_TB2V = 0, 1, 2, 3, 4, 5
SHIFT_REF, SHIFT_LOCAL = 0, 1
PROBE_FMA, PROBE_ADD, PROBE_MUL = 0, 1, 2
SHIFT_LOCAL_DW, SHIFT_LOCAL_SR, SHIFT_LOCAL_DW_SR, SHIFT_MOMENT_SR = 2, 3, 4, 5
SHIFTS = {"ref": SHIFT_REF, "local": SHIFT_LOCAL, "local_dw": SHIFT_LOCAL_DW, "local_sr": SHIFT_LOCAL_SR,
          "local_dw_sr": SHIFT_LOCAL_DW_SR, "moment_sr": SHIFT_MOMENT_SR}

FORMATS = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "df64": DF64}


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 4),
        ("compute", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("phi_ref", ctypes.c_double),
        ("fields", ctypes.c_int32), ("shift", ctypes.c_int32),
    ]


class Coeffs(ctypes.Structure):
    _fields_ = [
        ("u", ctypes.c_double * 2), ("b2", ctypes.c_double), ("c3", ctypes.c_double),
        ("A0", ctypes.c_double * 3), ("a2", ctypes.c_double), ("k0", ctypes.c_double),
        ("k2_mode", ctypes.c_int32), ("src_kind", ctypes.c_int32),
        ("k2", ctypes.c_double), ("src_const", ctypes.c_double),
        ("src_lam", ctypes.c_double), ("src_k", ctypes.c_double),
        ("src_alpha", ctypes.c_double * 4), ("wall_lam", ctypes.c_double),
        ("b_dir", ctypes.c_double * 2), ("b_q", ctypes.c_double),
        ("react_rate", ctypes.c_double), ("react_exp", ctypes.c_double),
    ]


class GridDesc3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 6),
        ("compute", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("shift", ctypes.c_int32), ("fields", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
        ("phi_ref", ctypes.c_double),
    ]


class Coeffs3(ctypes.Structure):
    _fields_ = [
        ("u", ctypes.c_double * 3), ("b2", ctypes.c_double), ("b_dir", ctypes.c_double * 3),
        ("b_q", ctypes.c_double), ("c3", ctypes.c_double),
        ("A0", ctypes.c_double * 6), ("a2", ctypes.c_double), ("k0", ctypes.c_double),
        ("k2_mode", ctypes.c_int32), ("src_kind", ctypes.c_int32),
        ("k2", ctypes.c_double), ("src_const", ctypes.c_double), ("src_lam", ctypes.c_double),
        ("react_rate", ctypes.c_double), ("react_exp", ctypes.c_double),
        ("wall", ctypes.c_double * 6), ("wall_lam", ctypes.c_double),
    ]


class BtrtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"btrt error {code}: {msg}")
        self.code = code


# (name, restype, argtypes) of every exported entry point
_vp, _dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_i32, _i64, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = [
    ("btrt_workspace_bytes", _sz, [ctypes.POINTER(GridDesc)]),
    ("btrt_create", ctypes.c_int, [ctypes.POINTER(GridDesc), _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    ("btrt_set_coeffs", ctypes.c_int, [_vp, ctypes.POINTER(Coeffs)]),
    ("btrt_set_boundary", ctypes.c_int, [_vp, _i32, _dp, _i32]),
    ("btrt_set_source_field", ctypes.c_int, [_vp, _dp]),
    ("btrt_set_diffusion_field", ctypes.c_int, [_vp, _dp, _dp, _dp]),
    ("btrt_init_phi", ctypes.c_int, [_vp, _vp, _i32, _i32, ctypes.c_double]),
    ("btrt_step", ctypes.c_int, [_vp, _i64]),
    ("btrt_step_residual", ctypes.c_int, [_vp, _i64, _dp]),
    ("btrt_read_phi", ctypes.c_int, [_vp, _vp, _i32, _i32]),
    ("btrt_read_f", ctypes.c_int, [_vp, _dp, _i32, _i32, _i32, _i32]),
    ("btrt_mass", ctypes.c_int, [_vp, _dp]),
    ("btrt_check", ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    ("btrt_set_sweep_variant", ctypes.c_int, [_vp, _i32]),
    ("btrt_get_time", ctypes.c_int, [_vp, ctypes.POINTER(_i64), _dp]),
    ("btrt_state_bytes", _sz, [_vp]),
    ("btrt_save", ctypes.c_int, [_vp, _vp, _sz]),
    ("btrt_load", ctypes.c_int, [_vp, _vp, _sz]),
    ("btrt_destroy", ctypes.c_int, [_vp]),
    ("btrt_batch_workspace_bytes", _sz, [ctypes.POINTER(_vp), _i32]),
    ("btrt_batch_workspace_bytes_desc", _sz, [ctypes.POINTER(GridDesc), _i32]),
    ("btrt_batch_create", ctypes.c_int, [ctypes.POINTER(_vp), _i32, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    ("btrt_batch_set_tiles", ctypes.c_int, [_vp, _i32, _i32, _i32, _i32]),
    ("btrt_batch_autotune", ctypes.c_int, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                           ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    ("btrt_batch_step", ctypes.c_int, [_vp, _i64, _i32]),
    ("btrt_batch_prepare", ctypes.c_int, [_vp, _i64, _i32]),
    ("btrt_batch_graphs", ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    ("btrt_batch_step_tol", ctypes.c_int, [_vp, _i64, ctypes.c_double, _vp, _vp, _i32]),
    ("btrt_batch_set_freeze", ctypes.c_int, [_vp, _i32]),
    ("btrt_settle", ctypes.c_int, [_vp, _i32, ctypes.POINTER(_i64)]),
    ("btrt_batch_residuals", ctypes.c_int, [_vp, _dp]),
    ("btrt_batch_check", ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    ("btrt_batch_member_flags", ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    ("btrt_batch_set_wait_limit", ctypes.c_int, [_vp, ctypes.c_uint64, _i32]),
    ("btrt_batch_destroy", ctypes.c_int, [_vp]),
    ("btrt_phi_sum_static", ctypes.c_int, [_vp, _i32, _i32, _i32, _i64, _vp, _dp]),
    ("btrt_probe_fp64_rate", ctypes.c_int, [_vp, _i32, _i32, _i64, _vp, _dp, _dp]),
    ("btrt3_workspace_bytes", _sz, [ctypes.POINTER(GridDesc3)]),
    ("btrt3_create", ctypes.c_int, [ctypes.POINTER(GridDesc3), _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    ("btrt3_set_coeffs", ctypes.c_int, [_vp, ctypes.POINTER(Coeffs3)]),
    ("btrt3_set_source_field", ctypes.c_int, [_vp, _dp]),
    ("btrt3_init_phi", ctypes.c_int, [_vp, _vp, _i32, _i32, ctypes.c_double]),
    ("btrt3_step", ctypes.c_int, [_vp, _i64]),
    ("btrt3_read_phi", ctypes.c_int, [_vp, _vp, _i32, _i32]),
    ("btrt3_read_f", ctypes.c_int, [_vp, _dp, _i32, _i32, _i32, _i32, _i32, _i32]),
    ("btrt3_mass", ctypes.c_int, [_vp, _dp]),
    ("btrt3_check", ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    ("btrt3_get_time", ctypes.c_int, [_vp, ctypes.POINTER(_i64), _dp]),
    ("btrt3_state_bytes", _sz, [_vp]),
    ("btrt3_save", ctypes.c_int, [_vp, _vp, _sz]),
    ("btrt3_load", ctypes.c_int, [_vp, _vp, _sz]),
    ("btrt3_destroy", ctypes.c_int, [_vp]),
    ("btrt_last_error", ctypes.c_char_p, []),
    ("btrt_version", ctypes.c_char_p, []),
]

_lib = None


def load():
    """Load libbtrt.so.  Raises if the library has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is None:
        # BTRT_LIBRARY selects another build of the same library (the index-checked
        # debug build in the tests); unset, the in-tree build is used
        path = Path(os.environ.get("BTRT_LIBRARY") or LIB_PATH)
        if not path.exists():
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(str(path))
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code: int):
    if code != OK:
        raise BtrtError(code, load().btrt_last_error().decode())
    return code
