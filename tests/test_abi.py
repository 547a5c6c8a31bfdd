"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
entry point declared in include/*.h, and rejects invalid descriptions before
touching the device."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(btrt3?_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_1902_09813_gb300 as pkg
    pkg.build()
    from paper_1902_09813_gb300 import _capi
    return _capi.load()


def test_header_declares_entry_points():
    names = _declared_symbols()
    for expect in ("btrt_create", "btrt_step", "btrt_set_coeffs", "btrt_set_boundary",
                   "btrt_init_phi", "btrt_read_phi", "btrt_mass", "btrt_workspace_bytes",
                   "btrt3_create", "btrt3_step", "btrt3_set_coeffs", "btrt3_read_f"):
        assert expect in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_every_symbol():
    from paper_1902_09813_gb300 import _capi
    bound = {name for name, _, _ in _capi.SIGNATURES}
    assert set(_declared_symbols()) <= bound


def _desc(**kw):
    from paper_1902_09813_gb300.lattice import grid_desc
    base = dict(nx=64, ny=48, dx=1.0, dt=1.0, bc=(0, 0, 1, 1), compute="f64", storage="f64")
    base.update(kw)
    return grid_desc(**base)


def test_workspace_layout(lib):
    from paper_1902_09813_gb300 import _capi as C
    d = _desc()
    n = lib.btrt_workspace_bytes(ctypes.byref(d))
    pitch = 64
    fbuf = 9 * pitch * 48 * 8
    # two population buffers and two phi planes (double-buffered together)
    assert n >= 2 * fbuf + 2 * pitch * 48 * 8
    assert n % 256 == 0
    d16 = _desc(compute="f32", storage="f16")
    n16 = lib.btrt_workspace_bytes(ctypes.byref(d16))
    assert n16 < n
    assert C.OK == 0


@pytest.mark.parametrize("kw", [dict(nx=2), dict(ny=70000), dict(bc=(0, 1, 0, 0)),
                                dict(compute="f64", storage="f16"), dict(compute="f32", storage="f64"),
                                dict(dx=0.0), dict(dt=-1.0)])
def test_invalid_descriptions_rejected(lib, kw):
    d = _desc(**kw)
    assert lib.btrt_workspace_bytes(ctypes.byref(d)) == 0
    assert len(lib.btrt_last_error()) > 0


def test_unknown_storage_shift_rejected(lib):
    d = _desc(compute="f32", storage="f16")
    for bad in (6, -1):
        d.shift = bad
        assert lib.btrt_workspace_bytes(ctypes.byref(d)) == 0
        assert b"shift" in lib.btrt_last_error()
    for good in (0, 1, 2, 3, 4, 5):
        d.shift = good
        assert lib.btrt_workspace_bytes(ctypes.byref(d)) > 0


def test_stochastic_rounding_needs_16bit_storage(lib):
    """BTRT_SHIFT_LOCAL_SR / _DW_SR round F16/BF16 storage stochastically: FP32
    compute with 16-bit storage only; the _DW_SR form holds the low-word planes."""
    from paper_1902_09813_gb300.lattice import workspace_bytes
    from paper_1902_09813_gb300 import _capi as C
    for comp, st in (("f32", "f32"), ("f64", "f64"), ("df64", "df64")):
        for sh in ("local_sr", "local_dw_sr", "moment_sr"):
            with pytest.raises(C.BtrtError):
                workspace_bytes(_desc(compute=comp, storage=st, shift=sh))
    for st in ("f16", "bf16"):
        loc = workspace_bytes(_desc(compute="f32", storage=st, shift="local"))
        assert workspace_bytes(_desc(compute="f32", storage=st, shift="local_sr")) == loc
        assert workspace_bytes(_desc(compute="f32", storage=st, shift="local_dw_sr")) == \
            workspace_bytes(_desc(compute="f32", storage=st, shift="local_dw"))
        # the first-moment form: two more planes of the storage format per buffer
        assert workspace_bytes(_desc(compute="f32", storage=st, shift="moment_sr")) >= loc + 2 * 2 * 64 * 48 * 2


def test_create_rejects_null_workspace(lib):
    from paper_1902_09813_gb300 import _capi as C
    d = _desc()
    h = ctypes.c_void_p()
    assert lib.btrt_create(ctypes.byref(d), None, 1 << 30, None, ctypes.byref(h)) == C.EINVAL
    assert not h.value


def test_version(lib):
    assert b"sm_103a" in lib.btrt_version()


def _desc3(**kw):
    from paper_1902_09813_gb300.lattice3 import grid_desc3
    base = dict(nx=32, ny=24, nz=16, dx=1.0, dt=1.0, bc=(0, 0, 1, 1, 0, 0), compute="f64", storage="f64")
    base.update(kw)
    return grid_desc3(**base)


def test_d3q19_workspace_layout(lib):
    d = _desc3()
    n = lib.btrt3_workspace_bytes(ctypes.byref(d))
    plane = 64 * 24 * 16
    assert n >= 2 * 19 * plane * 8 + 2 * plane * 8 and n % 256 == 0
    d16 = _desc3(compute="f32", storage="f16", shift="local")
    assert 0 < lib.btrt3_workspace_bytes(ctypes.byref(d16)) < n


@pytest.mark.parametrize("kw", [dict(nz=2), dict(nx=1), dict(bc=(0, 1, 0, 0, 0, 0)), dict(bc=(0, 0, 0, 0, 1, 0)),
                                dict(compute="df64", storage="df64"), dict(compute="f32", storage="f64"),
                                dict(compute="f64", storage="f16"), dict(dx=0.0),
                                dict(nx=1024, ny=1024, nz=200)])
def test_invalid_d3q19_descriptions_rejected(lib, kw):
    d = _desc3(**kw)
    assert lib.btrt3_workspace_bytes(ctypes.byref(d)) == 0
    assert len(lib.btrt_last_error()) > 0


def test_d3q19_rejects_unknown_shift_and_fields(lib):
    d = _desc3(compute="f32", storage="f16")
    d.shift = 3
    assert lib.btrt3_workspace_bytes(ctypes.byref(d)) == 0
    d = _desc3()
    d.fields = 2      # no diffusion-field planes in 3-D
    assert lib.btrt3_workspace_bytes(ctypes.byref(d)) == 0


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: with the library missing, the first call that needs it
    raises instead of computing anything."""
    import subprocess
    import sys
    code = ("import numpy as np, workloads as w\n"
            "from paper_1902_09813_gb300 import Lattice\n"
            "p = w.random_state_problem(8, 8, seed=1)\n"
            "try:\n"
            "    Lattice.from_problem(p, compute='f64')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', 'missing' in str(e))\n"
            "else:\n"
            "    print('no error')\n")
    env = dict(os.environ, BTRT_LIBRARY=str(tmp_path / "absent" / "libbtrt.so"), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT,
                       timeout=300)
    assert "raised: True" in r.stdout, (r.stdout, r.stderr[-2000:])


def test_double_word_phi_needs_fp32_compute(lib):
    """BTRT_SHIFT_LOCAL_DW keeps phi as two FP32 planes: FP32 compute only, and the
    workspace holds the low-word planes (one more plane per phi buffer)."""
    from paper_1902_09813_gb300.lattice import workspace_bytes
    from paper_1902_09813_gb300 import _capi as C
    with pytest.raises(C.BtrtError):
        workspace_bytes(_desc(compute="f64", storage="f64", shift="local_dw"))
    dw = workspace_bytes(_desc(compute="f32", storage="f16", shift="local_dw"))
    loc = workspace_bytes(_desc(compute="f32", storage="f16", shift="local"))
    assert dw - loc >= 2 * 64 * 48 * 4
