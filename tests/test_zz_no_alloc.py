"""btrt_phi_sum_static: the FP64 phi sum for callers that cannot allocate device
memory (a serving process that reserves its whole device budget at start-up and
forbids later allocations, or a plug-in inside a host framework that owns the
device allocator).  It keeps its partial sums in a fixed array of the library's
own device memory; its result must equal btrt_mass's, the workspace-backed sum,
bitwise (both run the library's one fixed-order FP64 reduction).

This file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def _static_sum(lib, t):
    import torch
    from paper_1902_09813_gb300 import _capi as C
    code = C.F64 if t.dtype == torch.float64 else C.F32
    out = ctypes.c_double()
    stream = torch.cuda.current_stream()
    rc = lib.btrt_phi_sum_static(ctypes.c_void_p(t.data_ptr()), code, t.shape[1], t.shape[0],
                                 t.stride(0), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
    C.check(rc)
    return out.value


@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_static_sum_matches_mass_twice(compute):
    import torch
    from paper_1902_09813_gb300 import Lattice, _capi as C
    lib = C.load()
    p = w.random_state_problem(301, 157, seed=21, bc=(1, 1, 0, 0))
    q = w.nonlinear_modes(n=256, nsteps=4)
    for prob in (p, q):
        lat = Lattice.from_problem(prob, compute=compute, storage=compute,
                                   stream=torch.cuda.current_stream())
        lat.init(prob.phi0()).step(5)
        for _ in range(2):          # two calls in a row share the static scratch
            ref = lat.mass()
            phi = lat.phi()         # dense device copy of the phi plane
            got = _static_sum(lib, phi)
            # the same reduction kernels over the same values in the same order
            assert got == ref
            lat.step(3)


def test_static_sum_padded_pitch():
    """A plane with row padding: only the first nx values of each row count."""
    import torch
    from paper_1902_09813_gb300 import _capi as C
    lib = C.load()
    base = torch.arange(40 * 70, dtype=torch.float64, device="cuda").reshape(40, 70) * 1e-3
    view = base[:, :61]
    got = _static_sum(lib, view)
    assert got == pytest.approx(float(view.sum().item()), rel=1e-12)


def test_static_sum_rejects_oversized_plane():
    import torch
    from paper_1902_09813_gb300 import _capi as C
    lib = C.load()
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    rc = lib.btrt_phi_sum_static(ctypes.c_void_p(t.data_ptr()), C.F64, 70000, 1, 70000, None,
                                 ctypes.byref(out))
    assert rc == C.EINVAL
    assert b"65536" in lib.btrt_last_error()
