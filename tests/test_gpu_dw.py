"""FP32 compute with the local shift and phi kept as a double-word pair
(BTRT_SHIFT_LOCAL_DW): the phi planes are never rounded to FP32.

Checked here: FP32/FP16/BF16 storage against the FP64 oracle within the FP32
tolerance and never less accurate than the plain local shift; phi and the
populations read back as high + low word; the FP64 mass of both words;
checkpoint/resume bitwise; the forms and batches that do not take it refuse it."""
import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _lattice(p, storage, shift="local_dw", **kw):
    from paper_1902_09813_gb300 import Lattice
    return Lattice.from_problem(p, compute="f32", storage=storage, shift=shift, **kw)


CASES = [(37, 29, (0, 0, 0, 0), True, "trig"), (37, 29, (1, 1, 1, 1), True, "trig"),
         (70, 65, (0, 0, 1, 1), True, "const"), (96, 40, (1, 1, 1, 1), False, "trig"),
         (3, 3, (1, 1, 1, 1), True, "const"), (5, 97, (1, 1, 0, 0), True, "reaction")]


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_dw_matches_oracle(case, storage):
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=13 * nx + ny, bc=bc, nonlinear=nonlin, source=src,
                               flux_q=2.5 if src == "reaction" else 2.0)
    steps = 10
    o = oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(steps)
    ref = o.phi()
    got = {}
    for shift in ("local_dw", "local"):
        lat = _lattice(p, storage, shift)
        lat.init(p.phi0(), t0=p.t0).step(steps)
        assert lat.check() == 0
        got[shift] = lat.phi_host()
        if shift == "local_dw" and storage == "f32":
            o.step(1)
            assert _rel(lat.read_f(), o.fpost) <= TOL32
    if storage == "f32":
        assert _rel(got["local_dw"], ref) <= TOL32
    # never the less accurate form (up to FP32 arithmetic noise)
    assert _rel(got["local_dw"], ref) <= _rel(got["local"], ref) * 1.05 + 1e-7


def test_dw_phi_reads_and_mass():
    """phi comes back as high + low word in FP64 (host and device copies agree),
    FP32 reads round it once, and the mass is the FP64 sum of both words."""
    import torch
    p = w.random_state_problem(130, 67, seed=3, bc=(1, 1, 0, 0), nonlinear=True)
    lat = _lattice(p, "f16").init(p.phi0(), t0=p.t0).step(7)
    host = lat.phi_host()
    dev = lat.phi(dtype=torch.float64).cpu().numpy()
    assert np.array_equal(host, dev)
    f32 = lat.phi_host(dtype=np.float32)
    assert np.array_equal(f32, host.astype(np.float32))
    assert lat.mass() == pytest.approx(float(host.sum()), rel=1e-12)
    # the low words carry information: phi is not a set of FP32 values
    assert np.any(host != host.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_dw_checkpoint_resume_bitwise(storage):
    p = w.random_state_problem(45, 33, seed=4, bc=(1, 1, 0, 0), nonlinear=True)
    a = _lattice(p, storage)
    a.init(p.phi0()).step(7)
    state = a.save()
    a.step(6)
    b = _lattice(p, storage)
    b.load(state)
    b.step(6)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    assert a.step_residual(3) == b.step_residual(3)
    c = _lattice(p, storage, "local")
    with pytest.raises(Exception):
        c.load(state)


def test_dw_refuses_other_forms_and_batches():
    from paper_1902_09813_gb300 import Batch, _capi as C
    p = w.random_state_problem(40, 30, seed=6)
    lat = _lattice(p, "f16").init(p.phi0())
    for form in ("vec", "tb2", "tb2v", "tma"):
        with pytest.raises(C.BtrtError):
            lat.set_sweep_variant(form)
    lat.set_sweep_variant("plain")
    lat.set_sweep_variant("auto")
    with pytest.raises(C.BtrtError):
        Batch([lat])
