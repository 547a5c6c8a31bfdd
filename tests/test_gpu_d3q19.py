"""GPU parity of the D3Q19 sweep (include/btrt3.h) against the FP64 D3Q19 oracle
on the same seeded inputs: relative L2 <= 1e-11 for FP64 compute and <= 2e-5
for FP32 compute with FP32 storage; reduced storage against the closed form;
conservation, the exact walled steady state, sampled nodes of a full-size
lattice and the non-finite flag."""
import numpy as np
import pytest

import workloads as w
from conftest import cpu_threads
from oracle import d3q19 as o3

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 2e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _lattice(p, compute="f64", storage=None, shift="auto"):
    from paper_1902_09813_gb300 import Lattice3
    return Lattice3.from_problem(p, compute=compute, storage=storage, shift=shift)


def _oracle(p, nsteps):
    """phi after nsteps and the post-collision populations the GPU keeps then."""
    lat = o3.OracleLattice3(p, nthreads=cpu_threads()).init()
    lat.step(nsteps)
    phi = lat.phi()
    lat.step(1)
    return phi, lat.fpost.copy()


CASES = [
    # nx, ny, nz, bc, nonlinear, source, q
    (17, 13, 11, (0,) * 6, True, "const", 2.0),
    (17, 13, 11, (1,) * 6, True, "const", 2.0),
    (20, 9, 14, (0, 0, 1, 1, 0, 0), False, "none", 2.0),
    (9, 16, 12, (1, 1, 0, 0, 1, 1), True, "reaction", 2.5),
    (12, 10, 9, (0, 0, 0, 0, 1, 1), True, "field", 1.5),
    (3, 3, 3, (0,) * 6, True, "const", 2.0),
    (3, 3, 3, (1,) * 6, True, "reaction", 2.0),
    (70, 5, 4, (1, 1, 0, 0, 0, 0), False, "const", 2.0),
]


def _case_id(c):
    return f"{c[0]}x{c[1]}x{c[2]}-bc{''.join(map(str, c[3]))}-{c[5]}-q{c[6]}"


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_fp64_random_states(case):
    nx, ny, nz, bc, nonlin, src, q = case
    p = w.random_state_problem3(nx, ny, nz, seed=nx + 7 * ny + 13 * nz, bc=bc, nonlinear=nonlin, source=src,
                                flux_q=q)
    steps = 8
    lat = _lattice(p).init(p.phi0()).step(steps)
    phi, fpost = _oracle(p, steps)
    assert _rel(lat.phi_host(), phi) <= TOL64
    assert _rel(lat.read_f(), fpost) <= TOL64
    assert lat.check() == 0


@pytest.mark.parametrize("shift", ["ref", "local"])
@pytest.mark.parametrize("case", CASES[:5], ids=_case_id)
def test_fp32_storage_random_states(case, shift):
    nx, ny, nz, bc, nonlin, src, q = case
    p = w.random_state_problem3(nx, ny, nz, seed=nx + 7 * ny + 13 * nz, bc=bc, nonlinear=nonlin, source=src,
                                flux_q=q)
    steps = 8
    lat = _lattice(p, "f32", "f32", shift).init(p.phi0()).step(steps)
    phi, fpost = _oracle(p, steps)
    assert _rel(lat.phi_host(), phi) <= TOL32
    assert _rel(lat.read_f(), fpost) <= TOL32


def _hill(n=24):
    dx = 1.0 / n
    dt = 2.0 * dx * dx
    return w.gaussian_hill3(n=n, sigma0=0.12, u=(0.3, -0.2, 0.1), A0=(0.04, 0.008, 0.0, 0.03, -0.006, 0.02),
                            nsteps=int(round(0.1 / dt)), dx=dx, dt=dt)


def test_gaussian_hill3_matches_oracle_and_mass():
    p = _hill()
    lat = _lattice(p).init(p.phi0()).step(p.nsteps)
    phi, _ = _oracle(p, p.nsteps)
    got = lat.phi_host()
    assert _rel(got, phi) <= TOL64
    m0 = p.phi0().sum()
    assert abs(lat.mass() - m0) <= 1e-12 * abs(m0)
    ex = w.gaussian_hill3_exact(p, p.nsteps * p.dt)
    assert w.gre(got, ex) == pytest.approx(w.gre(phi, ex), rel=1e-9)


@pytest.mark.parametrize("storage,bound", [("f32", 0.01), ("f16", 0.01), ("bf16", 0.05)])
def test_reduced_storage_discretisation_error(storage, bound):
    """Closed-form error with FP32 compute and reduced storage (local shift)
    against the FP64 result: FP32 and FP16 within 1 %, BF16 within 5 %."""
    p = _hill()
    ex = w.gaussian_hill3_exact(p, p.nsteps * p.dt)
    g64 = w.gre(_lattice(p).init(p.phi0()).step(p.nsteps).phi_host(), ex)
    g = w.gre(_lattice(p, "f32", storage, "local").init(p.phi0()).step(p.nsteps).phi_host(), ex)
    assert abs(g - g64) <= bound * g64, (g64, g)


def test_steady_diffusion_between_walls_exact():
    p = w.steady_diffusion3(n=5, k1=1.25, nsteps=4000)
    lat = _lattice(p).init(p.phi0()).step(p.nsteps)
    assert np.abs(lat.phi_host() - w.steady_diffusion3_exact(p)).max() < 1e-11


def test_full_size_sampled_nodes():
    """A 384^3 lattice (the benchmark size) against the oracle's collision at
    sampled nodes: pull the node's populations from the GPU state, collide with
    the oracle, compare with the GPU's next state."""
    n = 384
    p = w.gaussian_hill3(n=n, sigma0=20.0, u=(0.05, -0.03, 0.02), A0=(0.02, 0.004, 0.0, 0.015, -0.003, 0.01),
                         nsteps=3)
    lat = _lattice(p).init(p.phi0()).step(3)
    c, _ = o3.lattice()
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (191, 17, 300), (5, 383, 64), (200, 200, 200)]
    wins, phis = {}, {}
    ph = lat.phi()
    for pt in pts:
        fl = np.zeros(19)
        for i in range(19):
            sx, sy, sz = ((pt[0] - c[i, 0]) % n, (pt[1] - c[i, 1]) % n, (pt[2] - c[i, 2]) % n)
            fl[i] = lat.read_f(sx, sy, sz, 1, 1, 1)[i, 0, 0, 0]
        wins[pt] = fl
        phis[pt] = float(ph[pt[2], pt[1], pt[0]].item())
    _, t_now = lat.time()
    lat.step(1)
    for pt in pts:
        node = (pt[2] * n + pt[1]) * n + pt[0]
        ref = o3.collide(p, wins[pt], phis[pt], node, t_now + p.dt, t_now)
        got = lat.read_f(pt[0], pt[1], pt[2], 1, 1, 1)[:, 0, 0, 0]
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max()), pt


def test_nonfinite_flag():
    """A NaN in host-provided initial data is reported as EUNSTABLE (no device fault)."""
    from paper_1902_09813_gb300 import _capi as C
    p = w.random_state_problem3(8, 7, 6, seed=3, nonlinear=False, source="none")
    phi0 = p.phi0()
    phi0[2, 3, 4] = float("nan")
    lat = _lattice(p).init(phi0).step(3)
    with pytest.raises(C.BtrtError) as e:
        lat.check()
    assert e.value.code == C.EUNSTABLE
    assert _lattice(p).init(p.phi0()).step(3).check() == 0


@pytest.mark.parametrize("compute,storage", [("f64", "f64"), ("f32", "f16")])
def test_checkpoint_resume_bitwise(compute, storage):
    p = w.random_state_problem3(11, 9, 7, seed=6, bc=(1, 1, 0, 0, 1, 1), nonlinear=True, source="reaction")
    a = _lattice(p, compute, storage).init(p.phi0()).step(5)
    state = a.save()
    a.step(4)
    b = _lattice(p, compute, storage).load(state).step(4)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    assert a.time() == b.time()


def test_fp32_ill_conditioned_first_order_block():
    """A 3-D tensor with eigenvalues (1e4, 1e-3, 2e-3): the FP32 sweep inverts the
    ill-conditioned blocks in FP64 and meets the FP32 tolerance."""
    p = w.random_state_problem3(12, 10, 9, seed=14, bc=(0, 0, 1, 1, 0, 0), nonlinear=True, source="none")
    p = p.replace(A0=w.rot_tensor3((1.0e4, 1.0e-3, 2.0e-3), (0.3, 0.7, 1.1)), a2=0.3)
    steps = 8
    lat = _lattice(p, "f32", "f32", "ref").init(p.phi0()).step(steps)
    phi, _ = _oracle(p, steps)
    assert _rel(lat.phi_host(), phi) <= TOL32
    assert lat.check() == 0
