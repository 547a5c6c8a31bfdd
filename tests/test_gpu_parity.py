"""GPU parity: the CUDA sweep (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: relative L2 <= 1e-11 for FP64 compute and
<= 2e-5 for FP32 compute with FP32 storage."""
import math

import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 2e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _lattice(p, compute="f64", storage=None, **kw):
    from paper_1902_09813_gb300 import Lattice
    return Lattice.from_problem(p, compute=compute, storage=storage, **kw)


def _gpu_run(p, nsteps, compute="f64", storage=None):
    lat = _lattice(p, compute, storage)
    lat.init(p.phi0(), t0=p.t0).step(nsteps)
    return lat


def _oracle_run(p, nsteps):
    """Oracle after nsteps + 1 collisions: phi at t_n and the post-collision
    populations at t_n (the state the GPU keeps)."""
    lat = oracle.OracleLattice(p, nthreads=cpu_threads()).init()
    lat.step(nsteps)
    phi = lat.phi()
    lat.step(1)
    return phi, lat.fpost.copy()


CASES = [
    # (nx, ny, bc, nonlinear, source, steps)
    (37, 29, (0, 0, 0, 0), True, "trig", 12),
    (37, 29, (1, 1, 1, 1), True, "trig", 12),
    (70, 65, (0, 0, 1, 1), True, "const", 10),
    (70, 65, (1, 1, 0, 0), False, "none", 10),
    (96, 40, (1, 1, 1, 1), False, "trig", 9),
    (3, 3, (0, 0, 0, 0), True, "trig", 7),
    (3, 3, (1, 1, 1, 1), True, "const", 7),
    (5, 97, (1, 1, 0, 0), True, "trig", 6),
    (130, 3, (0, 0, 1, 1), True, "none", 6),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_fp64_random_states(case):
    nx, ny, bc, nonlin, src, steps = case
    p = w.random_state_problem(nx, ny, seed=nx * 131 + ny, bc=bc, nonlinear=nonlin, source=src)
    lat = _gpu_run(p, steps)
    phi_ref, fpost_ref = _oracle_run(p, steps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64
    f = lat.read_f()
    assert _rel(f, fpost_ref) <= TOL64
    assert np.max(np.abs(f - fpost_ref)) <= 1e-12 * np.max(np.abs(fpost_ref)) * 10


def test_fp64_wall_arrays_and_time_factor():
    """Per-node wall values carrying exp(lam t) (Table 3 setup, smaller grid)."""
    p = w.linear_cde(n=40, alpha=0.01, u=(0.3, 0.3), c=5.0, t_end=0.1, walls=True)
    lat = _gpu_run(p, p.nsteps)
    phi_ref, _ = _oracle_run(p, p.nsteps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64


def test_fp64_gaussian_hill_64():
    """64 x 64 periodic Gaussian hill, dx = dt = 1, 500 steps."""
    p = w.gaussian_hill()
    lat = _gpu_run(p, p.nsteps)
    phi_ref, _ = _oracle_run(p, p.nsteps)
    got = lat.phi_host()
    assert _rel(got, phi_ref) <= TOL64
    # mass conservation to rounding on the periodic grid
    m0 = p.phi0().sum()
    assert abs(lat.mass() - m0) <= 1e-12 * abs(m0)
    # same discretisation error against the closed form as the oracle
    ex = w.gaussian_hill_exact(p, p.nsteps * p.dt)
    assert w.gre(got, ex) == pytest.approx(w.gre(phi_ref, ex), rel=1e-9)


@pytest.mark.parametrize("n", [64, 128])
def test_fp64_manufactured_solution(n):
    """Full-tensor manufactured solution with HBB walls, diffusive scaling."""
    p = w.mms_sinsin(n=n)
    lat = _gpu_run(p, p.nsteps)
    phi_ref, _ = _oracle_run(p, p.nsteps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64


def test_fp64_nonlinear_modes_small():
    """Nonlinear anisotropic modes workload at 96 x 96, 60 steps."""
    p = w.nonlinear_modes(n=96, nsteps=60)
    lat = _gpu_run(p, p.nsteps)
    phi_ref, _ = _oracle_run(p, p.nsteps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64


def test_fp64_steady_diffusion_exact():
    """Half-way bounce-back steady state with Eq. 62 is exact on the GPU too."""
    p = w.steady_diffusion(n=10, nsteps=30000)
    lat = _gpu_run(p, p.nsteps)
    assert w.gre(lat.phi_host(), w.steady_diffusion_exact(p)) < 1e-12


@pytest.mark.parametrize("p_fn", [lambda: w.random_state_problem(70, 65, seed=9, bc=(1, 1, 0, 0)),
                                  lambda: w.nonlinear_modes(n=96, nsteps=60),
                                  lambda: w.mms_sinsin(n=64)],
                         ids=["random", "nonlinear", "mms"])
def test_fp32_compute_fp32_storage(p_fn):
    p = p_fn()
    steps = min(p.nsteps, 60)
    lat = _gpu_run(p, steps, compute="f32", storage="f32")
    phi_ref, _ = _oracle_run(p, steps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL32


def test_checkpoint_resume_bitwise():
    p = w.random_state_problem(45, 33, seed=4, bc=(1, 1, 1, 1))
    a = _gpu_run(p, 5)
    state = a.save()
    a.step(7)
    b = _lattice(p)
    b.load(state).step(7)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    assert a.time() == b.time()


def test_nonfinite_flag_reported():
    """A NaN in host-provided initial data is reported as EUNSTABLE (no device fault)."""
    from paper_1902_09813_gb300 import _capi as C
    p = w.random_state_problem(20, 20, seed=1)
    phi0 = p.phi0()
    phi0[3, 4] = float("nan")
    lat = _lattice(p)
    lat.init(phi0).step(3)
    with pytest.raises(C.BtrtError) as ei:
        lat.check()
    assert ei.value.code == C.EUNSTABLE
    ok = _gpu_run(p, 3)
    assert ok.check() == 0


def _window(lat, ix, iy):
    """3 x 3 x 9 window of post-collision populations around (ix, iy), periodically
    wrapped (entries beyond a wall are never used by the oracle)."""
    win = np.zeros((3, 3, 9))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            x, y = (ix + dx) % lat.nx, (iy + dy) % lat.ny
            win[dy + 1, dx + 1] = lat.read_f(x, y, 1, 1)[:, 0, 0]
    return win


@pytest.mark.parametrize("which", ["mms_8192", "nonlinear_8192"])
def test_full_size_sampled_nodes(which):
    """At the benchmark's full size and launch configuration: one more step of the
    GPU sweep at sampled nodes (corners, edges, interior) equals the oracle's
    single-node step from the GPU's own neighbourhood."""
    import torch
    if which == "mms_8192":
        p = w.mms_sinsin(n=8192, nsteps=3)
        compute = "f64"
        tol = 1e-13
    else:
        p = w.nonlinear_modes(n=8192, nsteps=3)
        compute = "f64"
        tol = 1e-13
    lat = _gpu_run(p, 3, compute=compute)
    n = p.nx
    pts = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1), (1, 0), (0, 5), (n - 1, 77),
           (4095, 0), (4096, n - 1), (31, 32), (32, 31), (5000, 6000), (n - 2, n - 2)]
    rng = np.random.default_rng(0)
    pts += [tuple(int(v) for v in rng.integers(0, n, size=2)) for _ in range(6)]
    wins = {pt: _window(lat, *pt) for pt in pts}
    phi_dev = lat.phi()
    phi_prev = {pt: float(phi_dev[pt[1], pt[0]].item()) for pt in pts}
    _, t_now = lat.time()
    lat.step(1)
    phi_dev = lat.phi()
    torch.cuda.synchronize()
    for pt in pts:
        fp, phi = oracle.node_step(p, wins[pt], pt[0], pt[1], phi_prev[pt], t_now + p.dt)
        got = lat.read_f(pt[0], pt[1], 1, 1)[:, 0, 0]
        assert np.allclose(got, fp, rtol=tol, atol=tol * np.abs(fp).max()), pt
        assert float(phi_dev[pt[1], pt[0]].item()) == pytest.approx(phi, rel=tol, abs=tol)


def test_full_size_mass_conservation_fp64():
    """8192^2 periodic nonlinear workload: FP64 mass is conserved to rounding."""
    p = w.nonlinear_modes(n=8192, nsteps=20)
    lat = _lattice(p)
    lat.init(p.phi0())
    m0 = lat.mass()
    lat.step(20)
    m1 = lat.mass()
    # both sums carry at most ~N eps |phi| ~ 1e-8 of rounding; a lost or duplicated
    # population would move the mass by O(1e-3) or more
    assert abs(m1 - m0) <= 1e-8


# ---------------------------------------------------------------- double-word path
@pytest.mark.parametrize("case", CASES[:5] + CASES[6:7], ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_df64_random_states(case):
    """Double-word (FP32-pair) arithmetic meets the FP64 tolerance against the oracle."""
    nx, ny, bc, nonlin, src, steps = case
    p = w.random_state_problem(nx, ny, seed=nx * 131 + ny, bc=bc, nonlinear=nonlin, source=src)
    lat = _gpu_run(p, steps, compute="df64", storage="df64")
    phi_ref, fpost_ref = _oracle_run(p, steps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64
    assert _rel(lat.read_f(), fpost_ref) <= TOL64


@pytest.mark.parametrize("p_fn", [lambda: w.mms_sinsin(n=64), lambda: w.gaussian_hill(),
                                  lambda: w.nonlinear_modes(n=96, nsteps=60)],
                         ids=["mms64", "gauss64x500", "nonlinear96"])
def test_df64_workloads(p_fn):
    p = p_fn()
    lat = _gpu_run(p, p.nsteps, compute="df64", storage="df64")
    phi_ref, _ = _oracle_run(p, p.nsteps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64


def test_df64_steady_diffusion_exact():
    p = w.steady_diffusion(n=10, nsteps=30000)
    lat = _gpu_run(p, p.nsteps, compute="df64", storage="df64")
    assert w.gre(lat.phi_host(), w.steady_diffusion_exact(p)) < 1e-11


# ---------------------------------------------------------------- TMA-staged FP32 sweep
TMA_CASES = [
    (100, 37, (0, 0, 0, 0), True, "trig"),
    (100, 37, (1, 1, 1, 1), True, "trig"),
    (65, 17, (0, 0, 1, 1), False, "const"),
    (130, 50, (1, 1, 0, 0), False, "none"),
    (3, 3, (0, 0, 0, 0), True, "trig"),
    (200, 33, (1, 1, 1, 1), False, "trig"),
]


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", TMA_CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_tma_sweep_bitwise_equals_plain(case, storage):
    """The TMA-staged tile kernel and the one-thread-per-node kernel do the same
    arithmetic on the same values: results are bitwise identical."""
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=7 * nx + ny, bc=bc, nonlinear=nonlin, source=src)
    a = _lattice(p, "f32", storage).set_sweep_variant("tma")
    b = _lattice(p, "f32", storage).set_sweep_variant("plain")
    a.init(p.phi0()).step(9)
    b.init(p.phi0()).step(9)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    assert a.check() == 0


def test_tma_sweep_fp32_matches_oracle_full_size_sample():
    """FP32 storage through the TMA kernel at 4096^2 against the oracle's
    single-node step at sampled nodes (FP32 tolerance)."""
    p = w.nonlinear_modes(n=4096, nsteps=3)
    lat = _lattice(p, "f32", "f32").set_sweep_variant("tma")
    lat.init(p.phi0()).step(3)
    n = p.nx
    pts = [(0, 0), (n - 1, n - 1), (63, 16), (64, 15), (2000, 1234), (31, 4095)]
    wins = {pt: _window(lat, *pt) for pt in pts}
    phi_dev = lat.phi()
    phi_prev = {pt: float(phi_dev[pt[1], pt[0]].item()) for pt in pts}
    _, t_now = lat.time()
    lat.step(1)
    for pt in pts:
        fp, _ = oracle.node_step(p, wins[pt], pt[0], pt[1], phi_prev[pt], t_now + p.dt)
        got = lat.read_f(pt[0], pt[1], 1, 1)[:, 0, 0]
        assert np.allclose(got, fp, rtol=2e-5, atol=2e-5 * np.abs(fp).max()), pt


# ---------------------------------------------------------------- per-node fields
@pytest.mark.parametrize("walls", [True, False])
@pytest.mark.parametrize("compute", ["f64", "df64"])
def test_variable_tensor_field(walls, compute):
    """Spatially varying diffusion tensor and a per-node source field (Eqs. 73-76)."""
    p = w.variable_tensor(n=48, alpha=1e-2, walls=walls, t_end=0.3)
    dt = 20.0 * p.dx ** 2
    p = p.replace(dt=dt, nsteps=int(round(0.3 / dt)))
    lat = _gpu_run(p, p.nsteps, compute=compute, storage=compute)
    phi_ref, _ = _oracle_run(p, p.nsteps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_variable_tensor_field_fp32_tma_equals_plain(storage):
    p = w.variable_tensor(n=70, alpha=1e-2, walls=True, t_end=0.2)
    dt = 20.0 * p.dx ** 2
    p = p.replace(dt=dt, nsteps=int(round(0.2 / dt)), phi_ref=0.0)
    a = _lattice(p, "f32", storage).set_sweep_variant("tma")
    b = _lattice(p, "f32", storage).set_sweep_variant("plain")
    a.init(p.phi0()).step(p.nsteps)
    b.init(p.phi0()).step(p.nsteps)
    assert np.array_equal(a.phi_host(), b.phi_host())
    if storage == "f32":
        phi_ref, _ = _oracle_run(p, p.nsteps)
        assert _rel(a.phi_host(), phi_ref) <= TOL32


# ---------------------------------------------------------------- power-law flux, reaction source
BF_CASES = [
    (40, 33, (0, 0, 0, 0), "reaction", 2.5),
    (40, 33, (1, 1, 1, 1), "reaction", 2.0),
    (37, 29, (1, 1, 0, 0), "trig", 1.5),
    (3, 3, (0, 0, 0, 0), "reaction", 3.0),
]


@pytest.mark.parametrize("case", BF_CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[3]}-q{c[4]}")
@pytest.mark.parametrize("compute", ["f64", "df64"])
def test_power_flux_reaction_random_states(case, compute):
    nx, ny, bc, src, q = case
    p = w.random_state_problem(nx, ny, seed=3 * nx + ny, bc=bc, nonlinear=True, source=src, flux_q=q)
    lat = _gpu_run(p, 10, compute=compute, storage=compute)
    phi_ref, fpost_ref = _oracle_run(p, 10)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64
    assert _rel(lat.read_f(), fpost_ref) <= TOL64


@pytest.mark.parametrize("compute,storage,tol", [("f64", "f64", TOL64), ("df64", "df64", TOL64),
                                                 ("f32", "f32", TOL32)])
def test_burgers_fisher_walls_per_step(compute, storage, tol):
    """Burgers-Fisher (Eq. 67) on [-1, 2]^2 with bounce-back walls re-evaluated
    from the exact solution before every step."""
    p = w.burgers_fisher(n=60, a=2.0, alpha=0.05, t_end=0.25)
    lat = _lattice(p, compute, storage)
    lat.init(p.phi0(), t0=p.t0).step_walls(p, p.nsteps)
    o = oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(p.nsteps)
    assert _rel(lat.phi_host(), o.phi()) <= tol
    assert lat.check() == 0


def test_burgers_fisher_reduced_storage_error():
    """Closed-form error with reduced storage against FP64's: FP32 storage within
    1 %; FP16 (local shift) within 5 % -- the steep front carries a convective
    part 3 w_i c_i.B of up to a tenth of phi, which the local shift leaves in the
    rounded value (measured 3.8 %)."""
    p = w.burgers_fisher(n=120, a=2.0, alpha=0.05, t_end=1.0)
    ex = w.burgers_fisher_exact(p, p.nsteps * p.dt)
    g64 = w.gre(_lattice(p, "f64").init(p.phi0()).step_walls(p, p.nsteps).phi_host(), ex)
    g32 = w.gre(_lattice(p, "f32", "f32").init(p.phi0()).step_walls(p, p.nsteps).phi_host(), ex)
    g16 = w.gre(_lattice(p, "f32", "f16").init(p.phi0()).step_walls(p, p.nsteps).phi_host(), ex)
    assert abs(g32 - g64) <= 0.01 * g64, (g64, g32)
    assert abs(g16 - g64) <= 0.05 * g64, (g64, g16)


def test_fp32_ill_conditioned_first_order_block():
    """A diffusion tensor with eigenvalues 1e4 and 1e-3 (lattice units) makes the
    per-node block 3 A^ + I/2 ill-conditioned (tr^2/det ~ 6e4); the FP32 sweep
    inverts such blocks in FP64 and still meets the FP32 tolerance."""
    from workloads.problems import _rot_tensor
    p = w.random_state_problem(40, 33, seed=12, bc=(1, 1, 0, 0), nonlinear=True, source="none")
    p = p.replace(A0=_rot_tensor(1.0e4, 1.0e-3, 0.4), a2=0.3)
    steps = 10
    lat = _gpu_run(p, steps, compute="f32", storage="f32")
    phi_ref, _ = _oracle_run(p, steps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL32
    assert lat.check() == 0


@pytest.mark.parametrize("model", ["lbgk", "mlbm", "rlbm", "ob-trirt"])
def test_table1_presets_match_oracle(model):
    """The comparison models of Table 1 run through the same kernels (k0 != 1,
    constant k2): GPU equals the oracle on the walled Table 3 problem and the
    Burgers-Fisher problem of Table 4."""
    from paper_1902_09813_gb300.presets import relaxation_preset
    p = w.linear_cde(n=50, alpha=0.01, u=(0.1, 0.1), c=5.0, t_end=0.1, walls=True)
    p = p.replace(**relaxation_preset(model, p.A0, p.dx, p.dt))
    lat = _gpu_run(p, p.nsteps)
    phi_ref, _ = _oracle_run(p, p.nsteps)
    assert _rel(lat.phi_host(), phi_ref) <= TOL64
    q = w.burgers_fisher(n=40, a=2.0, alpha=0.05, t_end=0.2)
    q = q.replace(**relaxation_preset(model, q.A0, q.dx, q.dt))
    lat = _lattice(q).init(q.phi0(), t0=q.t0).step_walls(q, q.nsteps)
    o = oracle.OracleLattice(q, nthreads=cpu_threads()).init().step(q.nsteps)
    assert _rel(lat.phi_host(), o.phi()) <= TOL64


# ---------------------------------------------------------------- two steps per launch
TB_CASES = [
    (100, 37, (0, 0, 0, 0), True, "trig"),
    (100, 37, (1, 1, 1, 1), True, "trig"),
    (65, 17, (0, 0, 1, 1), False, "const"),
    (130, 50, (1, 1, 0, 0), False, "none"),
    (3, 3, (0, 0, 0, 0), True, "trig"),
    (3, 3, (1, 1, 1, 1), True, "const"),
    (5, 97, (1, 1, 0, 0), True, "reaction"),
    (33, 17, (0, 0, 0, 0), True, "reaction"),
]


@pytest.mark.parametrize("steps", [9, 10])
@pytest.mark.parametrize("case", TB_CASES, ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_tb2_sweep_bitwise_equals_plain(case, steps):
    """Two steps per launch (first step kept in shared memory) and one step per
    launch do the same arithmetic node by node: results are bitwise identical,
    for odd step counts too (the last step runs in the plain form)."""
    _tb2_against_plain(case, steps, "f32")


@pytest.mark.parametrize("storage,shift", [("f16", "ref"), ("bf16", "ref"), ("f32", "local"), ("f16", "local"),
                                           ("bf16", "local")])
@pytest.mark.parametrize("case", TB_CASES[::2], ids=lambda c: f"{c[0]}x{c[1]}-bc{''.join(map(str, c[2]))}-{c[4]}")
def test_tb2_sweep_other_storage_bitwise_equals_plain(case, storage, shift):
    """The same with FP16 and BF16 storage (the first step's populations are kept
    in shared memory rounded to the storage format, as a stored step would be)
    and with the local shift (shared-memory values moved to the reading node's
    phi as the one-step pull does)."""
    _tb2_against_plain(case, 9, storage, shift)


@pytest.mark.parametrize("nonlinear", [True, False])
def test_default_form_bitwise_equals_plain(nonlinear):
    """AUTO (the default: the vector form for 16-bit storage on lattices of 2^21
    nodes or more, two steps per launch below) and the plain form give the same
    bits on walled lattices with FP16 storage, for constant and per-node
    coefficients."""
    p = w.random_state_problem(64, 40, seed=31, bc=(1, 1, 0, 0), nonlinear=nonlinear, source="const")
    q = w.random_state_problem(2100, 1000, seed=32, bc=(1, 1, 0, 0), nonlinear=nonlinear, source="const")
    a = _lattice(q, "f32", "f16", shift="local")
    b = _lattice(q, "f32", "f16", shift="local").set_sweep_variant("plain")
    a.init(q.phi0(), t0=q.t0).step(5)
    b.init(q.phi0(), t0=q.t0).step(5)
    assert np.array_equal(a.phi_host(), b.phi_host())
    a = _lattice(p, "f32", "f16", shift="local")
    b = _lattice(p, "f32", "f16", shift="local").set_sweep_variant("plain")
    a.init(p.phi0(), t0=p.t0).step(8)
    b.init(p.phi0(), t0=p.t0).step(8)
    assert np.array_equal(a.read_f(), b.read_f())


def _tb2_against_plain(case, steps, storage, shift="ref"):
    nx, ny, bc, nonlin, src = case
    p = w.random_state_problem(nx, ny, seed=3 * nx + ny, bc=bc, nonlinear=nonlin, source=src,
                               flux_q=2.5 if src == "reaction" else 2.0)
    a = _lattice(p, "f32", storage, shift=shift).set_sweep_variant("tb2")
    b = _lattice(p, "f32", storage, shift=shift).set_sweep_variant("plain")
    a.init(p.phi0(), t0=p.t0).step(steps)
    b.init(p.phi0(), t0=p.t0).step(steps)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert np.array_equal(a.read_f(), b.read_f())
    assert a.time() == b.time()
    assert a.check() == 0


def test_tb2_fields_and_large_ragged_grid():
    """Per-node tensor and source fields, and a 4099 x 4093 grid (ragged tiles at
    both far edges; FP32 storage with the reference shift and FP16 storage with
    the local shift): bitwise equal to the one-step sweep; the residual step
    after two-step launches also matches."""
    p = w.variable_tensor(n=70, alpha=1e-2, walls=True, t_end=0.2)
    p = p.replace(dt=20.0 * p.dx ** 2, nsteps=11, phi_ref=0.0)
    a = _lattice(p, "f32", "f32", shift="ref").set_sweep_variant("tb2")
    b = _lattice(p, "f32", "f32", shift="ref").set_sweep_variant("plain")
    a.init(p.phi0()).step(p.nsteps)
    b.init(p.phi0()).step(p.nsteps)
    assert np.array_equal(a.phi_host(), b.phi_host())
    assert a.step_residual(5) == b.step_residual(5)
    q = w.nonlinear_modes(n=4096, nsteps=4).replace(nx=4099, ny=4093)
    for storage, shift in (("f32", "ref"), ("f16", "local")):
        a = _lattice(q, "f32", storage, shift=shift).set_sweep_variant("tb2")
        a.init(q.phi0()).step(4)
        pa = a.phi_host()
        del a
        b = _lattice(q, "f32", storage, shift=shift).set_sweep_variant("plain")
        b.init(q.phi0()).step(4)
        assert np.array_equal(pa, b.phi_host())
        del b


@pytest.mark.parametrize("which", ["mms", "nonlinear"])
def test_tb2_full_size_matches_oracle_two_steps(which):
    """The default FP32 form (two steps per launch) at the benchmark's 8192^2
    against the oracle at sampled nodes (corners, edges, tile seams, interior):
    the oracle takes the nine neighbours one single-node step from the GPU's state,
    then the node itself a second step from those (FP32 tolerance)."""
    import torch
    n = 8192
    p = (w.mms_sinsin(n=n, nsteps=4) if which == "mms" else w.nonlinear_modes(n=n, nsteps=4))
    if which != "mms":
        p.phi_ref = float(p.phi0().mean())
    lat = _lattice(p, "f32", "f32", shift="ref")
    lat.init(p.phi0(), t0=p.t0).step(3)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (31, 15), (32, 16), (5000, 6001), (4095, 0), (17, 8191)]
    win5, phin = {}, {}
    phi_dev = lat.phi()
    for (x, y) in pts:
        w5 = np.zeros((5, 5, 9))
        ph = np.zeros((5, 5))
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                qx, qy = (x + dx) % n, (y + dy) % n
                w5[dy + 2, dx + 2] = lat.read_f(qx, qy, 1, 1)[:, 0, 0]
                ph[dy + 2, dx + 2] = float(phi_dev[qy, qx].item())
        win5[(x, y)], phin[(x, y)] = w5, ph
    _, t_now = lat.time()
    lat.step(2)   # one two-step launch
    torch.cuda.synchronize()
    walled = which == "mms"
    for (x, y) in pts:
        w5, ph = win5[(x, y)], phin[(x, y)]
        mid = np.zeros((3, 3, 9))
        phi1 = 0.0
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                qx, qy = x + dx, y + dy
                if walled and not (0 <= qx < n and 0 <= qy < n):
                    continue   # beyond a wall: never pulled
                f1, p1 = oracle.node_step(p, w5[dy + 1:dy + 4, dx + 1:dx + 4], qx % n, qy % n, ph[dy + 2, dx + 2],
                                          t_now + p.dt)
                mid[dy + 1, dx + 1] = f1
                if dx == 0 and dy == 0:
                    phi1 = p1
        f2, _ = oracle.node_step(p, mid, x, y, phi1, t_now + 2 * p.dt)
        got = lat.read_f(x, y, 1, 1)[:, 0, 0]
        assert np.allclose(got, f2, rtol=2e-5, atol=2e-5 * np.abs(f2).max()), (x, y)


def test_tb2_rejects_other_compute():
    """The two-step form serves FP32-compute lattices only."""
    from paper_1902_09813_gb300 import _capi as C
    p = w.random_state_problem(20, 20, seed=2)
    with pytest.raises(C.BtrtError):
        _lattice(p, "df64").set_sweep_variant("tb2")
    with pytest.raises(C.BtrtError):
        _lattice(p, "f64").set_sweep_variant("tb2")
