"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a printed matrix
or number from the paper, an identity of the equilibrium, an exact discrete
steady state, a closed-form PDE solution with its convergence order, or a
textbook scheme the method reduces to.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads, load_matrix, paper_value

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _problem(**kw):
    base = dict(name="unit", nx=4, ny=4, dx=0.1, dt=0.02, u=(0.3, -0.2), b2=0.7, c3=0.4,
                A0=(0.002, 0.0007, 0.001), a2=0.5, k0=1.1)
    base.update(kw)
    return w.Problem(**base)


# --------------------------------------------------------------- Eq. 9 / Eq. 10
@pytest.mark.parametrize("phi", [-0.7, 0.0, 0.35, 1.9])
def test_equilibrium_moments(phi):
    """sum f_eq = phi, sum c f_eq = B(phi), sum c c f_eq = cs^2 C(phi) I (Eq. 9)."""
    p = _problem()
    c = p.dx / p.dt
    cs2 = c * c / 3.0
    feq = oracle.feq(p, phi)
    cx, cy = c * EX, c * EY
    B = np.array([p.u[0] * phi + p.b2 * phi * phi / 2, p.u[1] * phi + p.b2 * phi * phi / 2])
    C = phi + p.c3 * phi ** 3
    assert feq.sum() == pytest.approx(phi, abs=1e-14)
    assert np.allclose([np.dot(cx, feq), np.dot(cy, feq)], B, atol=1e-13, rtol=0)
    M2 = np.array([[np.dot(cx * cx, feq), np.dot(cx * cy, feq)],
                   [np.dot(cy * cx, feq), np.dot(cy * cy, feq)]])
    assert np.allclose(M2, cs2 * C * np.eye(2), atol=1e-12, rtol=0)


def test_source_moments():
    """With f = f_eq and no time variation the collision adds dt S_i with
    sum S_i = S and sum c_i S_i = 0 (Eq. 8, Eq. 10)."""
    p = _problem(source=w.Source(kind="const", const=0.37), u=(0.0, 0.0), b2=0.0)
    phi = 0.8
    f = oracle.feq(p, phi)
    fp = oracle.collide(p, f, phi, 0.0, 0.0, 1.0, 1.0)
    d = fp - f
    assert d.sum() == pytest.approx(p.dt * 0.37, rel=1e-13)
    assert abs(np.dot(EX, d)) < 1e-16 and abs(np.dot(EY, d)) < 1e-16
    weights = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    assert np.allclose(d, p.dt * 0.37 * weights, rtol=1e-13, atol=0)


# --------------------------------------------------------------- appendix matrices
def _relax_matrix(k0, K1, K2, c=1.0):
    """Columns = relaxation term of Eq. 6 applied to unit non-equilibrium vectors."""
    M = np.zeros((9, 9))
    for j in range(9):
        e = np.zeros(9)
        e[j] = 1.0
        M[:, j] = oracle.relax(k0, K1, K2, c, e)
    return M


@pytest.mark.parametrize("k0,k1,k2", [(1.0, 1.25, 0.7273), (0.6, 1.7, 1.3), (1.4, 0.3, 1.9)])
@pytest.mark.parametrize("c", [1.0, 5.0])
def test_printed_R_and_P(k0, k1, k2, c):
    """k0 I + R + P with K1 = k1 I, K2 = k2 Ihat equals the printed Eqs. 78-79."""
    R, _ = load_matrix("d2q9_R.txt")
    P, _ = load_matrix("d2q9_P.txt")
    expect = k0 * np.eye(9) + (k1 - k0) / 12.0 * R + (k2 - k0) / 12.0 * P
    got = _relax_matrix(k0, k1 * np.eye(2), k2 * np.ones((2, 2)), c)
    assert np.allclose(got, expect, atol=1e-13, rtol=0)


def test_T_is_H_times_C():
    """T = H C (Eq. 87) with the printed Eqs. 85, 88, 90."""
    C, sc = load_matrix("d2q9_C.txt")
    H, sh = load_matrix("d2q9_H.txt")
    T, st = load_matrix("d2q9_T.txt")
    assert np.allclose((sh * H) @ (sc * C), st * T, atol=1e-15)


def test_T_rows_are_oracle_moments():
    """Row 0..5 of C are the moments the oracle relaxes: their columns are
    1, c_x, c_y, c_x^2, c_x c_y, c_y^2 of the velocity set (Eq. 83)."""
    C, _ = load_matrix("d2q9_C.txt")
    expect = np.stack([np.ones(9), EX, EY, EX * EX, EX * EY, EY * EY,
                       EX * EX * EY, EX * EY * EY, EX * EX * EY * EY])
    assert np.array_equal(C, expect)


@pytest.mark.parametrize("k0,k1,k2", [(1.0, 1.25, 0.7273), (0.6, 1.7, 1.3)])
def test_block_diagonal_Sf(k0, k1, k2):
    """T (k0 I + R + P) T^{-1} = diag(k0, k1, k1, k2, k2, k2, k0, k0, k0) (Eqs. 92, 95)."""
    T, st = load_matrix("d2q9_T.txt")
    T = st * T
    Om = _relax_matrix(k0, k1 * np.eye(2), k2 * np.ones((2, 2)))
    S = T @ Om @ np.linalg.inv(T)
    assert np.allclose(S, np.diag([k0, k1, k1, k2, k2, k2, k0, k0, k0]), atol=1e-13)


def test_full_block_Sf_general_K1_K2():
    """With general (non-symmetric) K1 and K2 the relaxation matrix is block
    diagonal with K1 on moments 1-2 and K2 entries on 3-5 (Eqs. 98-99)."""
    T, st = load_matrix("d2q9_T.txt")
    T = st * T
    k0 = 0.9
    K1 = np.array([[1.3, 0.21], [-0.17, 0.8]])
    K2 = np.array([[0.7, 0.45], [0.15, 1.6]])
    S = T @ _relax_matrix(k0, K1, K2) @ np.linalg.inv(T)
    expect = np.zeros((9, 9))
    expect[0, 0] = k0
    expect[1:3, 1:3] = K1
    expect[3, 3] = K2[0, 0]
    expect[4, 4] = 0.5 * (K2[0, 1] + K2[1, 0])
    expect[5, 5] = K2[1, 1]
    expect[6, 6] = expect[7, 7] = expect[8, 8] = k0
    assert np.allclose(S, expect, atol=1e-13)


# --------------------------------------------------------------- Eq. 30, Eq. 62
def test_K1_recovers_diffusion_tensor():
    """A = cs^2 (K1^{-1} - I/2) dt (Eq. 30) for the oracle's K1 at several phi."""
    p = _problem()
    c = p.dx / p.dt
    cs2 = c * c / 3.0
    for phi in (-0.5, 0.0, 1.3):
        K1 = oracle.K1(p, phi)
        s = 1.0 + p.a2 * phi * phi
        A = s * np.array([[p.A0[0], p.A0[1]], [p.A0[1], p.A0[2]]])
        assert np.allclose(cs2 * (np.linalg.inv(K1) - 0.5 * np.eye(2)) * p.dt, A, rtol=1e-12, atol=0)


def test_k2_relation_printed_value():
    """Eq. 62 at k1 = 1.25 gives the optimal k2 the paper prints (0.7273)."""
    assert round(oracle.k2_from_k1(1.25), 4) == paper_value("k2_optimal_k1_1.25")


# --------------------------------------------------------------- Sec. 3 / Sec. 4.1.1
@pytest.mark.parametrize("n", [5, 10])
def test_steady_diffusion_exact_with_eq62(n):
    """With k2 from Eq. 62 the half-way bounce-back steady state equals the exact
    solution phi0 + dphi y(2 - y) to machine precision (Sec. 4.1.1: GRE ~1e-10)."""
    p = w.steady_diffusion(n=n, nsteps=8000 if n == 5 else 30000)
    lat = oracle.run(p, nthreads=cpu_threads())
    err = w.gre(lat.phi(), w.steady_diffusion_exact(p))
    assert err < paper_value("gre_steady_obtrirt")
    assert err < 1e-12


@pytest.mark.parametrize("k2", [1.0, 0.5, 1.2])
def test_numerical_slip_eq61(k2):
    """With another k2 the steady state is the exact solution shifted by the
    numerical slip phi_s = (3 k1 k2 - 8 k1 - 12 k2 + 16) dphi / (12 k1 k2 N^2) (Eq. 61)."""
    n, k1 = 5, 1.25
    p = w.steady_diffusion(n=n, k1=k1, k2_mode="const", k2=k2, nsteps=20000)
    lat = oracle.run(p, nthreads=cpu_threads())
    diff = lat.phi() - w.steady_diffusion_exact(p)
    slip = (3 * k1 * k2 - 8 * k1 - 12 * k2 + 16) / (12 * k1 * k2) * 1.0 / n ** 2
    assert np.allclose(diff, slip, atol=1e-11, rtol=0)


# --------------------------------------------------------------- conservation, BGK
def test_mass_conservation_periodic():
    """sum phi is conserved to rounding on a periodic grid without a source,
    including the nonlinear B, C, A terms and the d_t B correction."""
    p = w.random_state_problem(24, 20, seed=3, nonlinear=True, source="none")
    lat = oracle.OracleLattice(p).init()
    m0 = lat.mass()
    lat.step(200)
    assert abs(lat.mass() - m0) < 1e-12 * abs(m0)


def _textbook_bgk_diffusion(phi0, tau, nsteps):
    """Textbook D2Q9 BGK for pure diffusion: f_eq = w phi, stream by np.roll."""
    wts = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = wts[:, None, None] * phi0[None]
    for _ in range(nsteps):
        phi = f.sum(0)
        feq = wts[:, None, None] * phi[None]
        f = f - (f - feq) / tau
        f = np.stack([np.roll(np.roll(f[i], EX[i], axis=1), EY[i], axis=0) for i in range(9)])
    return f.sum(0)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_reduces_to_textbook_bgk(tau):
    """k0 = k1 = k2 = 1/tau with A = cs^2 (tau - 1/2) dt is the LBGK model (Table 1)."""
    a = (tau - 0.5) / 3.0
    p = w.gaussian_hill(n=20, sigma0=3.0, u=(0.0, 0.0), A0=(a, 0.0, a), nsteps=60,
                        k2_mode="const", k2=1.0 / tau, k0=1.0 / tau)
    lat = oracle.run(p)
    ref = _textbook_bgk_diffusion(p.phi0(), tau, p.nsteps)
    assert np.allclose(lat.phi(), ref, atol=1e-13, rtol=0)


# --------------------------------------------------------------- closed forms
def test_gaussian_hill_second_order():
    """Full-tensor Gaussian hill (Eqs. 70-72): the error against the closed form
    falls by ~4 per halving of dx at fixed dx^2/dt (Sec. 4.2.1, Fig. 12)."""
    errs = []
    for m in (1, 2, 4):
        n = 48 * m
        p = w.gaussian_hill(n=n, sigma0=3.0, dx=1.0 / m, dt=1.0 / m ** 2, u=(0.05, 0.03),
                            A0=(0.01, 0.01, 0.02), nsteps=150 * m * m, k2_mode="const", k2=1.0)
        p.meta["centre"] = (24.0, 24.0)
        p.phi0_fn = lambda X, Y: np.exp(-((X - 24.0) ** 2 + (Y - 24.0) ** 2) / 18.0)
        lat = oracle.run(p, nthreads=cpu_threads())
        errs.append(w.gre(lat.phi(), w.gaussian_hill_exact(p, 150.0)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_manufactured_solution_second_order():
    """Full-tensor manufactured solution with bounce-back walls: second order."""
    errs = []
    for n in (16, 32, 64):
        p = w.mms_sinsin(n=n, kappa=4.0, t_end=0.1)
        lat = oracle.run(p, nthreads=cpu_threads())
        errs.append(w.gre(lat.phi(), w.mms_sinsin_exact(p, p.nsteps * p.dt)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


# --------------------------------------------------------------- printed errors
@pytest.mark.parametrize("u0,key", [(0.01, "gre_table3_u0.01"), (0.1, "gre_table3_u0.1"),
                                    (2.5, "gre_table3_u2.5")])
def test_paper_table3(u0, key):
    """Linear CDE with bounce-back walls carrying the exact solution,
    dx = 1/50, c = 5, tau = 0.8, t = 1 (Table 3): GRE within 10% of the print."""
    p = w.linear_cde(n=100, alpha=0.01, u=(u0, u0), c=5.0, t_end=1.0, walls=True)
    assert oracle.K1(p, 0.0)[0, 0] == pytest.approx(1.0 / 0.8, rel=1e-12)
    lat = oracle.run(p, nthreads=cpu_threads())
    err = w.gre(lat.phi(), w.linear_cde_exact(p, p.nsteps * p.dt))
    assert err == pytest.approx(paper_value(key), rel=0.10)


@pytest.mark.parametrize("alpha,key", [(0.01, "gre_lincde_200_a1e-2"), (1e-4, "gre_lincde_200_a1e-4")])
def test_paper_linear_cde_200(alpha, key):
    """Linear CDE on the periodic [0,2]^2, 200 x 200, c = 1, t = 3 (Sec. 4.1.2):
    GRE within 15% of the printed value."""
    p = w.linear_cde(n=200, alpha=alpha, u=(0.1, 0.1), c=1.0, t_end=3.0)
    lat = oracle.run(p, nthreads=cpu_threads())
    err = w.gre(lat.phi(), w.linear_cde_exact(p, p.nsteps * p.dt))
    assert err == pytest.approx(paper_value(key), rel=0.15)


# --------------------------------------------------------------- internal consistency
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (0, 0, 1, 1)])
def test_node_step_matches_grid_step(bc):
    """The single-node pull form used for sampled full-size checks equals the
    grid step (push form, Eq. 38 with Eqs. 54-56) at every node."""
    p = w.random_state_problem(7, 6, seed=5, bc=bc)
    lat = oracle.OracleLattice(p).init()
    lat.step(3)
    fpost_t = lat.fpost.copy()
    phi_prev = lat.phi_prev.copy()   # phi at the last collision time
    t_next = lat.t
    lat.step(1)
    for iy in range(p.ny):
        for ix in range(p.nx):
            win = np.zeros((3, 3, 9))
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    win[dy + 1, dx + 1] = fpost_t[:, (iy + dy) % p.ny, (ix + dx) % p.nx]
            fp, phi = oracle.node_step(p, win, ix, iy, phi_prev[iy, ix], t_next)
            assert np.allclose(fp, lat.fpost[:, iy, ix], rtol=0, atol=1e-14)
            assert phi == pytest.approx(lat.phi_prev[iy, ix], abs=1e-14)


@pytest.mark.parametrize("alpha,n,key,tol", [(1e-4, 200, "gre_table6_a1e-4_dx200", 0.06),
                                             (1e-6, 200, "gre_table6_a1e-6_dx200", 0.06),
                                             (1e-6, 400, "gre_table6_a1e-6_dx400", 0.06)])
def test_table6_variable_tensor_small_alpha(alpha, n, key, tol):
    """Table 6 (Sec. 4.2.2): periodic unit square, c = 1, t = 3, u = (0.1, 0.1), and
    k2 = 1 as the paper sets for its anisotropic runs."""
    from conftest import paper_value
    p = w.variable_tensor(n=n, alpha=alpha, walls=False, t_end=3.0).replace(k2_mode="const", k2=1.0)
    lat = oracle.run(p, nthreads=cpu_threads())
    err = w.gre(lat.phi(), w.variable_tensor_exact(p, p.nsteps * p.dt))
    assert err == pytest.approx(paper_value(key), rel=tol)


def test_variable_tensor_second_order():
    """Spatially varying diffusion tensor with its manufactured source (Sec. 4.2.2,
    Eqs. 73-76): second order under diffusive scaling (dt = 20 dx^2)."""
    errs = []
    for n in (25, 50, 100):
        p = w.variable_tensor(n=n, alpha=1e-2, walls=True, t_end=0.5)
        dt = 20.0 * p.dx ** 2
        p = p.replace(dt=dt, nsteps=int(round(0.5 / dt)))
        lat = oracle.run(p, nthreads=cpu_threads())
        errs.append(w.gre(lat.phi(), w.variable_tensor_exact(p, p.nsteps * p.dt)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.7 < r1 < 4.3 and 3.7 < r2 < 4.3, errs
