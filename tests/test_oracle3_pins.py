"""Pins of the D3Q19 oracle (oracle/btrt_oracle3.c) against what the paper and
the mathematics fix, independently of the oracle itself:

- the velocity set and moment matrix C of Eq. 86 (printed), the relaxation
  matrices R and P of Eq. 77 against the printed Eqs. 80 and 81 (one printed
  entry of Eq. 80 is a sign misprint, checked against the row structure),
- T of Eq. 89 block-diagonalises k0 I + R + P into the S_f of Eq. 96, and
  general K1, K2 into the blocks of Eq. 100 (a non-symmetric K1 catches a
  transposed operand),
- the equilibrium moments of Eq. 9, mass conservation, reduction to a textbook
  D3Q19 BGK scheme (Table 1), the exact parabolic steady state between
  bounce-back walls with k2 from Eq. 62, and second-order convergence to the
  closed-form anisotropic Gaussian hill.
"""
import numpy as np
import pytest

import workloads as w
from conftest import cpu_threads, load_matrix
from oracle import d3q19 as o3

C3 = 1.0   # lattice speed for the matrix pins


def _matrix(k0, K1, K2):
    """k0 I + R + P as a 19 x 19 matrix (columns from unit vectors)."""
    cols = [o3.RP(k0, K1, K2, C3, np.eye(19)[j]) for j in range(19)]
    return np.array(cols).T + k0 * np.eye(19)


def _R(k0, k1):
    return _matrix(k0, k1 * np.eye(3), np.full((3, 3), k0)) - k0 * np.eye(19)


def _P(k0, k2):
    return _matrix(k0, k0 * np.eye(3), np.full((3, 3), k2)) - k0 * np.eye(19)


def test_velocity_set_and_C_matrix():
    c, wt = o3.lattice()
    Cp, s = load_matrix("d3q19_C.txt")
    order = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 0, 1), (1, 1, 0), (0, 1, 1), (0, 2, 0),
             (0, 0, 2), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 0, 2), (0, 1, 2), (0, 2, 1), (2, 2, 0), (2, 0, 2),
             (0, 2, 2)]
    C = np.array([[c[i, 0] ** a * c[i, 1] ** b * c[i, 2] ** g for i in range(19)] for a, b, g in order])
    assert np.array_equal(C, Cp * s)
    # weights: isotropy up to fourth order with cs^2 = 1/3
    assert wt.sum() == pytest.approx(1.0, abs=1e-15)
    for a in range(3):
        for b in range(3):
            assert (wt * c[:, a] * c[:, b]).sum() == pytest.approx(1 / 3 if a == b else 0.0, abs=1e-15)
    assert (wt * c[:, 0] ** 2 * c[:, 1] ** 2).sum() == pytest.approx(1 / 9, abs=1e-15)
    assert (wt * c[:, 0] ** 4).sum() == pytest.approx(1 / 3, abs=1e-15)


def test_R_matches_eq80_up_to_one_misprint():
    k0, k1 = 0.9, 1.9
    R = _R(k0, k1) / (k1 - k0)
    Rp, s = load_matrix("d3q19_R.txt")
    Rp = Rp * s
    bad = [tuple(int(v) for v in ij) for ij in np.argwhere(np.abs(R - Rp) > 1e-12)]
    # Eq. 80 prints R[2][7] = +2/12; c_2 = -c_1 makes row 2 the negative of row 1,
    # and the printed row 1 has R[1][7] = +2/12, so the entry must be -2/12
    assert bad == [(2, 7)]
    assert Rp[1, 7] == pytest.approx(2 / 12) and R[2, 7] == pytest.approx(-Rp[1, 7])
    assert np.allclose(R[2], -R[1], atol=1e-15)


def test_P_matches_eq81():
    k0, k2 = 1.1, 0.6
    P = _P(k0, k2) / (k2 - k0)
    Pp, s = load_matrix("d3q19_P.txt")
    assert np.allclose(P, Pp * s, atol=1e-14, rtol=0)


def test_T_diagonalises_into_eq96():
    Tp, s = load_matrix("d3q19_T.txt")
    T = Tp * s
    k0, k1, k2 = 1.0, 1.37, 0.62
    D = T @ _matrix(k0, k1 * np.eye(3), np.full((3, 3), k2)) @ np.linalg.inv(T)
    expect = np.diag([k0] + [k1] * 3 + [k2] * 6 + [k0] * 9)
    assert np.allclose(D, expect, atol=1e-13)


def test_general_blocks_eq100():
    """Non-symmetric K1 and general K2: the moment-space matrix is the block form
    of Eq. 100 (K1 in the first-order rows, the symmetrised K2 entries on the
    second-order diagonal)."""
    rng = np.random.default_rng(5)
    k0 = 0.95
    K1 = rng.uniform(0.3, 1.6, size=(3, 3))
    K2 = rng.uniform(0.3, 1.6, size=(3, 3))
    Tp, s = load_matrix("d3q19_T.txt")
    T = Tp * s
    D = T @ _matrix(k0, K1, K2) @ np.linalg.inv(T)
    S = np.zeros((19, 19))
    S[0, 0] = k0
    S[1:4, 1:4] = K1
    S[4, 4] = K2[0, 0]
    S[5, 5] = 0.5 * (K2[0, 2] + K2[2, 0])
    S[6, 6] = 0.5 * (K2[0, 1] + K2[1, 0])
    S[7, 7] = 0.5 * (K2[1, 2] + K2[2, 1])
    S[8, 8] = K2[1, 1]
    S[9, 9] = K2[2, 2]
    for k in range(10, 19):
        S[k, k] = k0
    assert np.allclose(D, S, atol=1e-13)


@pytest.mark.parametrize("phi", [-0.4, 0.3, 1.7])
def test_equilibrium_moments_eq9(phi):
    p = w.random_state_problem3(6, 5, 4, seed=2, nonlinear=True).replace(dx=0.5, dt=0.25)
    c, wt = o3.lattice()
    cl = p.dx / p.dt
    f = o3.feq(p, phi)
    assert f.sum() == pytest.approx(phi, abs=1e-14)
    assert np.allclose((cl * c * f[:, None]).sum(0), o3.B(p, phi), atol=1e-14)
    M2 = np.einsum("i,ia,ib->ab", f, cl * c, cl * c)
    Cphi = phi + p.c3 * phi ** 3
    assert np.allclose(M2, cl * cl / 3.0 * Cphi * np.eye(3), atol=1e-13)


def test_mass_conservation_periodic():
    p = w.random_state_problem3(9, 7, 6, seed=11, nonlinear=True, source="none")
    lat = o3.OracleLattice3(p, nthreads=cpu_threads()).init()
    m0 = lat.phi().sum()
    lat.step(12)
    assert abs(lat.phi().sum() - m0) <= 1e-13 * abs(m0)


def _bgk_d3q19(phi0, tau, nsteps):
    """Textbook D3Q19 BGK for pure diffusion: f_eq = w_i phi, relax by 1/tau, stream."""
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0], [1, 0, 1], [-1, 0, 1], [1, 0, -1],
                  [-1, 0, -1], [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1]])
    wt = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = wt[:, None, None, None] * phi0[None]
    for _ in range(nsteps):
        phi = f.sum(0)
        f = f - (f - wt[:, None, None, None] * phi[None]) / tau
        for i in range(19):
            f[i] = np.roll(f[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
    return f.sum(0)


def test_lbgk_reduction_table1():
    tau = 0.85
    a = (tau - 0.5) / 3.0
    p = w.gaussian_hill3(n=10, sigma0=2.0, u=(0.0, 0.0, 0.0), A0=(a, 0.0, 0.0, a, 0.0, a), nsteps=15,
                         k0=1.0 / tau, k2_mode="const", k2=1.0 / tau)
    lat = o3.run(p, nthreads=cpu_threads())
    assert np.allclose(lat.phi(), _bgk_d3q19(p.phi0(), tau, p.nsteps), atol=1e-14, rtol=0)


def test_steady_diffusion_between_walls_exact_with_eq62():
    """Parabolic steady state between bounce-back walls: exact to rounding when k2
    follows Eq. 62 (the D3Q19 form of Sec. 4.1.1)."""
    p = w.steady_diffusion3(n=5, k1=1.25, nsteps=4000)
    lat = o3.run(p, nthreads=cpu_threads())
    err = np.abs(lat.phi() - w.steady_diffusion3_exact(p)).max()
    assert err < 1e-11
    # another k2 leaves a discrete slip of the order of the grid error
    q = p.replace(k2_mode="const", k2=1.0)
    lat = o3.run(q, nthreads=cpu_threads())
    assert np.abs(lat.phi() - w.steady_diffusion3_exact(q)).max() > 1e-4


def test_gaussian_hill3_second_order():
    """Diffusive scaling on the unit periodic cube: errors against the closed form
    fall by about four per halving of dx."""
    errs = []
    for n in (12, 24):
        dx = 1.0 / n
        dt = 2.0 * dx * dx
        p = w.gaussian_hill3(n=n, sigma0=0.12, u=(0.3, -0.2, 0.1),
                             A0=(0.04, 0.008, 0.0, 0.03, -0.006, 0.02), nsteps=int(round(0.1 / dt)),
                             dx=dx, dt=dt)
        lat = o3.run(p, nthreads=cpu_threads())
        errs.append(w.gre(lat.phi(), w.gaussian_hill3_exact(p, p.nsteps * p.dt)))
    assert 3.0 < errs[0] / errs[1] < 6.0, errs
