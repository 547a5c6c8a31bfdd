"""The GPU collision evaluates some terms of the scheme in rearranged forms to
take fewer operations; these tests check symbolically that each rearrangement is
an identity (exact algebra, rounding aside):

- the first-order term of Eq. 95 with the correction of Eq. 11,
  k0 B - (K1 - k0 I)(M1 - B) + (I - K1/2) dB  ==  K1 (B - M1 - dB/2) + k0 M1 + dB,
  and, for B = u phi and dB = u dphi with dphi = phi - phi_prev,
  K1 u phi - (K1 - k0 I) M1 + (I - K1/2) u phi - (I - K1/2) u phi_prev
  (2-D with a general 2 x 2 K1, 3-D with a general 3 x 3 K1);
- the D2Q9 second-order weights: w1 kap / 6 == (2/3) w5 kap == (k2 - k0) / 12 and
  w0 kap / 3 == (2/3)(k2 - k0), kap = (9/2)(k2 - k0);
- the D3Q19 second-order terms: with M2 = Pi - (C - rs)/3 I, t3 = tr(M2)/3 and
  h_a = Pi_aa - tr(Pi)/3, M2_aa - t3 == h_a and M2_aa + M2_bb - t3 == t3 - h_c for the
  face diagonals normal to axis c; w_i kap == (3/2, 1/4, 1/8)(k2 - k0)."""
import pytest

sp = pytest.importorskip("sympy")


def _first_order_identity(dim):
    K1 = sp.Matrix(dim, dim, lambda i, j: sp.Symbol(f"K{i}{j}"))
    k0 = sp.Symbol("k0")
    I = sp.eye(dim)
    B = sp.Matrix(dim, 1, lambda i, _: sp.Symbol(f"B{i}"))
    M1 = sp.Matrix(dim, 1, lambda i, _: sp.Symbol(f"j{i}"))
    dB = sp.Matrix(dim, 1, lambda i, _: sp.Symbol(f"dB{i}"))
    paper = k0 * B - (K1 - k0 * I) * (M1 - B) + (I - K1 / 2) * dB
    gpu = K1 * (B - M1 - dB / 2) + k0 * M1 + dB
    assert sp.simplify(paper - gpu) == sp.zeros(dim, 1)
    # constant coefficients: B = u phi, dB = u (phi - phi_prev)
    u = sp.Matrix(dim, 1, lambda i, _: sp.Symbol(f"u{i}"))
    phi, phi_prev = sp.symbols("phi phi_prev")
    paper_lin = paper.subs({**{B[i]: u[i] * phi for i in range(dim)},
                            **{dB[i]: u[i] * (phi - phi_prev) for i in range(dim)}})
    P = K1 * u
    g = u - P / 2
    gpu_lin = (P + g) * phi - g * phi_prev - (K1 - k0 * I) * M1
    assert sp.simplify(paper_lin - gpu_lin) == sp.zeros(dim, 1)


def test_first_order_term_2d():
    _first_order_identity(2)


def test_first_order_term_3d():
    _first_order_identity(3)


def test_d2q9_second_order_weights():
    k0, k2 = sp.symbols("k0 k2")
    kap = sp.Rational(9, 2) * (k2 - k0)
    w0, w1, w5 = sp.Rational(4, 9), sp.Rational(1, 9), sp.Rational(1, 36)
    assert sp.simplify(w1 * kap / 6 - (k2 - k0) / 12) == 0
    assert sp.simplify(sp.Rational(2, 3) * w5 * kap - (k2 - k0) / 12) == 0
    assert sp.simplify(w0 * kap / 3 - sp.Rational(2, 3) * (k2 - k0)) == 0


def test_d3q19_second_order_terms():
    Pxx, Pyy, Pzz, cmid = sp.symbols("Pxx Pyy Pzz cmid")
    M = {a: P - cmid / 3 for a, P in (("x", Pxx), ("y", Pyy), ("z", Pzz))}
    t3 = (M["x"] + M["y"] + M["z"]) / 3
    trP = Pxx + Pyy + Pzz
    h = {a: P - trP / 3 for a, P in (("x", Pxx), ("y", Pyy), ("z", Pzz))}
    assert sp.simplify(t3 - (trP / 3 - cmid / 3)) == 0
    for a in "xyz":
        assert sp.simplify(M[a] - t3 - h[a]) == 0
    for a, b, c in (("x", "y", "z"), ("x", "z", "y"), ("y", "z", "x")):
        assert sp.simplify(M[a] + M[b] - t3 - (t3 - h[c])) == 0
    k0, k2 = sp.symbols("k0 k2")
    kap = sp.Rational(9, 2) * (k2 - k0)
    for w, c in ((sp.Rational(1, 3), sp.Rational(3, 2)), (sp.Rational(1, 18), sp.Rational(1, 4)),
                 (sp.Rational(1, 36), sp.Rational(1, 8))):
        assert sp.simplify(w * kap - c * (k2 - k0)) == 0
