"""Config-2 convergence sweep on the GPU: the manufactured solution
phi* = exp(-t) sin(pi x) sin(pi y) with bounce-back walls on the unit square,
anisotropic A = R(pi/6) diag(0.05, 0.01) R(pi/6)^T, u = (0.05, 0.02), under
diffusive scaling dt = 4 dx^2 up to T_end = 0.1, at N = 64 ... 512.

Checked here:
- the FP64 sweep equals the FP64 oracle element-wise (rel L2 <= 1e-11) at every N;
- the FP64 sweep is second order in dx (the paper's claim for its anisotropic
  tests, Sec. 4.2.2 and Table 6), observed order within [1.9, 2.1];
- the reduced-precision bar: a format's GRE against the closed form (Eq. 63)
  within 1 % of the FP64 sweep's, at every (N, format) this design claims;
- where a format misses the bar, a regression test pins the measured relative
  GRE change, so that the miss is reported as it is and any change to it shows.

Under diffusive scaling a step changes phi by O(dx^2) relative, a few FP32 ulps
at N = 512, so an FP32-compute path whose phi plane is rounded to FP32 every step
drifts from the FP64 result as N grows, whatever the storage format.  FP64 and
double-word compute do not, nor does FP32 compute with FP32 storage and phi kept
as a double-word pair (BTRT_SHIFT_LOCAL_DW); with 16-bit storage the rounding of
the stored deviations then dominates, and the pair does not move the bar.  Rounding the stored 16-bit deviations
stochastically (BTRT_SHIFT_LOCAL_SR) removes the error that round-to-nearest
repeats step after step and cuts the misses by one to three orders of magnitude;
with FP16 deviations scaled by 2^12 (out of FP16's subnormal range) FP16 storage
stays within the bar through 512^2, BF16 (8 significant bits) only at 64^2."""
import math

import numpy as np
import pytest

import oracle
import workloads as w
from conftest import cpu_threads

pytestmark = pytest.mark.gpu

SIDES = (64, 128, 256, 512)
BAR = 0.01
TOL64 = 1e-11

# (compute, storage, shift) -> the N at which the design claims the 1 % bar
CLAIMED = {
    ("df64", "df64", "ref"): (64, 128, 256, 512),
    ("f32", "f32", "ref"): (64,),
    ("f32", "f32", "local"): (64, 128),
    ("f32", "f16", "local"): (64, 128),
    ("f32", "bf16", "local"): (64,),
    # phi as a double-word pair: FP32 storage within the bar at every N (2048^2: -0.98 %)
    ("f32", "f32", "local_dw"): (64, 128, 256, 512),
    ("f32", "f16", "local_dw"): (64, 128),
    ("f32", "bf16", "local_dw"): (64,),
    # stochastically rounded 16-bit deviations (FP16 scaled by 2^12): FP16 within the bar
    # through 512^2 (1024^2: -1.6 %, with the double-word phi +1.04 %), BF16 at 64^2
    ("f32", "f16", "local_sr"): (64, 128, 256, 512),
    ("f32", "bf16", "local_sr"): (64,),
    ("f32", "f16", "local_dw_sr"): (64, 128, 256, 512),
    ("f32", "bf16", "local_dw_sr"): (64,),
    # the first-moment form (deviations from w_i (phi + 3 e_i . j), stochastic rounding of
    # them and of phi): FP16 and BF16 within the bar through 1024^2
    ("f32", "f16", "moment_sr"): (64, 128, 256, 512),
    ("f32", "bf16", "moment_sr"): (64, 128, 256, 512),
}
# measured misses: (compute, storage, shift, N) -> (low, high) bounds of the
# relative GRE change against the FP64 sweep (measured value in the comment)
MISSES = {
    ("f32", "f32", "ref", 128): (-0.030, -0.018),     # -0.0241
    ("f32", "f32", "ref", 512): (9.0, 14.5),          # 11.65
    ("f32", "f32", "local", 256): (-0.080, -0.045),   # -0.0624
    ("f32", "f32", "local", 512): (2.0, 3.2),         # 2.562
    ("f32", "f16", "local", 256): (0.080, 0.130),     # 0.1043
    ("f32", "f16", "local", 512): (1.8, 2.8),         # 2.260
    ("f32", "bf16", "local", 128): (0.180, 0.280),    # 0.2273
    ("f32", "bf16", "local", 256): (4.8, 7.4),        # 6.077
    ("f32", "f16", "local_dw", 256): (0.085, 0.135),  # 0.1075: the 16-bit deviations' rounding, not phi
    ("f32", "bf16", "local_dw", 128): (0.18, 0.28),   # 0.2243
    ("f32", "bf16", "local_sr", 128): (0.013, 0.033),  # 0.0217 (round-to-nearest: 0.2273)
    ("f32", "bf16", "local_sr", 256): (0.028, 0.068),  # 0.0455 (round-to-nearest: 6.077)
    ("f32", "bf16", "local_sr", 512): (0.055, 0.135),  # 0.0894
    ("f32", "bf16", "local_dw_sr", 128): (0.014, 0.035),  # 0.0230
    ("f32", "f16", "local_sr", 1024): (-0.022, -0.0115),   # -0.01604: the FP32 phi plane's rounding
    ("f32", "f16", "local_dw_sr", 1024): (0.0101, 0.016),  # 0.01038, just past the bar
}


def _problem(n):
    return w.mms_sinsin(n=n)


_CACHE = {}


def _gre_gpu(n, compute, storage, shift):
    key = (n, compute, storage, shift)
    if key not in _CACHE:
        from paper_1902_09813_gb300 import Lattice
        p = _problem(n)
        lat = Lattice.from_problem(p, compute=compute, storage=storage, shift=shift)
        lat.init(p.phi0(), t0=p.t0).step(p.nsteps)
        phi = lat.phi_host()
        assert lat.check() == 0
        _CACHE[key] = (phi, w.gre(phi, w.mms_sinsin_exact(p, p.t0 + p.nsteps * p.dt)))
    return _CACHE[key]


@pytest.mark.parametrize("n", SIDES)
def test_fp64_sweep_equals_oracle_across_the_sweep(n):
    p = _problem(n)
    phi, _ = _gre_gpu(n, "f64", "f64", "ref")
    ref = oracle.OracleLattice(p, nthreads=cpu_threads()).init().step(p.nsteps).phi()
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err <= TOL64, (n, err)


def test_fp64_sweep_is_second_order():
    g = [_gre_gpu(n, "f64", "f64", "ref")[1] for n in SIDES]
    orders = [math.log2(g[i - 1] / g[i]) for i in range(1, len(g))]
    assert all(1.9 <= o <= 2.1 for o in orders), (g, orders)


@pytest.mark.parametrize("fmt,n", [(f, n) for f, ns in CLAIMED.items() for n in ns],
                         ids=lambda v: "-".join(v) if isinstance(v, tuple) else str(v))
def test_reduced_format_within_bar(fmt, n):
    g64 = _gre_gpu(n, "f64", "f64", "ref")[1]
    g = _gre_gpu(n, *fmt)[1]
    assert abs(g / g64 - 1.0) <= BAR, (fmt, n, g, g64)


@pytest.mark.parametrize("case", list(MISSES), ids=lambda c: "-".join(map(str, c)))
def test_reduced_format_misses_bar_regression(case):
    """Not a bar: the measured miss, pinned so that it stays reported as it is."""
    c, s, sh, n = case
    lo, hi = MISSES[case]
    rel = _gre_gpu(n, c, s, sh)[1] / _gre_gpu(n, "f64", "f64", "ref")[1] - 1.0
    assert abs(rel) > BAR
    assert lo <= rel <= hi, (case, rel)


def test_double_word_phi_within_bar_at_1024():
    """FP32 compute and storage with phi as a double-word pair at 1024^2 (26214
    steps): within the bar and second order from 512^2, where the FP32 phi plane
    drifts by 2282 %."""
    g64 = [_gre_gpu(n, "f64", "f64", "ref")[1] for n in (512, 1024)]
    g = [_gre_gpu(n, "f32", "f32", "local_dw")[1] for n in (512, 1024)]
    assert abs(g[1] / g64[1] - 1.0) <= BAR, (g, g64)
    assert 1.9 <= math.log2(g[0] / g[1]) <= 2.1


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_first_moment_form_within_bar_at_1024(storage):
    """FP16 and BF16 storage of the first-moment form (BTRT_SHIFT_MOMENT_SR) at 1024^2
    (26214 steps): within the bar (FP16 -0.16 %, BF16 -0.95 %) and second order from
    512^2; with the local shift BF16 misses by +48 % there (stochastic rounding) or
    +1.5e5 % (round to nearest)."""
    g64 = [_gre_gpu(n, "f64", "f64", "ref")[1] for n in (512, 1024)]
    g = [_gre_gpu(n, "f32", storage, "moment_sr")[1] for n in (512, 1024)]
    assert abs(g[1] / g64[1] - 1.0) <= BAR, (g, g64)
    assert 1.9 <= math.log2(g[0] / g[1]) <= 2.1
