"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them: a dropped term, a wrong sign, a transposed operand, a
wrong index or time level.  Each mutant is compiled from a textual edit of
oracle/btrt_oracle.c into a temporary library and the pin suite runs against it.
"""
import os
import subprocess
import sys
import tempfile

import pytest

from conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "btrt_oracle.c")

MUTATIONS = {
    "G_sign": ("+ dt * G + dt * Si", "- dt * G + dt * Si"),
    "drop_source_derivative": ("+ 0.5 * dt * dt * DSi", "+ 0.0 * dt * dt * DSi"),
    "K1_transposed": ("QM1[a] += (K1[2 * a + b]", "QM1[a] += (K1[2 * b + a]"),
    "dtB_sign": ("dtB[a] = (Bn[a] - Bp[a]) / dt", "dtB[a] = (Bp[a] - Bn[a]) / dt"),
    "dtB_dropped": ("dtB[a] = (Bn[a] - Bp[a]) / dt", "dtB[a] = 0.0 * (Bn[a] - Bp[a]) / dt"),
    "dtB_K1_factor": ("Gv[a] += (((a == b) ? 1.0 : 0.0) - 0.5 * K1[2 * a + b]) * dtB[b];",
                      "Gv[a] += (((a == b) ? 1.0 : 0.0) - 1.0 * K1[2 * a + b]) * dtB[b];"),
    "k2_relation": ("return 8.0 * (k1 - 2.0) / (3.0 * (k1 - 4.0));",
                    "return 8.0 * (k1 - 2.0) / (3.0 * (k1 - 3.0));"),
    "second_order_trace_sign": ("second += (ci[a] * ci[b] - ((a == b) ? cs2 : 0.0)) * HM2[a][b];",
                                "second += (ci[a] * ci[b] + ((a == b) ? cs2 : 0.0)) * HM2[a][b];"),
    "feq_convective_factor": ("feq[i] = weight(i) * (phi + cB / cs2 + second / (2.0 * cs2));",
                              "feq[i] = weight(i) * (phi + cB / (2.0 * cs2) + second / (2.0 * cs2));"),
    "feq_C_term_dropped": ("second += Dm * Q;", "second += 0.0 * Dm * Q;"),
    "source_prev_time": ("const double t_prev = first ? t : t - p->dt;", "const double t_prev = t;"),
    "wall_factor": ("return 2.0 * weight(i) * (phi_w", "return 1.0 * weight(i) * (phi_w"),
    "velocity_order": ("static const int EY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};",
                       "static const int EY[NQ] = {0, 0, 1, 0, -1, 1, -1, -1, 1};"),
    "K1_half": ("M[0] += 0.5;", "M[0] += 0.25;"),
    "A_offdiag": ("A[1] = s * p->A0[1];", "A[1] = -s * p->A0[1];"),
    "wall_time": ("link_target(p, ix, iy, i, t + p->dt,", "link_target(p, ix, iy, i, t,"),
    "reaction_sign": ("return p->react_rate * phi * (1.0 - phi_pow(phi, p->react_exp));",
                      "return p->react_rate * phi * (1.0 + phi_pow(phi, p->react_exp));"),
    "flux_direction": ("B[0] = p->u[0] * phi + p->b2 * p->b_dir[0] * g;",
                       "B[0] = p->u[0] * phi + p->b2 * p->b_dir[1] * g;"),
    "flux_exponent_scale": ("double g = phi_pow(phi, p->b_q) / p->b_q;", "double g = phi_pow(phi, p->b_q) / 2.0;"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/found: {old!r}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           str(mutant), "-o", str(lib), "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True)
    except subprocess.CalledProcessError:
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True)
    env = dict(os.environ, BTRT_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_burgers_fisher.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"
