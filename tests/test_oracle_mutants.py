"""Plant plausible mistakes in a copy of the oracle and check that a pin catches each.

Every mutant is a one-token change to oracle/pip_oracle.c (a sign, an index, a
constant, a dropped term, a boundary convention).  The copy is compiled into
a temporary directory, and tests/test_oracle_pins.py runs against it in a
child process; the mutant must make at least one pin fail.  Nothing here
touches a GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pip_oracle.c")

MUTANTS = {
    "eq8_sign_of_c_term": ("double e1 = -2.0 * c * a;", "double e1 = 2.0 * c * a;"),
    "eq8_weight_sign": ("w12 = -2.0 * a * b;", "w12 = 2.0 * a * b;"),
    "eq8_transposed_weight": ("double d2 = w21 * g0x + w22 * g0y;",
                              "double d2 = w22 * g0x + w21 * g0y;"),
    "eq4_constant": ("*cx = sx / (6.0 * a);", "*cx = sx / (3.0 * a);"),
    "alg3_rolled_index": ("sx += (x[k] + x[km]) * Ak;", "sx += (x[k] + x[k]) * Ak;"),
    "alg4_line_b_sign": ("double b = x[km] - x[k];\n        double c = -(a * x[k] + b * y[k]);\n        double w11",
                         "double b = x[k] - x[km];\n        double c = -(a * x[k] + b * y[k]);\n        double w11"),
    "orient_dropped_term": ("    len = grow_product(e, len, +1.0, ay, cx);\n    return expansion_sign(e, len);",
                            "    return expansion_sign(e, len);"),
    "inside_open_boundary": ("        if (s == -sigma) return 0;\n    }\n    return 1;\n}\n\n/* exact integer",
                             "        if (s != sigma) return 0;\n    }\n    return 1;\n}\n\n/* exact integer"),
    "inside_int_open_boundary": ("        int s = (cr > 0) - (cr < 0);\n        if (s == -sigma) return 0;",
                                 "        int s = (cr > 0) - (cr < 0);\n        if (s != sigma) return 0;"),
    "alg5_reversed_comparison": ("if (!(M0 <= Mk)) in = 0;", "if (!(Mk <= M0)) in = 0;"),
    "alg1_even_is_inside": ("isin[i] = (uint8_t)((crossings % 2) == 1);",
                            "isin[i] = (uint8_t)((crossings % 2) == 0);"),
    "alg2_rolled_index": ("double rhs = y[km] * dvx - x[km] * dvy;\n            sumD",
                          "double rhs = y[k] * dvx - x[km] * dvy;\n            sumD"),
    "winding_check_loosened": ("if (changes > 2) return ORC_NONCONVEX;",
                               "if (changes > 4) return ORC_NONCONVEX;"),
    "margin_sign": ("double mk = (n0 - nk) / (2.0 * D);\n            if (mk > best) best = mk;",
                    "double mk = (nk - n0) / (2.0 * D);\n            if (mk > best) best = mk;"),
    "penalty_dtheta_sign": ("gth += gm * (dmx * by - dmy * bx);", "gth += gm * (dmx * by + dmy * bx);"),
    "penalty_eq8_back_index": ("grad_v[2 * k] += dLc * y[km];", "grad_v[2 * k] += dLc * y[k];"),
    "penalty_centroid_back_sign": ("double mu = -(G0x * g0x + G0y * g0y) / S;",
                                   "double mu = (G0x * g0x + G0y * g0y) / S;"),
    "penalty_sigmoid_sign": ("double gm = -sigmoid(-best / tau) / tau;",
                             "double gm = -sigmoid(best / tau) / tau;"),
    "raster_centre_two_roundings": ("= fmaf((float)c, dx, x0);", "= (float)c * dx + x0;"),
    "raster_row_spacing": ("fmaf((float)r, dy, y0);", "fmaf((float)r, dx, y0);"),
    "first_hit_takes_the_last": ("if (in) { out[i] = j; break; }", "if (in) { out[i] = j; }"),
    "ragged_drops_a_point": ("poffs[j + 1] - poffs[j], out + poffs[j]);",
                             "poffs[j + 1] - poffs[j] - 1, out + poffs[j]);"),
}


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, "mutation anchor for %s not unique" % name
    mutated = source.replace(old, new)
    csrc = tmp_path / "mutant.c"
    csrc.write_text(mutated)
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(lib), str(csrc), "-lm"])
    env = dict(os.environ, PIP_ORACLE_LIB_OVERRIDE=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutant %s survived every pin:\n%s" % (name, r.stdout[-2000:])
