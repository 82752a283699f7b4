"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a shifted index,
a swapped operand) in a copy of the oracle's C source (at the first occurrence
of its anchor, i.e. in the forward definition when the adjoint repeats a
line), builds it on the CPU,
and runs the pin suites against it in a subprocess: at least one pin must
fail.  The unmodified source must pass the same suites.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gtb_oracle.c")
PINS = ["tests/test_oracle_hdiff.py", "tests/test_oracle_vadv.py", "tests/test_oracle_adjoint.py"]

MUTATIONS = {
    "lap_sign": ("LAP(i, j) = 4.0 * AT(in, i, j, k) - s;", "LAP(i, j) = s - 4.0 * AT(in, i, j, k);"),
    "lap_drop_term": ("s = s + AT(in, i, j - 1, k);", ";"),
    "limiter_nonstrict": ("if (f * g > 0.0) f = 0.0;\n                FX", "if (f * g >= 0.0) f = 0.0;\n                FX"),
    "limiter_gradient_sign": ("double g = AT(in, i + 1, j, k) - AT(in, i, j, k);",
                              "double g = AT(in, i, j, k) - AT(in, i + 1, j, k);"),
    "flux_index": ("double f = LAP(i + 1, j) - LAP(i, j);", "double f = LAP(i, j) - LAP(i - 1, j);"),
    "drop_fy": ("double div = (FX(i, j) - FX(i - 1, j)) + (FY(i, j) - FY(i, j - 1));",
                "double div = (FX(i, j) - FX(i - 1, j));"),
    "update_sign": ("AT(out, i, j, k) = AT(in, i, j, k) - t;", "AT(out, i, j, k) = AT(in, i, j, k) + t;"),
    "a_sign": ("double g = -0.5 * w;", "double g = 0.5 * w;"),
    "c_face_index": ("0.5 * (AT(wcon, i, j, k + 1) + AT(wcon, i + 1, j, k + 1))",
                     "0.5 * (AT(wcon, i, j, k) + AT(wcon, i + 1, j, k))"),
    "c_face_index_literal": (": AT(wcon, i, j, k + 1);", ": AT(wcon, i, j, k);"),
    "average_partner": ("0.5 * (AT(wcon, i, j, k) + AT(wcon, i + 1, j, k))",
                        "0.5 * (AT(wcon, i, j, k) + AT(wcon, i, j, k))"),
    "b_sign": ("double bk = (dtr - ak) - ck;", "double bk = (dtr - ak) + ck;"),
    "rhs_operand": ("double dk = dtr * AT(u_pos, i, j, k)", "double dk = dtr * AT(u_stage, i, j, k)"),
    "explicit_sign": ("if (k >= 1) dk = dk - ask *", "if (k >= 1) dk = dk + ask *"),
    "pivot_sign": ("b[k] - a[k] * cp[k - 1]", "b[k] + a[k] * cp[k - 1]"),
    "backsub_sign": ("x[k] = dp[k] - cp[k] * x[k + 1];", "x[k] = dp[k] + cp[k] * x[k + 1];"),
    "output_operand": ("double r = x[k] - AT(u_pos, i, j, k);", "double r = x[k] - AT(u_stage, i, j, k);"),
    "adj_dropped_identity": ("                AT(in_bar, i, j, k) += ob;\n", "\n"),
    "adj_div_cotangent_sign": ("double q = -AT(coeff, i, j, k) * ob;", "double q = AT(coeff, i, j, k) * ob;"),
    "adj_west_flux_sign": ("if (KX(i - 1, j)) { LAPB(i, j) -= q;      LAPB(i - 1, j) += q; }",
                           "if (KX(i - 1, j)) { LAPB(i, j) += q;      LAPB(i - 1, j) -= q; }"),
    "adj_lap_neighbour_sign": ("AT(in_bar, i + 1, j, k) -= lb;", "AT(in_bar, i + 1, j, k) += lb;"),
    "adj_coeff_bar_sign": ("AT(coeff_bar, i, j, k) += -div * ob;", "AT(coeff_bar, i, j, k) += div * ob;"),
    "adj_untransposed_solve": ("double sup = (k == K - 1) ? 0.0 : a[k + 1];", "double sup = (k == K - 1) ? 0.0 : c[k];"),
    "adj_dropped_dtr": ("r[k] = dtr * AT(y_bar, i, j, k);", "r[k] = AT(y_bar, i, j, k);"),
    "adj_u_pos_direct_term": ("AT(u_pos_bar, i, j, k) = dtr * z[k] - dtr * yb;", "AT(u_pos_bar, i, j, k) = dtr * z[k];"),
    "adj_explicit_index": ("s -= as[k + 1] * z[k + 1];", "s -= as[k] * z[k + 1];"),
    "top_boundary": ("double ak = 0.0, ck = 0.0, ask = 0.0, csk = 0.0;\n        if (k >= 1) {",
                     "double ak = 0.0, ck = 0.0, ask = 0.0, csk = 0.0;\n        if (k >= 0) {"),
}


def _run_pins(env):
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))  # the first occurrence: the forward definition
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                           "-o", str(lib), str(mutated)])
    env = dict(os.environ, GTB_ORACLE_LIB=str(lib))
    r = _run_pins(env)
    assert r.returncode != 0, f"no pin caught mutation {name}:\n{r.stdout[-2000:]}"
