"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a swapped operand, a wrong sign, a dropped term, a
wrong index order) in a private copy of the oracle source, builds it with gcc,
and runs the pin suite against that build.  The suite has to fail every time.
All of this runs on the CPU; the oracle in the repository is untouched.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dfacto_oracle.c")

MUTATIONS = {
    "mttkrp_factor_swap": ("out[io * R + r] += x * F[in][ii * R + r] * F[f][iff * R + r];",
                           "out[io * R + r] += x * F[in][ii * R + r] * F[in][ii * R + r];"),
    "mode_axes_swapped": ("static int ax_in(int mode) { return (mode + 1) % 3; }",
                          "static int ax_in(int mode) { return (mode + 2) % 3; }\n"
                          "static int ax_f_unused(int mode) { return (mode + 1) % 3; }"),
    "csr_order_f_before_o": ("  if (x->o != y->o) return x->o < y->o ? -1 : 1;\n"
                             "  if (x->f != y->f) return x->f < y->f ? -1 : 1;",
                             "  if (x->f != y->f) return x->f < y->f ? -1 : 1;\n"
                             "  if (x->o != y->o) return x->o < y->o ? -1 : 1;"),
    "gradient_sign_plus_N": ("Gout[mode][i * R + r] = -Gout[mode][i * R + r] + s;",
                             "Gout[mode][i * R + r] = Gout[mode][i * R + r] + s;"),
    "ridge_term_dropped": ("for (int r = 0; r < R; ++r) Gf[r * R + r] += lambda_reg;",
                           "(void)lambda_reg;"),
    "fit_cross_term_halved": ("double res2 = nx2 - 2.0 * ip + nm2;",
                              "double res2 = nx2 - ip + nm2;"),
    "gram_hadamard_uses_one_gram": ("Gf[r * R + s] *= Gi[r * R + s];",
                                    "Gf[r * R + s] *= Gf[r * R + s];"),
    "armijo_ignores_previous_step": (
        "lambda_reg, A, B, C);\n  double alpha = (*alpha_io > 0.0) ? fmin(2.0 * (*alpha_io), 1.0) : 1.0;",
        "lambda_reg, A, B, C);\n  double alpha = 1.0;"),
    "backtracking_factor_wrong": ("    alpha *= 0.5;\n  }\n  if (g2_out) *g2_out = g2;\n  int st",
                                  "    alpha *= 0.25;\n  }\n  if (g2_out) *g2_out = g2;\n  int st"),
    "gd_update_sign": ("T[m][t] = F[m][t] - alpha * G[m][t];\n    fa = orc_loss(",
                       "T[m][t] = F[m][t] + alpha * G[m][t];\n    fa = orc_loss("),
    "joint_armijo_ignores_previous_step": (
        "lambda, A, B, C);\n  double alpha = (*alpha_io > 0.0) ? fmin(2.0 * (*alpha_io), 1.0) : 1.0;",
        "lambda, A, B, C);\n  double alpha = 1.0;"),
    "joint_update_sign": ("T[m][t] = F[m][t] - alpha * G[m][t];\n    fa = orc_joint_loss(",
                          "T[m][t] = F[m][t] + alpha * G[m][t];\n    fa = orc_joint_loss("),
    "normalisation_inverted": ("for (int64_t i = 0; i < n; ++i) F[o][i * R + r] /= s;",
                               "for (int64_t i = 0; i < n; ++i) F[o][i * R + r] *= s;"),
    "backsubstitution_transposed": ("for (int k = r + 1; k < R; ++k) s -= L[k * R + r] * X[i * R + k];",
                                    "for (int k = r + 1; k < R; ++k) s -= L[r * R + k] * X[i * R + k];"),
    "jacobi_rotation_sign": ("double c = 1.0 / sqrt(t * t + 1.0), s = t * c;",
                             "double c = 1.0 / sqrt(t * t + 1.0), s = -t * c;"),
    "ray_step_sign": ("const double u0 = F[n][row * R + r], u1 = -G[n][row * R + r];",
                      "const double u0 = F[n][row * R + r], u1 = G[n][row * R + r];"),
    "ray_gram_cross_term_halved": ("M[n][R * R + r * R + s] -= fr * gs + gr * fs;",
                                   "M[n][R * R + r * R + s] -= fr * gs;"),
    "ray_ridge_slope_dropped": ("        coef[1] -= lambda_reg * F[n][t] * G[n][t];\n", "\n"),
    "joint_row_gram_dropped": ("      for (int s = 0; s < R; ++s) H[r * R + s] += other[o * R + r] * other[o * R + s];",
                               "      (void)0;"),
    "joint_rating_side_swapped": ("    const int64_t o = yidx[(int64_t)(1 - side) * nnzY + t];",
                                  "    const int64_t o = yidx[(int64_t)side * nnzY + t];"),
    "joint_tensor_term_unweighted": ("    rhs[r] = mu * N[row * R + r];", "    rhs[r] = N[row * R + r];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(lib),
                           str(mutated), "-lm"])
    env = dict(os.environ, DFACTO_ORACLE_LIB=str(lib))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, "pins did not catch mutation %s:\n%s" % (name, res.stdout[-2000:])
