"""Plants plausible mistakes in the oracle (on the CPU) and checks the pins catch each one.

Each mutant is a copy of oracle/pk_oracle.c with one edit (a flipped sign, a swapped
operand, an off-by-one index, a dropped factor), compiled with gcc into a temporary
library; the pin suite then runs against it in a subprocess and must fail.
"""
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
SRC = (ROOT / "oracle" / "pk_oracle.c").read_text()

MUTANTS = {
    "cg_pipelined_beta_sign": ("alpha * alpha * apap / rr - 1.0", "alpha * alpha * apap / rr + 1.0"),
    "cg_residual_sign": ("r[k] -= alpha * ap[k]", "r[k] += alpha * ap[k]"),
    "cg_classical_beta_inverted": ("double beta = rr_new / rr;", "double beta = rr / rr_new;"),
    "cg_pipelined_pap_operand": ("pap = orc_dot(n, p, ap);                      /* <p_i, Ap_i> */",
                                 "pap = orc_dot(n, ap, ap);                     /* <p_i, Ap_i> */"),
    "bicgstab_pipelined_beta_sign": ("double beta = -asr0s / apr0s;", "double beta = asr0s / apr0s;"),
    "bicgstab_p_update_sign": ("beta * (p[k] - omega * ap[k])", "beta * (p[k] + omega * ap[k])"),
    "bicgstab_omega_inverted": ("double omega = ass / asas;", "double omega = asas / ass;"),
    "bicgstab_x_drops_omega_s": ("x[k] += alpha * p[k] + omega * s[k];", "x[k] += alpha * p[k];"),
    "gmres_xi_wrong_vector": ("xii = orc_dot(n, VEC(0), vi);", "xii = orc_dot(n, VEC(1), vi);"),
    "gmres_backsub_multiplies": ("eta[i] = s / RR(i, i);", "eta[i] = s * RR(i, i);"),
    "gmres_cgs_includes_v0": [("for (int32_t j = 1; j <= i - 1; ++j) RR(j, i) = orc_dot",
                               "for (int32_t j = 0; j <= i - 1; ++j) RR(j, i) = orc_dot"),
                              ("for (int32_t j = 1; j <= i - 1; ++j) {\n        double rji",
                               "for (int32_t j = 0; j <= i - 1; ++j) {\n        double rji")],
    "gmres_update_index_shift": ("a += eta[i] * VEC(i - 1)[k];", "a += eta[i] * VEC(i)[k];"),
    "gmres_update_drops_rho0": ("x[k] += rho0 * a;", "x[k] += a;"),
    "spmv_transposed_gather": ("s += va[j] * x[ci[j]];", "s += va[j] * x[i];"),
}

# mutants of the preconditioned solvers and of CGS2, checked against their own pin files
EXTRA_MUTANTS = {
    "pcg_beta_sign": ([("beta = alpha * alpha * qdq / gamma - 1.0;", "beta = alpha * alpha * qdq / gamma + 1.0;")],
                      "test_oracle_pcg.py"),
    "pcg_qdq_unpreconditioned": ([("z[k] = ap[k] * dinv[k];", "z[k] = ap[k];")], "test_oracle_pcg.py"),
    "pcg_p_update_unpreconditioned": ([("p[k] = r[k] * dinv[k] + beta * p[k];", "p[k] = r[k] + beta * p[k];")],
                                      "test_oracle_pcg.py"),
    "jacobi_right_scales_rows": ([("va_out[j] = va[j] * dinv_out[ci[j]];", "va_out[j] = va[j] * dinv_out[i];")],
                                 "test_oracle_jacobi_right.py"),
    "jacobi_right_y0_unscaled": ([("x[i] = x[i] * d;", "x[i] = x[i];")], "test_oracle_jacobi_right.py"),
    "jacobi_right_end_skipped": ([("x[i] = dinv[i] * x[i];", "x[i] = x[i];")], "test_oracle_jacobi_right.py"),
    # (the second pass's coefficients are O(eps ||A v_{i-1}||): leaving them out of R is not
    # observable above rounding, so that edit is not a mutant; the second pass acts through v_i)
    "cgs2_second_pass_not_subtracted": ([("for (int32_t k = 0; k < n; ++k) vi[k] -= c2[j] * vj[k];", "")],
                                        "test_oracle_cgs2.py"),
    "cgs2_second_pass_sign": ([("for (int32_t k = 0; k < n; ++k) vi[k] -= c2[j] * vj[k];",
                                "for (int32_t k = 0; k < n; ++k) vi[k] += c2[j] * vj[k];")], "test_oracle_cgs2.py"),
    # the three-kernel GMRES: the shift's sign in the identity's last coefficient, the norm
    # identity without the projections, the shift left out of w (but kept in the
    # coefficient), and the shift rule taking <v_{i-1}, w> instead of the Rayleigh quotient
    # (exact arithmetic does not see the shift's value, so this one is caught by the
    # closed-form check of the first shifts)
    "shift3_coefficient_sign": ([("double c = j == i - 1 ? RR(j, i) - sigma : RR(j, i);",
                                  "double c = j == i - 1 ? RR(j, i) + sigma : RR(j, i);")], "test_oracle_shift3.py"),
    "shift3_norm_without_projections": ([("double rii2 = nu - sum2;", "double rii2 = nu;")], "test_oracle_shift3.py"),
    "shift3_w_not_shifted": ([("acc[k] = vi[k] - sigma * vp[k];", "acc[k] = vi[k];")], "test_oracle_shift3.py"),
    "shift3_rule_uses_w": ([("double rq = orc_dot(n, vp, vi);", "double rq = orc_dot(n, vp, acc);")],
                           "test_oracle_shift3.py"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS) + sorted(EXTRA_MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    if name in MUTANTS:
        edits, pins = MUTANTS[name], "test_oracle_pins.py"
    else:
        edits, pins = EXTRA_MUTANTS[name]
    edits = edits if isinstance(edits, list) else [edits]
    text = SRC
    for old, new in edits:
        assert old in text, f"mutation site vanished: {name}"
        text = text.replace(old, new)
    src = tmp_path / "mutant.c"
    src.write_text(text)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o",
                    str(so), str(src), "-lm"], check=True)
    env = dict(os.environ, PK_ORACLE_LIB=str(so))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          str(ROOT / "tests" / pins)],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode != 0, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"
