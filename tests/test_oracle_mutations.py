"""Plausible mistakes planted in copies of the oracle are caught by its pins.

Each mutation edits one line of dose_oracle.c (a dropped term, a wrong index,
a wrong sign, a wrong rounding rule), compiles the copy on the CPU and runs the
pin tests against it in a subprocess: every mutant must fail at least one pin.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dose_oracle.c")

MUTATIONS = {
    "spmv_drops_last_entry": (
        "        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += a[k] * x[col[k]];\n"
        "        d[i] = s;",
        "        for (uint32_t k = row_ptr[i]; k + 1 < row_ptr[i + 1]; ++k) s += a[k] * x[col[k]];\n"
        "        d[i] = s;"),
    "spmv_wrong_x_index": (
        "        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += a[k] * x[col[k]];\n"
        "        d[i] = s;",
        "        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += a[k] * x[col[k] ? col[k] - 1 : 0];\n"
        "        d[i] = s;"),
    "adjoint_transposed_operand": (
        "for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) g[col[k]] += a[k] * r[i];",
        "for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) g[i % ncols] += a[k] * r[col[k] % nrows];"),
    "objective_residual_sign": ("if (r) r[i] = 2.0 * w[i] * e;", "if (r) r[i] = -2.0 * w[i] * e;"),
    "objective_drops_weight": ("f += w[i] * e * e;", "f += e * e;"),
    "pg_no_projection": ("x[j] = t > 0.0 ? t : 0.0;", "x[j] = t;"),
    "fp8_wrong_bias": ("v = ldexp(1.0 + (double)m / 8.0, e - 7);", "v = ldexp(1.0 + (double)m / 8.0, e - 8);"),
    "fp8_ties_not_even": ("if (dd < bestd || (dd == bestd && (c & 1) == 0 && (best & 1) == 1)) {",
                          "if (dd < bestd) {"),
    "bf16_truncates": ("q = ldexp(nearbyint(ldexp(m, 8)), ex - 8);", "q = ldexp(floor(ldexp(m, 8)), ex - 8);"),
    "f16_truncates": ("q = ldexp(nearbyint(ldexp(m, 11)), ex - 11);", "q = ldexp(floor(ldexp(m, 11)), ex - 11);"),
    "f16_wrong_bias": ("v = ldexp(1.0 + (double)m / 1024.0, e - 15);", "v = ldexp(1.0 + (double)m / 1024.0, e - 14);"),
    "f16_subnormal_quantum": ("v = ldexp((double)m / 1024.0, -14);", "v = ldexp((double)m / 1024.0, -15);"),
    "robust_expected_drops_probability": ("for (uint32_t s = 0; s < S; ++s) F += prob[s] * f_s[s];",
                                          "for (uint32_t s = 0; s < S; ++s) F += f_s[s] / S;"),
    "robust_worst_takes_the_smallest": ("if (f_s[s] > f_s[best]) best = s;", "if (f_s[s] < f_s[best]) best = s;"),
    "spmm_wrong_vector_stride": ("s += a[k] * X[(uint64_t)col[k] * nvec + v];", "s += a[k] * X[(uint64_t)col[k] + v];"),
    "spmv_rows_ignores_selection": ("        uint32_t i = rows[t];", "        uint32_t i = (uint32_t)t;"),
    "abs_adjoint_keeps_sign_of_r": ("g[col[k]] += fabs(a[k]) * fabs(r[i]);", "g[col[k]] += fabs(a[k]) * r[i];"),
    "gradient_swaps_target_and_weight": ("double f = oracle_objective(nrows, d, p, w, r);",
                                         "double f = oracle_objective(nrows, d, w, p, r);"),
    "pg_ascends": ("double t = x[j] - eta * grad[j];", "double t = x[j] + eta * grad[j];"),
    "power_iteration_unnormalised": ("for (uint32_t j = 0; j < ncols; ++j) v[j] /= nv;",
                                     "for (uint32_t j = 0; j < ncols; ++j) v[j] /= 1.0;"),
    "fp8_search_skips_largest_code": ("for (int c = 0; c < 0x7F; ++c) { /* 0x7F is NaN */",
                                      "for (int c = 0; c < 0x7E; ++c) { /* 0x7F is NaN */"),
    "fp8_rowscale_wrong_divisor": ("float s = rmax > 0.0 ? (float)(rmax / 448.0) : 1.0f;",
                                   "float s = rmax > 0.0 ? (float)(rmax / 480.0) : 1.0f;"),
    "robust_expected_gradient_of_first_scenario": ("for (uint32_t s = 0; s < S; ++s) t += prob[s] * g_s[(size_t)s * ncols + j];",
                                                   "for (uint32_t s = 0; s < S; ++s) t += prob[s] * g_s[j];"),
    "u16_decode_in_fp32": ("for (uint64_t k = 0; k < nnz; ++k) a[k] = (double)scale * (double)q[k];",
                           "for (uint64_t k = 0; k < nnz; ++k) a[k] = (double)(scale * (float)q[k]);"),
    "u16_round_half_up": ("double t = nearbyint(v[k] / (double)s);", "double t = floor(v[k] / (double)s + 0.5);"),
    "u16_scale_off_by_one": ("float s = vmax > 0.0 ? (float)(vmax / 65535.0) : 1.0f;",
                             "float s = vmax > 0.0 ? (float)(vmax / 65536.0) : 1.0f;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           str(mutant), "-o", str(so), "-lm"])
    env = dict(os.environ, DOSE_ORACLE_SO=str(so))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutant {name} passed every pin:\n{res.stdout[-2000:]}"
