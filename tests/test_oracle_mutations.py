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
