"""The host legs of bench.py: the all-cores oracle timing computes the same f
and A^T r as the single-thread oracle (its row blocks cover every row once)."""
import os

import numpy as np
import pytest

import bench
import dosegen
import oracle


@pytest.fixture(scope="module")
def tiny():
    b = dosegen.TINY
    csr = dosegen.generate(b)
    p, w = dosegen.ellipsoid_target(b, semi_axes=(8.0, 8.0, 4.0))
    return csr, p, w, dosegen.spot_weights(csr.ncols, 3)


@pytest.mark.parametrize("n", [1, 3, 16, 200000])
def test_row_blocks_cover_the_rows_and_sum_to_the_oracle(tiny, n):
    csr, p, w, x = tiny
    enc = oracle.encode(csr, oracle.U16_SCALE)
    blocks = bench.oracle_row_blocks(enc.row_ptr, enc.col, enc.decoded, p, w, n)
    assert len(blocks) == n
    assert sum(b[0] for b in blocks) == csr.nrows
    assert sum(int(b[1][-1]) for b in blocks) == csr.nnz
    if n <= 16:  # equal entry counts up to one row
        lens = np.diff(enc.row_ptr.astype(np.int64))
        assert max(int(b[1][-1]) for b in blocks) <= csr.nnz / n + lens.max() + 1
    f_ref, g_ref = oracle.fgrad(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, x, p, w)
    parts = [oracle.fgrad(b[0], csr.ncols, b[1], b[2], b[3], x, b[4], b[5]) for b in blocks]
    f = sum(fb for fb, _ in parts)
    g = np.sum([gb for _, gb in parts], axis=0)
    assert f == pytest.approx(f_ref, rel=1e-12)
    absg = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded,
                             oracle.objective(oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x), p, w)[1])
    assert np.all(np.abs(g - g_ref) <= 1e-12 * absg)


def test_all_cores_leg_reports_its_threads(tiny):
    csr, p, w, x = tiny
    out = bench.cpu_baseline_all_cores(csr, x, p, w, budget_s=0.2)
    assert out["cores"] == (os.cpu_count() or 1) and out["kind"] == "oracle" and out["value"] > 0


def test_fp64_dose_rows_is_the_oracles_row_sample(tiny):
    """The precision workload's exact-values dose on sampled rows (numpy) equals
    the oracle's, empty rows included."""
    csr, _, _, x = tiny
    rows = np.unique(np.random.default_rng(8).choice(csr.nrows, 700, replace=False))
    got = bench.fp64_dose_rows(csr.row_ptr, csr.col, csr.val, x, rows)
    ref = oracle.spmv_rows(rows, csr.row_ptr, csr.col, csr.val, x)
    lens = np.diff(csr.row_ptr.astype(np.int64))[rows]
    assert (lens == 0).any() and (lens > 0).any()
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)
    assert np.all(got[lens == 0] == 0.0)
