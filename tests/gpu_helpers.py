"""Shared helpers of the GPU parity tests: build matrices through the C ABI from
oracle-encoded CSR data, and compare GPU results with the FP64 oracle."""
import numpy as np

import dosegen
import oracle
import paper_2103_09683_gb300 as dose

OFMT = {"u16": oracle.U16_SCALE, "bf16": oracle.BF16, "fp8": oracle.FP8E4M3_ROWSCALE, "f16": oracle.F16,
        "f32": oracle.F32}

# Max relative error of an FP32-accumulated row sum of non-negative terms
# against the FP64 oracle on the same decoded matrix.
FWD_RTOL = 1e-5
U32 = 2.0 ** -24


def plain_row_bound(lens, lanes):
    """Per-row relative bound for plain FP32 accumulation of non-negative terms:
    1e-5 for rows of up to 4096 entries; a longer row of n entries summed by
    `lanes` lanes, each with four accumulators of consecutive-group terms that
    are combined pairwise and then reduced over the lanes in a tree, has at most
    ceil(n / (4 lanes)) + 2 + ceil(log2 lanes) rounding steps on any term, so
    (that count) u with u = 2^-24 (first-order bound, all terms >= 0)."""
    lens = np.asarray(lens, dtype=np.float64)
    steps = np.ceil(lens / (4.0 * lanes)) + 2 + np.ceil(np.log2(max(lanes, 1)))
    return np.where(lens <= 4096, FWD_RTOL, np.maximum(FWD_RTOL, steps * U32))


def make(csr, fmt="u16", **kw):
    """(GPU handle, oracle encoding) of a dosegen CSR in the given format.

    The oracle encodes; the library receives the stored codes, so both sides
    compute with the same decoded matrix."""
    enc = oracle.encode(csr, OFMT[fmt])
    A = dose.DoseMatrix.from_csr(enc.row_ptr, enc.col, ncols=csr.ncols, fmt=fmt, values=enc.values,
                                 scales=enc.scales, **kw)
    return A, enc


def fwd_check(d_gpu, d_ref, rtol=FWD_RTOL):
    """Per-row relative error (rows with d_ref != 0); rows with d_ref == 0 exactly 0.
    rtol: one bound for every row, or an array with each row's bound."""
    d_gpu = np.asarray(d_gpu, dtype=np.float64)
    nz = d_ref != 0
    assert np.all(d_gpu[~nz] == 0.0), "rows with zero dose must be exactly 0"
    rel = np.abs(d_gpu[nz] - d_ref[nz]) / np.abs(d_ref[nz])
    bound = np.broadcast_to(np.asarray(rtol, dtype=np.float64), d_ref.shape)[nz]
    worst = float(np.max(rel / bound)) if rel.size else 0.0
    bad = np.nonzero(rel > bound)[0]
    assert bad.size == 0, (f"{bad.size} rows over their bound; worst {worst:.3f} x the bound "
                           f"(row {np.nonzero(nz)[0][bad[0]]}, error {rel[bad[0]]:.3e})")
    return worst


def adj_check(g_gpu, g_ref, g_abs, rtol=1e-5):
    """Componentwise |g - g_ref| <= rtol * (|A|^T |r|)_j."""
    g_gpu = np.asarray(g_gpu, dtype=np.float64)
    err = np.abs(g_gpu - g_ref)
    bound = rtol * g_abs + 1e-30
    worst = float(np.max(err / bound)) if err.size else 0.0
    assert np.all(err <= bound), f"adjoint error {worst:.3f} x the bound"
    return worst


def edge_case_matrices():
    """Small matrices covering the schedule's corner cases."""
    cases = {}
    cases["one_by_one"] = dosegen.random_csr(1, 1, seed=1, lengths=[1])
    cases["empty_matrix"] = dosegen.random_csr(7, 5, seed=2, lengths=[0] * 7)
    cases["one_row"] = dosegen.random_csr(1, 300, seed=3, lengths=[257])
    # row lengths at every bin and chunk boundary, and the last column used
    lens = [0, 1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 1023, 1024, 1025,
            4095, 4096, 4097, 8193, 16000, 0, 0, 5]
    cases["boundaries"] = dosegen.random_csr(len(lens), 20000, seed=4, lengths=lens)
    lens2 = list(np.random.default_rng(5).integers(0, 40, 3000)) + [2000, 0, 1]
    cases["ragged_small_nc"] = dosegen.random_csr(len(lens2), 64, seed=6, lengths=np.minimum(lens2, 64))
    return cases


def long_row_matrices():
    """The boundary rows (compensation threshold 128/129, 4095-4097, the
    whole-CTA rows 8193 and 16000) and a band of rows of 400-8192 entries, some
    of them with values falling over four decades along the row (plain FP32
    loses the most digits there)."""
    cases = {"boundaries": edge_case_matrices()["boundaries"]}
    rng = np.random.default_rng(31)
    lens = rng.integers(400, 8193, 96)
    band = dosegen.random_csr(len(lens), 9000, seed=32, lengths=lens)
    rp = band.row_ptr.astype(np.int64)
    val = band.val.copy()
    for i in range(0, len(lens), 3):
        val[rp[i]:rp[i + 1]] = np.geomspace(1.0, 1e-4, lens[i])
    cases["band_400_8192"] = dosegen.CSR(band.nrows, band.ncols, band.row_ptr, band.col, val)
    return cases
