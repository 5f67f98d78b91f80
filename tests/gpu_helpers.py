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


def make(csr, fmt="u16", **kw):
    """(GPU handle, oracle encoding) of a dosegen CSR in the given format.

    The oracle encodes; the library receives the stored codes, so both sides
    compute with the same decoded matrix."""
    enc = oracle.encode(csr, OFMT[fmt])
    A = dose.DoseMatrix.from_csr(enc.row_ptr, enc.col, ncols=csr.ncols, fmt=fmt, values=enc.values,
                                 scales=enc.scales, **kw)
    return A, enc


def fwd_check(d_gpu, d_ref, rtol=FWD_RTOL):
    """Per-row relative error (rows with d_ref != 0); rows with d_ref == 0 exactly 0."""
    d_gpu = np.asarray(d_gpu, dtype=np.float64)
    nz = d_ref != 0
    assert np.all(d_gpu[~nz] == 0.0), "rows with zero dose must be exactly 0"
    rel = np.abs(d_gpu[nz] - d_ref[nz]) / np.abs(d_ref[nz])
    worst = float(rel.max()) if rel.size else 0.0
    assert worst <= rtol, f"max relative error {worst:.3e} > {rtol:.1e}"
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
