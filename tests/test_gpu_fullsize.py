"""Parity at the benchmark sizes, in the launch configuration bench.py times
(default tuning): the clinical beam (256x256x160 voxels x 4000 spots, 1.5e8
entries) for the dose, the fused objective pass and the adjoint, and the 27
scenario matrices x 16 weight vectors of the batched SpMM.  Doses are compared
on seeded samples of rows that the FP64 oracle computes one by one; the
objective and the gradient (4000 values) against the oracle over the whole
matrix."""
import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import adj_check, fwd_check, make

pytestmark = pytest.mark.gpu


def _to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sub_csr(enc, rows):
    """The listed rows of an encoded matrix as a standalone CSR (decoded values)."""
    rp = enc.row_ptr.astype(np.int64)
    lens = rp[rows + 1] - rp[rows]
    sub_rp = np.zeros(len(rows) + 1, dtype=np.uint32)
    np.cumsum(lens, out=sub_rp[1:])
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if lens.sum() else np.zeros(0, np.int64)
    return sub_rp, enc.col[idx], enc.decoded[idx]


@pytest.fixture(scope="module")
def clinical():
    beam = dosegen.CLINICAL
    csr = dosegen.generate(beam)
    A, enc = make(csr, "u16")
    p, w = dosegen.ellipsoid_target(beam, semi_axes=(30.0, 20.0, 16.0))
    x = dosegen.spot_weights(csr.ncols, dosegen.weight_seed(beam))
    return csr, A, enc, p, w, x


def _sample_rows(nrows, row_ptr, n, seed):
    """Seeded rows: half drawn among non-empty rows, half uniformly (mostly empty)."""
    rng = np.random.default_rng(seed)
    lens = np.diff(row_ptr.astype(np.int64))
    ne = np.nonzero(lens > 0)[0]
    rows = np.concatenate([rng.choice(ne, n // 2, replace=False), rng.choice(nrows, n // 2, replace=False)])
    return np.unique(rows)


def test_clinical_dose_sampled_rows(clinical):
    csr, A, enc, p, w, x = clinical
    d = A.spmv(_to(x)).cpu().numpy()
    rows = _sample_rows(csr.nrows, enc.row_ptr, 6000, 1)
    ref = oracle.spmv_rows(rows, enc.row_ptr, enc.col, enc.decoded, x)
    fwd_check(d[rows], ref)
    # every empty row is exactly 0
    empty = np.diff(enc.row_ptr.astype(np.int64)) == 0
    assert np.all(d[empty] == 0.0)


@pytest.mark.parametrize("fmt", ["bf16", "fp8", "f16", "f32"])
def test_clinical_dose_every_stored_format_sampled_rows(clinical, fmt):
    """The other stored formats at the clinical size (bench.py --workload
    precision): the dose of the same decoded matrix on sampled rows, with
    compensated rows and with 16-bit column indices too."""
    csr, _, _, _, _, x = clinical
    enc = oracle.encode(csr, oracle.U16_SCALE if fmt == "u16" else {
        "bf16": oracle.BF16, "fp8": oracle.FP8E4M3_ROWSCALE, "f16": oracle.F16, "f32": oracle.F32}[fmt])
    rows = _sample_rows(csr.nrows, enc.row_ptr, 4000, 5)
    ref = oracle.spmv_rows(rows, enc.row_ptr, enc.col, enc.decoded, x)
    empty = np.diff(enc.row_ptr.astype(np.int64)) == 0
    for kw in (dict(), dict(compensated=True), dict(index16=True)):
        A = dose.DoseMatrix.from_csr(enc.row_ptr, enc.col, ncols=csr.ncols, fmt=fmt, values=enc.values,
                                     scales=enc.scales, **kw)
        d = A.spmv(_to(x)).cpu().numpy()
        fwd_check(d[rows], ref)
        assert np.all(d[empty] == 0.0)
        A.device_status()
        A.close()


def test_clinical_fused_objective_and_gradient(clinical):
    csr, A, enc, p, w, x = clinical
    f, g, d = A.fwd_adj_quadratic(_to(x), _to(p), _to(w), want_d=True)
    f, g, d = float(f.item()), g.cpu().numpy(), d.cpu().numpy()
    rows = _sample_rows(csr.nrows, enc.row_ptr, 6000, 2)
    fwd_check(d[rows], oracle.spmv_rows(rows, enc.row_ptr, enc.col, enc.decoded, x))
    f_own, r_own = oracle.objective(d.astype(np.float64), p, w)
    assert abs(f - f_own) <= 1e-12 * f_own
    g_ref = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r_own)
    gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r_own)
    adj_check(g, g_ref, gabs)
    # the standalone adjoint of the same residual
    g2 = A.adjoint(_to(r_own.astype(np.float32))).cpu().numpy()
    adj_check(g2, g_ref, gabs)
    A.device_status()


def test_clinical_sell_dose_sampled_rows(clinical):
    """The default SELL-32-2^20 copy of the clinical beam (bench.py --workload sell)."""
    csr, _, enc, p, w, x = clinical
    A = dose.DoseMatrix.from_csr(enc.row_ptr, enc.col, ncols=csr.ncols, fmt="u16", values=enc.values,
                                 scales=enc.scales, sell=True)
    d = A.spmv(_to(x)).cpu().numpy()
    rows = _sample_rows(csr.nrows, enc.row_ptr, 6000, 4)
    fwd_check(d[rows], oracle.spmv_rows(rows, enc.row_ptr, enc.col, enc.decoded, x))
    assert np.all(d[np.diff(enc.row_ptr.astype(np.int64)) == 0] == 0)
    A.device_status()
    A.close()


@pytest.mark.parametrize("native", [False, True])
def test_clinical_half_double_sampled_rows(native):
    """The paper's Half/double configuration at the clinical size: F16 values,
    16-bit column indices, FP64 spot weights and dose (bench.py --workload
    halfdouble), sampled rows against the oracle under the bounds of the FP64
    parity tests."""
    beam = dosegen.CLINICAL
    csr = dosegen.generate(beam)
    A, enc = make(csr, "f16", index16=True)
    x = dosegen.spot_weights_f64(csr.ncols, dosegen.weight_seed(beam))
    d = A.spmv_f64(_to(x), native=native).cpu().numpy()
    rows = _sample_rows(csr.nrows, enc.row_ptr, 6000, 3)
    ref = oracle.spmv_rows(rows, enc.row_ptr, enc.col, enc.decoded, x)
    absref = oracle.spmv_rows(rows, enc.row_ptr, enc.col, np.abs(enc.decoded), np.abs(x))
    n = np.diff(enc.row_ptr.astype(np.int64))[rows].astype(np.float64)
    u = 2.0 ** -53
    if native:
        bound = 2 * (n + 2) * u * absref
    else:
        g = n * 2.0 ** -24 / (1 - n * 2.0 ** -24)
        bound = (2.0 ** -45 + g * g) * absref + u * np.abs(d[rows]) + (n + 2) * u * absref
    err = np.abs(d[rows] - ref)
    assert np.all(err <= bound)
    nz = absref > 0
    assert np.all(d[rows][~nz] == 0.0)
    assert np.max(err[nz] / absref[nz]) <= 2.0 ** -40
    assert np.all(d[np.diff(enc.row_ptr.astype(np.int64)) == 0] == 0.0)
    A.device_status()


def test_batched_27_scenarios_16_vectors_sampled_rows():
    """All 27 scenario matrices in one launch (bench.py --workload batched),
    64 sampled rows x 16 vectors per matrix against the oracle."""
    nvec = 16
    handles, Xs, checks = [], [], []
    for i, beam in enumerate(dosegen.batched_beams()):
        csr = dosegen.generate(beam)
        A, enc = make(csr, "u16")
        X = dosegen.spot_weights(csr.ncols, 300 + i, nvec=nvec).reshape(csr.ncols, nvec)
        rows = _sample_rows(csr.nrows, enc.row_ptr, 64, 10 + i)
        sub_rp, sub_col, sub_a = _sub_csr(enc, rows)
        ref = oracle.spmm(len(rows), sub_rp, sub_col, sub_a, X.astype(np.float64))
        handles.append(A)
        Xs.append(_to(X))
        checks.append((rows, ref))
        del csr, enc
    Ds = dose.spmv_batched(handles, Xs)
    for D, (rows, ref) in zip(Ds, checks):
        fwd_check(D[torch.from_numpy(rows).cuda()].cpu().numpy().reshape(-1), ref.reshape(-1))
    for A in handles:
        A.device_status()


def test_liver1_shaped_dose_sampled_rows():
    """The paper's own matrix shape (Table I, liver beam 1: 2.97e6 x 6.8e4,
    1.48e9 entries; bench.py --workload liver1): x does not fit in shared memory,
    so the forward kernels stage column windows (FP32) or read x from L2
    (Half/double).  FP32 dose and the Half/double dose on sampled rows against
    the oracle."""
    beam = dosegen.LIVER1_SHAPED
    csr = dosegen.generate(beam)
    rp = csr.row_ptr.astype(np.int64)
    rows = _sample_rows(csr.nrows, csr.row_ptr, 2000, 5)
    lens = rp[rows + 1] - rp[rows]
    sub_rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=sub_rp[1:])
    take = np.repeat(rp[rows] - sub_rp[:-1], lens) + np.arange(int(sub_rp[-1]))
    sub = dosegen.CSR(len(rows), csr.ncols, sub_rp.astype(np.uint32), csr.col[take], csr.val[take])
    A = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="f16", values_f64=csr.val)
    nrows, ncols = csr.nrows, csr.ncols
    empty = np.nonzero(np.diff(rp) == 0)[0]
    del csr, take
    assert 0 < A.info()["fwd_window"] < ncols
    enc = oracle.encode(sub, oracle.F16)   # elementwise: the same codes the library stores
    x = dosegen.spot_weights(ncols, dosegen.weight_seed(beam))
    d = A.spmv(_to(x)).cpu().numpy()
    fwd_check(d[rows], oracle.spmv(len(rows), enc.row_ptr, enc.col, enc.decoded, x))
    assert np.all(d[empty] == 0)
    x64 = dosegen.spot_weights_f64(ncols, dosegen.weight_seed(beam))
    d64 = A.spmv_f64(_to(x64)).cpu().numpy()[rows]
    ref = oracle.spmv(len(rows), enc.row_ptr, enc.col, enc.decoded, x64)
    absref = oracle.spmv(len(rows), enc.row_ptr, enc.col, np.abs(enc.decoded), x64)
    nz = absref > 0
    assert np.all(d64[~nz] == 0) and np.max(np.abs(d64[nz] - ref[nz]) / absref[nz]) <= 2.0 ** -40
    A.device_status()
    A.close()
