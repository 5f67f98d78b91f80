"""dose_spmv_f64 (FP64 spot weights and dose; the paper's Half/double
interface) against the FP64 oracle, through the C ABI.

Tolerances, per row i with n entries, A = |a_ik x_k| summed over the row:
  double-float (default): |d - d_ref| <= (2^-45 + g(n)^2) A + 2^-53 |d| + (n + 2) 2^-53 A
  native FP64 FMA:        |d - d_ref| <= 2 (n + 2) 2^-53 A
where g(n) = n 2^-24 / (1 - n 2^-24) and the last term of each is the oracle's
own rounding (it sums in FP64 in row order).  The double-float bound takes n,
the row length, for the number of terms any one accumulator adds (a loose but
safe choice); a second check keeps the observed error of the default schedule
under 2^-40 A on every row.  Rows of zero dose are exactly 0, and unit vectors
give the stored values bit-exactly in both modes.
"""
import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import edge_case_matrices, make

pytestmark = pytest.mark.gpu

FMTS = ["f16", "u16", "bf16", "fp8", "f32"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    dose.build()
    dose.load()


@pytest.fixture(scope="module")
def tiny():
    return dosegen.generate(dosegen.TINY)


def _to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f64_check(d, enc, x, native, guard=2.0 ** -40):
    """Compare an FP64 dose with the oracle under the bounds above."""
    d = np.asarray(d, dtype=np.float64)
    ref = oracle.spmv(enc.nrows, enc.row_ptr, enc.col, enc.decoded, x)
    absref = oracle.spmv(enc.nrows, enc.row_ptr, enc.col, np.abs(enc.decoded), np.abs(x))
    n = np.diff(enc.row_ptr.astype(np.int64)).astype(np.float64)
    u = 2.0 ** -53
    if native:
        bound = 2 * (n + 2) * u * absref
    else:
        g = n * 2.0 ** -24 / (1 - n * 2.0 ** -24)
        bound = (2.0 ** -45 + g * g) * absref + u * np.abs(d) + (n + 2) * u * absref
    err = np.abs(d - ref)
    zero = absref == 0
    assert np.all(d[zero] == 0.0), "rows with no contribution must be exactly 0"
    assert np.all(err <= bound), f"worst error {float(np.max(err / np.maximum(bound, 1e-300))):.3f} x the bound"
    nz = ~zero
    if nz.any():
        worst = float(np.max(err[nz] / absref[nz]))
        assert worst <= guard, f"observed error {worst:.3e} of sum |a x| above {guard:.1e}"
        return worst
    return 0.0


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("native", [False, True])
@pytest.mark.parametrize("index16", [False, True])
@pytest.mark.parametrize("layout", [2, 1])
def test_spmv_f64_tiny_beam(tiny, fmt, native, index16, layout):
    """Row groups (fwd_layout 2) and CSR (1, also the default form of dose_spmv_f64)."""
    A, enc = make(tiny, fmt, index16=index16, tuning=dict(fwd_layout=layout))
    assert A.info()["spmv_layout"] == layout
    x = dosegen.spot_weights_f64(tiny.ncols, 21)
    d = A.spmv_f64(_to(x), native=native).cpu().numpy()
    f64_check(d, enc, x, native)
    d2 = A.spmv_f64(_to(x), native=native).cpu().numpy()
    assert np.array_equal(d.view(np.uint64), d2.view(np.uint64)), "not bitwise repeatable"
    A.device_status()


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("native", [False, True])
@pytest.mark.parametrize("layout", [2, 1])
def test_spmv_f64_unit_vectors_give_stored_values_exactly(tiny, fmt, native, layout):
    A, enc = make(tiny, fmt, tuning=dict(fwd_layout=layout))
    rng = np.random.default_rng(2)
    rows_of = np.repeat(np.arange(tiny.nrows), np.diff(enc.row_ptr.astype(np.int64)))
    for j in rng.choice(tiny.ncols, 8, replace=False):
        e = np.zeros(tiny.ncols)
        e[j] = 1.0
        d = A.spmv_f64(_to(e), native=native).cpu().numpy()
        expect = np.zeros(tiny.nrows)
        sel = enc.col == j
        expect[rows_of[sel]] = enc.decoded[sel]   # s * q, s_r * e4m3(q) and half values are exact in FP64
        assert np.array_equal(d, expect), (fmt, j)


@pytest.mark.parametrize("native", [False, True])
@pytest.mark.parametrize("layout", [2, 1])
def test_spmv_f64_signed_weights_across_magnitudes(tiny, native, layout):
    """x of both signs over 2^-30 .. 2^30 (cancellation inside rows)."""
    A, enc = make(tiny, "f16", tuning=dict(fwd_layout=layout))
    rng = np.random.default_rng(3)
    x = (dosegen.spot_weights_f64(tiny.ncols, 22) - 0.5) * np.exp2(rng.integers(-30, 31, tiny.ncols))
    d = A.spmv_f64(_to(x), native=native).cpu().numpy()
    f64_check(d, enc, x, native)


@pytest.mark.parametrize("name", list(edge_case_matrices().keys()))
@pytest.mark.parametrize("native", [False, True])
def test_spmv_f64_edge_cases(name, native):
    """Empty and one-entry matrices, rows at every lane-bin and chunk boundary,
    a 16000-entry row, 20000 columns (x read from global memory under the
    default tiles, from shared memory under the small ones)."""
    csr = edge_case_matrices()[name]
    for fmt in ("f16", "fp8"):
        # the default form (row groups where the matrix takes them) and the CSR
        # form under two schedules
        for tuning in (None, dict(tile_nnz=256, tile_rows=32, coop_nnz=64, stages=2, consumer_warps=4, fwd_layout=1),
                       dict(tile_nnz=8192, tile_rows=4096, coop_nnz=8192, stages=2, consumer_warps=16, row_order=1,
                            fwd_layout=1)):
            for index16 in (False, True):
                if index16 and csr.ncols > 65536:
                    continue
                A, enc = make(csr, fmt, tuning=tuning, index16=index16)
                x = dosegen.spot_weights_f64(csr.ncols, 23)
                f64_check(A.spmv_f64(_to(x), native=native).cpu().numpy(), enc, x, native)
                A.device_status()


def test_spmv_f64_many_columns_global_x():
    """60000 spots (the liver beams' size, Table I): x does not fit in shared
    memory beside the default ring and is read from the L2-resident copy."""
    lens = np.random.default_rng(7).integers(0, 300, 4000)
    csr = dosegen.random_csr(4000, 60000, seed=9, lengths=lens)
    for native in (False, True):
        A, enc = make(csr, "f16", index16=True)
        x = dosegen.spot_weights_f64(csr.ncols, 24)
        f64_check(A.spmv_f64(_to(x), native=native).cpu().numpy(), enc, x, native)
        A.device_status()


def test_spmv_f64_byte_model_is_the_papers(tiny):
    """F16 values, 32-bit indices, FP64 vectors: 6 nnz + 12 nr + 8 nc (+4 for
    row_ptr's extra entry), the traffic model of Sec. V."""
    A, enc = make(tiny, "f16")
    inf = A.info()
    assert inf["spmv_f64_bytes"] == 6 * tiny.nnz + 12 * tiny.nrows + 8 * tiny.ncols + 4
    A16, _ = make(tiny, "f16", index16=True)
    assert A16.info()["spmv_f64_bytes"] == inf["spmv_f64_bytes"] - 2 * tiny.nnz


def test_spmv_f64_rejects_bad_arguments(tiny):
    A, _ = make(tiny, "f16")
    x = torch.zeros(tiny.ncols, dtype=torch.float64, device="cuda")
    d = torch.zeros(tiny.nrows + 1, dtype=torch.float64, device="cuda")
    lib = dose.load()
    st = lib.dose_spmv_f64(A._h, x.data_ptr(), d.data_ptr() + 4, 0, None)   # d not 8-byte aligned (host check)
    assert st == 1
    st = lib.dose_spmv_f64(A._h, x.data_ptr(), d.data_ptr(), 0x10, None)    # unknown flag
    assert st == 1
    A.device_status()
