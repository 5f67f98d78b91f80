"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Forward: max relative error per row <= 1e-5 (FP32 accumulation of
non-negative terms; rows of zero dose exactly 0).  Adjoint: componentwise
|g - g_ref| <= 1e-5 (|A|^T |r|)_j.  Index work is bit-exact (unit vectors give
the stored column exactly).  Every result is bitwise repeatable.
"""
import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import adj_check, edge_case_matrices, fwd_check, long_row_matrices, make, plain_row_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    dose.build()
    dose.load()


def _x(n, seed=11):
    return dosegen.spot_weights(n, seed)


def _to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def tiny():
    return dosegen.generate(dosegen.TINY)


# ---------------------------------------------------------------- forward

@pytest.mark.parametrize("fmt", ["u16", "bf16", "fp8", "f16", "f32"])
@pytest.mark.parametrize("compensated", [False, True])
def test_forward_tiny_beam(tiny, fmt, compensated):
    A, enc = make(tiny, fmt, compensated=compensated)
    x = _x(tiny.ncols)
    d = A.spmv(_to(x)).cpu().numpy()
    ref = oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x)
    fwd_check(d, ref)
    d2 = A.spmv(_to(x)).cpu().numpy()
    assert np.array_equal(d.view(np.uint32), d2.view(np.uint32)), "not bitwise repeatable"
    A.device_status()


@pytest.mark.parametrize("name", list(edge_case_matrices().keys()))
@pytest.mark.parametrize("fmt", ["u16", "fp8"])
def test_forward_edge_cases(name, fmt):
    csr = edge_case_matrices()[name]
    for tuning in (None, dict(tile_nnz=256, tile_rows=32, coop_nnz=64, stages=2, consumer_warps=4),
                   dict(tile_nnz=8192, tile_rows=4096, coop_nnz=8192, stages=2, consumer_warps=16, row_order=1)):
        A, enc = make(csr, fmt, tuning=tuning)
        x = _x(csr.ncols, seed=3)
        d = A.spmv(_to(x)).cpu().numpy()
        ref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x)
        # 1e-5 on rows of up to 4096 entries; a longer row is summed by at least
        # 8 lanes in these schedules, and plain FP32 is held to that bound
        fwd_check(d, ref, rtol=plain_row_bound(csr.row_lengths(), lanes=8))
        A.device_status()


@pytest.mark.parametrize("fmt", ["u16", "bf16", "fp8", "f16", "f32"])
@pytest.mark.parametrize("compensated", [False, True])
def test_forward_16bit_column_indices(tiny, fmt, compensated):
    """DOSE_CREATE_U16_INDEX: dose_spmv reads 16-bit column indices; results
    equal the 32-bit path bitwise (same schedule, same order), the byte model
    counts 2-byte indices, and the other kernels keep working on the handle."""
    A32, enc = make(tiny, fmt, compensated=compensated)
    A16, _ = make(tiny, fmt, compensated=compensated, index16=True)
    x = _x(tiny.ncols)
    d16 = A16.spmv(_to(x)).cpu().numpy()
    fwd_check(d16, oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x))
    assert np.array_equal(d16.view(np.uint32), A32.spmv(_to(x)).cpu().numpy().view(np.uint32))
    i16, i32 = A16.info(), A32.info()
    assert i32["spmv_bytes"] - i16["spmv_bytes"] == 2 * tiny.nnz
    r = np.random.default_rng(4).normal(size=tiny.nrows).astype(np.float32)
    assert np.array_equal(A16.adjoint(_to(r)).cpu().numpy(), A32.adjoint(_to(r)).cpu().numpy())
    A16.device_status()


@pytest.mark.parametrize("name", list(edge_case_matrices().keys()))
def test_forward_16bit_column_indices_edge_cases(name):
    csr = edge_case_matrices()[name]
    for tuning in (None, dict(tile_nnz=256, tile_rows=32, coop_nnz=64, stages=2, consumer_warps=4),
                   dict(tile_nnz=8192, tile_rows=4096, coop_nnz=8192, stages=2, consumer_warps=16, row_order=1)):
        A, enc = make(csr, "u16", tuning=tuning, index16=True)
        x = _x(csr.ncols, seed=5)
        fwd_check(A.spmv(_to(x)).cpu().numpy(), oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x))
        A.device_status()


@pytest.mark.parametrize("fmt", ["u16", "fp8", "bf16", "f16", "f32"])
def test_unit_vectors_reproduce_stored_columns_bit_exact(tiny, fmt):
    A, enc = make(tiny, fmt)
    rng = np.random.default_rng(0)
    M_cols = {}
    rp = enc.row_ptr.astype(np.int64)
    rows_of = np.repeat(np.arange(tiny.nrows), np.diff(rp))
    for j in rng.choice(tiny.ncols, 12, replace=False):
        e = np.zeros(tiny.ncols, dtype=np.float32)
        e[j] = 1.0
        d = A.spmv(_to(e)).cpu().numpy()
        sel = enc.col == j
        expect = np.zeros(tiny.nrows, dtype=np.float32)
        # the stored value rounded once to FP32: fl32(s*q) (u16), fl32(s_r*e4m3) (fp8)
        expect[rows_of[sel]] = enc.decoded[sel].astype(np.float32)
        assert np.array_equal(d.view(np.uint32), expect.view(np.uint32)), j


@pytest.mark.parametrize("fmt", ["u16", "bf16", "fp8", "f16", "f32"])
@pytest.mark.parametrize("sigma", [1, 32, 1024, 1 << 20])
@pytest.mark.parametrize("index16", [False, True])
def test_forward_sell_storage(tiny, fmt, sigma, index16):
    """DOSE_CREATE_SELL: dose_spmv on the SELL-32-sigma copy (one row per lane)
    against the oracle; padding counted in sell_entries; bitwise repeatable;
    unit vectors give the stored values bit-exactly."""
    A, enc = make(tiny, fmt, sell=True, index16=index16, tuning=dict(sell_sigma=sigma))
    x = _x(tiny.ncols)
    d = A.spmv(_to(x)).cpu().numpy()
    fwd_check(d, oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x))
    assert np.array_equal(d.view(np.uint32), A.spmv(_to(x)).cpu().numpy().view(np.uint32))
    # padding: every chunk of 32 consecutive rows (after sorting inside windows of
    # sigma rows) is padded to its longest row, rounded up to 4
    lens = np.diff(enc.row_ptr.astype(np.int64))
    order = np.concatenate([w[np.argsort(-lens[w], kind="stable")] for w in
                            np.array_split(np.arange(tiny.nrows), np.arange(sigma, tiny.nrows, sigma))]) \
        if sigma > 1 else np.arange(tiny.nrows)
    chunks = [lens[order[c:c + 32]].max() for c in range(0, tiny.nrows, 32)]
    assert A.info()["sell_entries"] == sum(128 * ((m + 3) // 4) for m in chunks)
    rows_of = np.repeat(np.arange(tiny.nrows), lens)
    for j in np.random.default_rng(1).choice(tiny.ncols, 4, replace=False):
        e = np.zeros(tiny.ncols, dtype=np.float32)
        e[j] = 1.0
        expect = np.zeros(tiny.nrows, dtype=np.float32)
        sel = enc.col == j
        expect[rows_of[sel]] = enc.decoded[sel].astype(np.float32)
        assert np.array_equal(A.spmv(_to(e)).cpu().numpy().view(np.uint32), expect.view(np.uint32))
    # the other calls still use the CSR arrays
    r = np.random.default_rng(4).normal(size=tiny.nrows).astype(np.float32)
    g = A.adjoint(_to(r)).cpu().numpy()
    adj_check(g, oracle.spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r),
              oracle.abs_spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r))
    A.device_status()


@pytest.mark.parametrize("name", list(edge_case_matrices().keys()))
def test_forward_sell_edge_cases(name):
    csr = edge_case_matrices()[name]
    for sigma in (1, 64, 4096):
        for fmt in ("u16", "fp8"):
            A, enc = make(csr, fmt, sell=True, tuning=dict(sell_sigma=sigma))
            x = _x(csr.ncols, seed=3)
            # one lane per row (four accumulators): the per-row bound with 1 lane
            fwd_check(A.spmv(_to(x)).cpu().numpy(), oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x),
                      rtol=plain_row_bound(csr.row_lengths(), lanes=1))
            A.device_status()


@pytest.mark.parametrize("fmt", ["u16", "f16"])
def test_forward_column_windows_for_wide_matrices(fmt):
    """20000 spots (more than shared memory holds as one x): the forward schedule
    gets column windows and each CTA stages its window of x; FP32 and FP64
    vectors against the oracle, and the same with a window too wide to stage."""
    from dataclasses import replace
    beam = replace(dosegen.TINY, grid=(24, 40, 8), lattice=(100, 200), spacing=(0.24, 0.2), sigma=2.0, tau=0.3)
    csr = dosegen.generate(beam)
    assert csr.ncols == 20000
    # row blocks of 64 or 32 rows span ~3 voxel rows of y, so their windows are
    # narrow; the default 2048-row blocks span the whole 40-voxel grid
    for tuning in (None, dict(tile_nnz=2048, tile_rows=64), dict(tile_nnz=1024, tile_rows=32, stages=2)):
        A, enc = make(csr, fmt, tuning=tuning)
        inf = A.info()
        assert 0 < inf["fwd_window"] <= csr.ncols
        if tuning:
            assert inf["fwd_window"] < csr.ncols // 2
        x = _x(csr.ncols, seed=12)
        fwd_check(A.spmv(_to(x)).cpu().numpy(), oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x))
        x64 = dosegen.spot_weights_f64(csr.ncols, 13)
        d64 = A.spmv_f64(_to(x64)).cpu().numpy()
        ref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x64)
        absref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, np.abs(enc.decoded), x64)
        nz = absref > 0
        assert np.all(d64[~nz] == 0) and np.max(np.abs(d64[nz] - ref[nz]) / absref[nz]) <= 2.0 ** -40
        A.device_status()


def _banded_65536():
    """65536 spots, the most 16-bit column indices can address: 4096 rows of 48
    entries inside a 160-column band that slides across all the columns, so
    row 0 holds column 0 and the last row column 65535 (narrow column windows
    for both schedules)."""
    nrows, ncols, n, band = 4096, 65536, 48, 160
    rng = np.random.default_rng(65536)
    rp = np.arange(nrows + 1, dtype=np.uint32) * n
    cols = []
    for i in range(nrows):
        lo = (i * (ncols - band)) // (nrows - 1)
        c = np.sort(rng.choice(band, n, replace=False)) + lo
        if i == 0:
            c[0] = 0
        if i == nrows - 1:
            c[-1] = ncols - 1
        cols.append(c)
    col = np.concatenate(cols).astype(np.uint32)
    return dosegen.CSR(nrows, ncols, rp, col, rng.uniform(1e-3, 1.0, col.size))


@pytest.mark.parametrize("fmt", ["u16", "f16"])
@pytest.mark.parametrize("index16", [False, True])
def test_largest_16bit_column_range(fmt, index16):
    """Column 65535 through every path that reads column indices: the dose
    (FP32 and FP64 vectors, CSR and SELL), the adjoint and the fused pass."""
    csr = _banded_65536()
    assert csr.col.max() == 65535 and csr.col.min() == 0
    x = _x(csr.ncols, seed=14)
    x64 = dosegen.spot_weights_f64(csr.ncols, 15)
    for sell in (False, True):
        A, enc = make(csr, fmt, index16=index16, sell=sell)
        ref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x)
        fwd_check(A.spmv(_to(x)).cpu().numpy(), ref)
        if sell:
            continue
        d64 = A.spmv_f64(_to(x64)).cpu().numpy()
        ref64 = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x64)
        absref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, np.abs(enc.decoded), x64)
        assert np.max(np.abs(d64 - ref64) / absref) <= 2.0 ** -40
        r = np.random.default_rng(16).normal(size=csr.nrows).astype(np.float32)
        g_ref = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        g_abs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        adj_check(A.adjoint(_to(r)).cpu().numpy(), g_ref, g_abs)
        p = np.where(np.arange(csr.nrows) % 3 == 0, 1.0, 0.0).astype(np.float32)
        w = np.ones(csr.nrows, dtype=np.float32)
        f, g = A.fwd_adj_quadratic(_to(x), _to(p), _to(w))
        f_ref, g2_ref = oracle.fgrad(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, x, p, w)
        assert abs(float(f.item()) - f_ref) <= 1e-4 * f_ref
        _, r2 = oracle.objective(ref, p, w)
        g2_abs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r2)
        adj_check(g.cpu().numpy(), g2_ref, g2_abs, rtol=1e-4)
        A.device_status()


@pytest.mark.parametrize("storage", ["csr", "csr_index16", "sell"])
@pytest.mark.parametrize("fmt", ["u16", "fp8", "bf16", "f16", "f32"])
def test_compensated_long_rows_meet_1e5_on_every_row(storage, fmt):
    """Compensated accumulation where plain FP32 cannot promise 1e-5: the
    threshold rows (128 / 129), 4095-4097, the whole-CTA rows (8193, 16000) and
    a band of 400-8192-entry rows (a third with values falling over four
    decades), on the CSR kernel, with 16-bit column indices and on SELL; every
    row within 1e-5 of the FP64 oracle; plain sums on the same matrices within
    their per-row bound."""
    for name, csr in long_row_matrices().items():
        kw = dict(index16=storage == "csr_index16", sell=storage == "sell")
        if storage == "sell":
            kw["tuning"] = dict(sell_sigma=64)
        x = _x(csr.ncols, seed=9)
        for comp in (True, False):
            A, enc = make(csr, fmt, compensated=comp, **kw)
            ref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x)
            d = A.spmv(_to(x)).cpu().numpy()
            if comp:
                fwd_check(d, ref, rtol=1e-5)
            else:
                fwd_check(d, ref, rtol=plain_row_bound(csr.row_lengths(), lanes=1 if storage == "sell" else 8))
            d2 = A.spmv(_to(x)).cpu().numpy()
            assert np.array_equal(d.view(np.uint32), d2.view(np.uint32)), (name, comp)
            A.device_status()


def test_compensated_long_rows_adversarial():
    # descending magnitudes over 16000 entries: plain FP32 loses digits
    n = 16000
    rp = np.array([0, n], dtype=np.uint32)
    col = np.arange(n, dtype=np.uint32)
    val = np.geomspace(1.0, 1e-4, n)
    csr = dosegen.CSR(1, n, rp, col, val)
    A, enc = make(csr, "u16", compensated=True)
    x = np.ones(n, dtype=np.float32)
    d = A.spmv(_to(x)).cpu().numpy()
    ref = oracle.spmv(1, enc.row_ptr, enc.col, enc.decoded, x)
    rel = abs(float(d[0]) - ref[0]) / ref[0]
    # Dot2: about 2u of the result, then one rounding by the scale
    assert rel <= 4 * 2.0 ** -24, rel


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("fmt", ["u16", "bf16", "fp8", "f16", "f32"])
def test_adjoint_tiny_beam(tiny, fmt):
    A, enc = make(tiny, fmt)
    r = np.random.default_rng(4).normal(size=tiny.nrows).astype(np.float32)
    g = A.adjoint(_to(r)).cpu().numpy()
    ref = oracle.spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r)
    gabs = oracle.abs_spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r)
    adj_check(g, ref, gabs)
    g2 = A.adjoint(_to(r)).cpu().numpy()
    assert np.array_equal(g.view(np.uint32), g2.view(np.uint32))
    A.device_status()


@pytest.mark.parametrize("name", list(edge_case_matrices().keys()))
def test_adjoint_edge_cases(name):
    csr = edge_case_matrices()[name]
    if csr.ncols > 16384:
        csr = dosegen.random_csr(csr.nrows, 9000, seed=8,
                                 lengths=np.minimum(csr.row_lengths(), 9000))
    for tuning in (None, dict(tile_nnz=256, tile_rows=32, coop_nnz=64, stages=2, consumer_warps=4,
                              adj_tile_nnz=256, adj_tile_rows=32, adj_stages=2, adj_forward_warps=2,
                              adj_scatter_warps=3, adj_row_order=1)):
        A, enc = make(csr, "u16", tuning=tuning)
        r = np.random.default_rng(9).normal(size=csr.nrows).astype(np.float32)
        g = A.adjoint(_to(r)).cpu().numpy()
        ref = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        adj_check(g, ref, gabs)


def _banded_csr(nrows=30000, ncols=7000, span=180, long_row=None, seed=21):
    """Row i draws its columns from [start_i, start_i + span), start_i rising with i
    (a pencil beam's row blocks see only nearby spots); optionally one row holds
    every column."""
    rng = np.random.default_rng(seed)
    rp, cols = [0], []
    for i in range(nrows):
        if i == long_row:
            c = np.arange(ncols)
        else:
            start = (i * (ncols - span)) // nrows
            n = int(rng.integers(0, 48))
            c = start + np.sort(rng.choice(span, size=n, replace=False))
        cols.append(c)
        rp.append(rp[-1] + len(c))
    col = np.concatenate(cols).astype(np.uint32)
    val = rng.uniform(0.01, 1.0, col.size)
    return dosegen.CSR(nrows, ncols, np.asarray(rp, dtype=np.uint32), col, val)


@pytest.mark.parametrize("long_row", [None, 777])
def test_adjoint_column_windows(long_row):
    """Each CTA's adjoint works on a window of columns: banded matrices get a
    narrow window (wide with one row spanning every column), and the adjoint and
    the fused pass stay within tolerance of the oracle either way."""
    csr = _banded_csr(long_row=long_row)
    for tuning in (None, dict(adj_tile_nnz=512, adj_tile_rows=64, adj_stages=2, adj_scatter_warps=0)):
        A, enc = make(csr, "u16", tuning=tuning)
        info = A.info()
        if long_row is None:
            assert 32 <= info["adj_window"] < csr.ncols // 2, info["adj_window"]
        else:
            assert info["adj_window"] == (csr.ncols + 31) // 32 * 32
        rng = np.random.default_rng(3)
        r = rng.normal(size=csr.nrows).astype(np.float32)
        g = A.adjoint(_to(r)).cpu().numpy()
        ref = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        adj_check(g, ref, gabs)
        x = rng.uniform(0, 1, csr.ncols).astype(np.float32)
        p = np.where(rng.uniform(size=csr.nrows) < 0.3, 60.0, 0.0).astype(np.float32)
        w = np.where(p > 0, 10.0, 1.0).astype(np.float32)
        f, g2, d = A.fwd_adj_quadratic(_to(x), _to(p), _to(w), want_d=True)
        d = d.cpu().numpy()
        fwd_check(d, oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x))
        f_own, r2 = oracle.objective(d.astype(np.float64), p, w)
        assert abs(float(f.item()) - f_own) <= 1e-12 * f_own
        ref2 = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r2)
        gabs2 = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r2)
        adj_check(g2.cpu().numpy(), ref2, gabs2)
        A.device_status()


def test_adjoint_identity_on_gpu(tiny):
    A, enc = make(tiny, "u16")
    x = _x(tiny.ncols)
    y = np.random.default_rng(2).uniform(-1, 1, tiny.nrows).astype(np.float32)
    Ax = A.spmv(_to(x)).cpu().numpy().astype(np.float64)
    ATy = A.adjoint(_to(y)).cpu().numpy().astype(np.float64)
    scale = np.dot(oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x), np.abs(y))
    assert abs(np.dot(Ax, y) - np.dot(x.astype(np.float64), ATy)) <= 1e-5 * scale


# ------------------------------------------------------ fused objective pass

@pytest.fixture(scope="module")
def objective_inputs(tiny):
    p, w = dosegen.ellipsoid_target(dosegen.TINY)
    x = _x(tiny.ncols, seed=dosegen.weight_seed(dosegen.TINY))
    return p, w, x


@pytest.mark.parametrize("fmt", ["u16", "fp8"])
def test_fused_forward_adjoint_quadratic(tiny, objective_inputs, fmt):
    p, w, x = objective_inputs
    A, enc = make(tiny, fmt)
    f, g, d = A.fwd_adj_quadratic(_to(x), _to(p), _to(w), want_d=True)
    f, g, d = float(f.item()), g.cpu().numpy(), d.cpu().numpy()
    d_ref = oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x)
    fwd_check(d, d_ref)
    # f from the GPU's own FP32 dose, reduced in FP64 (tight), and end to end
    f_own, r_own = oracle.objective(d.astype(np.float64), p, w)
    assert abs(f - f_own) <= 1e-12 * f_own
    f_ref, _ = oracle.objective(d_ref, p, w)
    assert abs(f - f_ref) <= 1e-4 * f_ref
    g_ref = oracle.spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r_own)
    gabs = oracle.abs_spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r_own)
    adj_check(g, g_ref, gabs)
    # the unfused path gives the same gradient up to rounding
    g2 = A.adjoint(_to(r_own.astype(np.float32))).cpu().numpy()
    adj_check(g2, g_ref, gabs)


def test_gradient_matches_central_differences(tiny, objective_inputs):
    p, w, x = objective_inputs
    A, enc = make(tiny, "u16")
    f0, g = A.fwd_adj_quadratic(_to(x), _to(p), _to(w))
    g = g.cpu().numpy()
    _, g_exact = oracle.fgrad(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, x, p, w)
    h = 0.5
    for j in np.random.default_rng(6).choice(tiny.ncols, 20, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fp = float(A.fwd_adj_quadratic(_to(xp), _to(p), _to(w))[0].item())
        fm = float(A.fwd_adj_quadratic(_to(xm), _to(p), _to(w))[0].item())
        fd = (fp - fm) / (2 * h)
        scale = max(abs(g_exact[j]), 1e-3 * np.abs(g_exact).max())
        assert abs(fd - g[j]) <= 1e-3 * scale, (j, fd, g[j])
        assert abs(g[j] - g_exact[j]) <= 1e-4 * scale


def test_pg_100_iterations_in_one_graph(tiny, objective_inputs):
    p, w, x0 = objective_inputs
    A, enc = make(tiny, "u16")
    eta = oracle.pg_step_size(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, w)
    x_ref, f_ref = oracle.pg(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, x0, p, w, eta, 100)
    xg = _to(x0.copy())
    solver = dose.PGSolver(A, xg, _to(p), _to(w), eta, 100, use_graph=True)
    fh = solver.run().cpu().numpy()
    assert np.all(np.abs(fh - f_ref) <= 1e-4 * f_ref)
    np.testing.assert_allclose(xg.cpu().numpy(), x_ref, rtol=1e-3, atol=1e-4 * np.abs(x_ref).max())
    assert np.all(np.diff(fh) <= 1e-6 * fh[0])
    # eager replay of the same steps gives the same bits as the graph
    xe = _to(x0.copy())
    fe = dose.PGSolver(A, xe, _to(p), _to(w), eta, 100, use_graph=False).run().cpu().numpy()
    assert np.array_equal(fe.view(np.uint64), fh.view(np.uint64))
    assert np.array_equal(xe.cpu().numpy().view(np.uint32), xg.cpu().numpy().view(np.uint32))


# ---------------------------------------------------------------- autograd

def test_autograd_function_uses_adjoint(tiny, objective_inputs):
    p, w, x = objective_inputs
    A, enc = make(tiny, "u16")
    xt = _to(x).requires_grad_(True)
    d = dose.dose_spmv(A, xt)
    r = torch.randn(tiny.nrows, device="cuda", dtype=torch.float32)
    (d * r).sum().backward()
    g_ref = oracle.spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r.cpu().numpy())
    gabs = oracle.abs_spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r.cpu().numpy())
    adj_check(xt.grad.cpu().numpy(), g_ref, gabs)
    xt2 = _to(x).requires_grad_(True)
    f = dose.QuadraticDoseObjective(A, xt2, _to(p), _to(w))
    (2.0 * f).backward()
    _, g = A.fwd_adj_quadratic(_to(x), _to(p), _to(w))
    assert torch.equal(xt2.grad, 2.0 * g)


# ----------------------------------------------------------------- batched

@pytest.mark.parametrize("nvec", [1, 5, 8, 12, 16])
def test_batched_spmm_small(nvec):
    """Mixed formats and row lengths: rows of ~6 to 700 entries take 1 to 32
    lanes per row, and a 2500-entry row the long-row path."""
    mats = [dosegen.random_csr(500 + 97 * i, 60 + 13 * i, seed=20 + i, density=0.1) for i in range(5)]
    mats.append(dosegen.random_csr(40, 3000, seed=30, lengths=[0, 2500] + [7] * 38))
    for k, n in enumerate((40, 100, 150, 700)):
        mats.append(dosegen.random_csr(48 + k, 1200, seed=40 + k, lengths=[n] * (48 + k)))
    handles, encs, Xs = [], [], []
    for i, m in enumerate(mats):
        A, enc = make(m, ("u16", "fp8", "bf16", "f16", "f32")[i % 5])
        handles.append(A)
        encs.append(enc)
        Xs.append(_to(dosegen.spot_weights(m.ncols, 100 + i, nvec=nvec).reshape(m.ncols, nvec)))
    Ds = dose.spmv_batched(handles, Xs)
    for m, enc, X, D in zip(mats, encs, Xs, Ds):
        ref = oracle.spmm(m.nrows, enc.row_ptr, enc.col, enc.decoded, X.cpu().numpy().astype(np.float64))
        fwd_check(D.cpu().numpy().reshape(-1), ref.reshape(-1))
    Ds2 = dose.spmv_batched(handles, Xs)
    for D, D2 in zip(Ds, Ds2):
        assert torch.equal(D, D2)


def _small_beam_batch():
    """Six pencil beams: two grids x three lateral setup shifts."""
    from dataclasses import replace
    b2 = replace(dosegen.TINY, grid=(40, 36, 24), lattice=(30, 24), spacing=(40 / 30, 36 / 24),
                 seed=dosegen.SEED0 + 50)
    out = []
    for base in (dosegen.TINY, b2):
        for sh in ((-3.0, 0.0), (0.0, 0.0), (3.0, 3.0)):
            out.append(dosegen.generate(replace(base, shift=sh)))
    return out


def test_batched_spmm_pencil_beams_staged_and_graph():
    """Sixteen weight vectors over six pencil beams (mixed formats) in one launch:
    the staged form (each CTA's window of X in shared memory), checked against the
    oracle, bitwise repeatable, and identical when replayed from a CUDA graph."""
    mats = _small_beam_batch()
    fmts = ["u16", "bf16", "fp8", "f16", "f32", "bf16"]
    handles, encs, Xs = [], [], []
    for i, (m, f) in enumerate(zip(mats, fmts)):
        A, enc = make(m, f)
        handles.append(A)
        encs.append(enc)
        Xs.append(_to(dosegen.spot_weights(m.ncols, 200 + i, nvec=16).reshape(m.ncols, 16)))
    Ds = dose.spmv_batched(handles, Xs)
    for m, enc, X, D in zip(mats, encs, Xs, Ds):
        ref = oracle.spmm(m.nrows, enc.row_ptr, enc.col, enc.decoded, X.cpu().numpy().astype(np.float64))
        fwd_check(D.cpu().numpy().reshape(-1), ref.reshape(-1))
    first = [D.clone() for D in Ds]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        dose.spmv_batched(handles, Xs, Ds, stream=s)  # warm up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    for D in Ds:
        D.zero_()
    with torch.cuda.graph(graph, stream=s):
        dose.spmv_batched(handles, Xs, Ds, stream=s)
    for D in Ds:
        D.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    for D, F in zip(Ds, first):
        assert torch.equal(D, F)
    for A in handles:
        A.device_status()


@pytest.mark.parametrize("nvec", [4, 8, 12, 16])
def test_batched_spmm_staged_writes_stay_inside_d(nvec):
    """The staged form with every vector count that stores whole quads (nvec a
    multiple of 4): each D is the head of a larger buffer whose tail must come
    back untouched (nvec = 12 runs four quads of vectors, the fourth past the
    row)."""
    mats = _small_beam_batch()[:3]
    handles, encs, Xs, bufs, Ds = [], [], [], [], []
    for i, m in enumerate(mats):
        A, enc = make(m, ("u16", "bf16", "fp8")[i])
        handles.append(A)
        encs.append(enc)
        Xs.append(_to(dosegen.spot_weights(m.ncols, 300 + i, nvec=nvec).reshape(m.ncols, nvec)))
        buf = torch.full((m.nrows * nvec + 64,), 7.0, dtype=torch.float32, device="cuda")
        bufs.append(buf)
        Ds.append(buf[:m.nrows * nvec].view(m.nrows, nvec))
    dose.spmv_batched(handles, Xs, Ds)
    for m, enc, X, D, buf in zip(mats, encs, Xs, Ds, bufs):
        ref = oracle.spmm(m.nrows, enc.row_ptr, enc.col, enc.decoded, X.cpu().numpy().astype(np.float64))
        fwd_check(D.cpu().numpy().reshape(-1), ref.reshape(-1))
        assert torch.all(buf[m.nrows * nvec:] == 7.0)
    for A in handles:
        A.device_status()


def test_autotune_keeps_parity(tiny, objective_inputs):
    p, w, x = objective_inputs
    A, enc = make(tiny, "u16")
    best = A.autotune(_to(x))
    assert best["tile_nnz"] in (2048, 4096, 8192) and best["adj_tile_nnz"] in (2048, 4096, 5120, 6144, 8192)
    assert A.info()["tuning"] == best
    d = A.spmv(_to(x)).cpu().numpy()
    fwd_check(d, oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x))
    f, g = A.fwd_adj_quadratic(_to(x), _to(p), _to(w))
    f_ref, g_ref = oracle.fgrad(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, x, p, w)
    assert abs(float(f.item()) - f_ref) <= 1e-4 * f_ref
    _, r = oracle.objective(oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x), p, w)
    gabs = oracle.abs_spmv_t(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, r)
    adj_check(g.cpu().numpy(), g_ref, gabs, rtol=1e-4)
    A.device_status()


def test_bounded_wait_runs_out_and_the_context_stays_usable(tiny):
    """Failure detection without a fault: a wait on an mbarrier phase that never
    completes gives up after 20 ms and reports DOSE_ERR_TIMEOUT; the next call
    on the same context computes correctly."""
    import time
    t0 = time.perf_counter()
    assert dose.selftest_bounded_wait(20000) == 5
    assert time.perf_counter() - t0 < 5.0
    A, enc = make(tiny, "u16")
    x = _x(tiny.ncols)
    fwd_check(A.spmv(_to(x)).cpu().numpy(), oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x))
