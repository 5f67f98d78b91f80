"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something other than itself: brute-force
dense products, library routines (scipy.sparse, torch dtype conversions),
closed forms, algebraic identities, or values the paper prints (Table I and the
Sec. V operational intensity, stored under tests/golden/).  Chosen so that a
dropped term, a wrong index, a transposed operand or a wrong rounding rule in
the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import dosegen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(csr_or_enc, a=None):
    nr, nc = csr_or_enc.nrows, csr_or_enc.ncols
    vals = csr_or_enc.val if a is None else a
    M = np.zeros((nr, nc))
    rp = csr_or_enc.row_ptr.astype(np.int64)
    for i in range(nr):
        for k in range(rp[i], rp[i + 1]):
            M[i, csr_or_enc.col[k]] += vals[k]
    return M


def _tiny_cases():
    out = [dosegen.random_csr(37, 23, seed=s, density=0.3) for s in range(4)]
    out.append(dosegen.random_csr(5, 7, seed=9, lengths=[0, 7, 1, 0, 3]))
    out.append(dosegen.random_csr(1, 1, seed=10, lengths=[1]))
    out.append(dosegen.random_csr(6, 4, seed=11, lengths=[0] * 6))
    return out


# ------------------------------------------------------------ SpMV: d = A x

@pytest.mark.parametrize("case", range(7))
def test_spmv_matches_dense_brute_force(case):
    A = _tiny_cases()[case]
    x = np.random.default_rng(case).uniform(0, 1, A.ncols)
    d = oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, x)
    # Pure-Python loop over the dense matrix in ascending column order: the same
    # order as CSR storage (columns ascending), so the sums agree exactly.
    M = _dense(A)
    ref = np.array([sum(M[i, j] * x[j] for j in range(A.ncols) if M[i, j] != 0.0)
                    for i in range(A.nrows)], dtype=np.float64)
    assert np.array_equal(d, ref)
    assert np.allclose(d, M @ x, rtol=1e-14, atol=0)


def test_spmv_matches_scipy_and_rows_sampling():
    A = dosegen.random_csr(300, 120, seed=3, density=0.05)
    x = np.random.default_rng(1).uniform(0, 1, A.ncols)
    d = oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, x)
    S = sp.csr_matrix((A.val, A.col.astype(np.int64), A.row_ptr.astype(np.int64)),
                      shape=(A.nrows, A.ncols))
    np.testing.assert_allclose(d, S @ x, rtol=1e-13, atol=0)
    rows = np.array([0, 5, 299, 17, 5], dtype=np.uint32)
    assert np.array_equal(oracle.spmv_rows(rows, A.row_ptr, A.col, A.val, x), d[rows])


def test_spmv_linearity():
    A = dosegen.random_csr(200, 60, seed=5, density=0.2)
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, A.ncols), rng.uniform(0, 1, A.ncols)
    al, be = 0.37, -1.9
    lhs = oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, al * x + be * y)
    rhs = al * oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, x) + \
        be * oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, y)
    scale = oracle.spmv(A.nrows, A.row_ptr, A.col, np.abs(A.val), np.abs(al * x) + np.abs(be * y))
    assert np.all(np.abs(lhs - rhs) <= 1e-14 * scale + 1e-300)


def test_spmv_unit_vectors_reproduce_columns_exactly():
    A = dosegen.random_csr(50, 12, seed=6, density=0.4)
    M = _dense(A)
    for j in range(A.ncols):
        e = np.zeros(A.ncols)
        e[j] = 1.0
        assert np.array_equal(oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, e), M[:, j])


def test_spmv_special_cases():
    n = 9
    ident = dosegen.CSR(n, n, np.arange(n + 1, dtype=np.uint32), np.arange(n, dtype=np.uint32),
                        np.ones(n))
    x = np.random.default_rng(3).uniform(0, 1, n)
    assert np.array_equal(oracle.spmv(n, ident.row_ptr, ident.col, ident.val, x), x)
    A = dosegen.random_csr(40, 10, seed=7, density=0.5)
    rs = oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, np.ones(A.ncols))
    ref = np.array([math.fsum(A.val[A.row_ptr[i]:A.row_ptr[i + 1]]) for i in range(A.nrows)])
    np.testing.assert_allclose(rs, ref, rtol=1e-15, atol=0)
    Z = dosegen.random_csr(8, 5, seed=8, lengths=[0] * 8)
    assert np.array_equal(oracle.spmv(8, Z.row_ptr, Z.col, Z.val, np.ones(5)), np.zeros(8))


def test_spmm_equals_columnwise_dense():
    A = dosegen.random_csr(64, 20, seed=12, density=0.3)
    X = np.random.default_rng(4).uniform(0, 1, (A.ncols, 5))
    D = oracle.spmm(A.nrows, A.row_ptr, A.col, A.val, X)
    np.testing.assert_allclose(D, _dense(A) @ X, rtol=1e-14, atol=0)


# ------------------------------------------------------------ adjoint: A^T r

def test_adjoint_identity_and_transpose():
    A = dosegen.random_csr(150, 40, seed=13, density=0.2)
    rng = np.random.default_rng(5)
    x, y = rng.uniform(0, 1, A.ncols), rng.normal(size=A.nrows)
    Ax = oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, x)
    ATy = oracle.spmv_t(A.nrows, A.ncols, A.row_ptr, A.col, A.val, y)
    scale = np.dot(oracle.spmv(A.nrows, A.row_ptr, A.col, A.val, np.abs(x)), np.abs(y))
    assert abs(np.dot(Ax, y) - np.dot(x, ATy)) <= 1e-13 * scale
    # A^T of the explicitly transposed CSR (scipy) matches the scatter form.
    S = sp.csr_matrix((A.val, A.col.astype(np.int64), A.row_ptr.astype(np.int64)),
                      shape=(A.nrows, A.ncols))
    T = S.T.tocsr()
    g_t = oracle.spmv(A.ncols, T.indptr.astype(np.uint32), T.indices.astype(np.uint32), T.data, y)
    np.testing.assert_allclose(ATy, g_t, rtol=1e-13, atol=1e-13 * np.abs(y).sum())
    np.testing.assert_allclose(ATy, _dense(A).T @ y, rtol=1e-12, atol=1e-13 * np.abs(y).sum())
    absg = oracle.abs_spmv_t(A.nrows, A.ncols, A.row_ptr, A.col, A.val, y)
    np.testing.assert_allclose(absg, np.abs(_dense(A)).T @ np.abs(y), rtol=1e-13, atol=0)


# ---------------------------------------------------- objective and gradient

def test_objective_closed_form():
    d = np.array([1.0, 2.0, 0.0, 5.0])
    p = np.array([0.0, 2.0, 60.0, 1.0])
    w = np.array([1.0, 10.0, 10.0, 1.0])
    f, r = oracle.objective(d, p, w)
    assert f == 1.0 + 0.0 + 36000.0 + 16.0
    assert np.array_equal(r, [2.0, 0.0, -1200.0, 8.0])


def test_gradient_central_differences_exact_for_quadratic():
    beam = dosegen.TINY
    A = dosegen.generate(beam)
    p, w = dosegen.ellipsoid_target(beam)
    x = dosegen.spot_weights(A.ncols, dosegen.weight_seed(beam)).astype(np.float64)
    f0, g = oracle.fgrad(A.nrows, A.ncols, A.row_ptr, A.col, A.val, x, p, w)
    h = 0.5
    spots = np.random.default_rng(6).choice(A.ncols, 20, replace=False)
    for j in spots:
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fp, _ = oracle.fgrad(A.nrows, A.ncols, A.row_ptr, A.col, A.val, xp, p, w)
        fm, _ = oracle.fgrad(A.nrows, A.ncols, A.row_ptr, A.col, A.val, xm, p, w)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-9 * max(abs(g[j]), 1e-6 * f0)


def test_pg_closed_form_on_diagonal_and_monotone_on_beam():
    n = 16
    rng = np.random.default_rng(7)
    a = rng.uniform(0.5, 2.0, n)
    diag = dosegen.CSR(n, n, np.arange(n + 1, dtype=np.uint32), np.arange(n, dtype=np.uint32), a)
    p = rng.uniform(0, 3, n)
    w = rng.choice([1.0, 10.0], n)
    x0 = rng.uniform(0, 1, n)
    eta = 0.01
    x1, fh = oracle.pg(n, n, diag.row_ptr, diag.col, diag.val, x0, p, w, eta, 1)
    ref = np.maximum(0.0, x0 - eta * 2 * w * a * (a * x0 - p))
    np.testing.assert_allclose(x1, ref, rtol=1e-15, atol=1e-15)
    assert fh[0] == pytest.approx(np.sum(w * (a * x0 - p) ** 2), rel=1e-15)
    # lambda_max(A^T A) of a diagonal matrix is max a^2.
    lam = oracle.norm2_sq(n, n, diag.row_ptr, diag.col, diag.val, iters=2000)
    assert lam == pytest.approx(np.max(a) ** 2, rel=1e-6)

    beam = dosegen.TINY
    A = dosegen.generate(beam)
    enc = oracle.encode(A, oracle.U16_SCALE)
    pt, wt = dosegen.ellipsoid_target(beam)
    eta = oracle.pg_step_size(A.nrows, A.ncols, enc.row_ptr, enc.col, enc.decoded, wt)
    xs = dosegen.spot_weights(A.ncols, dosegen.weight_seed(beam))
    xf, fh = oracle.pg(A.nrows, A.ncols, enc.row_ptr, enc.col, enc.decoded, xs, pt, wt, eta, 30)
    assert np.all(xf >= 0)
    assert np.all(np.diff(fh) <= 1e-12 * fh[0])
    assert fh[-1] < fh[0]


# ------------------------------------------------- multi-beam and robust objective

def _merge_beams(beams):
    """Horizontal concatenation [A_1 A_2 ...] of CSR matrices with one row count."""
    nrows = beams[0].nrows
    offs = np.cumsum([0] + [b.ncols for b in beams])
    lens = sum(b.row_lengths() for b in beams)
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.empty(int(rp[-1]), dtype=np.uint32)
    val = np.empty(int(rp[-1]))
    for i in range(nrows):
        k = rp[i]
        for b, o in zip(beams, offs):
            a, e = b.row_ptr[i], b.row_ptr[i + 1]
            col[k:k + e - a] = b.col[a:e] + o
            val[k:k + e - a] = b.val[a:e]
            k += e - a
    return dosegen.CSR(nrows, int(offs[-1]), rp.astype(np.uint32), col, val)


def test_multibeam_dose_is_the_concatenated_product():
    """sum_b A_b x_b = [A_1 A_2 A_3][x_1; x_2; x_3], checked against the dense sum."""
    from dataclasses import replace
    beam = replace(dosegen.TINY, grid=(16, 14, 10), lattice=(8, 6), spacing=(2.0, 2.0))
    beams = [dosegen.generate_along(replace(beam, seed=beam.seed + k), ax) for k, ax in enumerate("zxy")]
    xs = [dosegen.spot_weights_f64(b.ncols, 30 + k) for k, b in enumerate(beams)]
    d = oracle.multibeam_spmv([(b.nrows, b.row_ptr, b.col, b.val) for b in beams], xs)
    dense = sum(sp.csr_matrix((b.val, b.col, b.row_ptr), shape=(b.nrows, b.ncols)).toarray() @ x
                for b, x in zip(beams, xs))
    assert np.allclose(d, dense, rtol=1e-14, atol=0)
    m = _merge_beams(beams)
    dm = oracle.spmv(m.nrows, m.row_ptr, m.col, m.val, np.concatenate(xs))
    assert np.allclose(d, dm, rtol=1e-14, atol=0)


def _scenarios(n=4):
    from dataclasses import replace
    base = replace(dosegen.TINY, grid=(16, 14, 10), lattice=(8, 6), spacing=(2.0, 2.0))
    out = []
    for k in range(n):
        m = dosegen.generate(replace(base, shift=(float(k % 3) - 1.0, float(k // 3) - 1.0)))
        out.append(m)
    return out


def test_robust_single_scenario_is_the_quadratic():
    m = _scenarios(1)[0]
    x = dosegen.spot_weights_f64(m.ncols, 5)
    p = np.where(np.arange(m.nrows) % 7 == 0, 60.0, 0.0)
    w = np.where(p > 0, 10.0, 1.0)
    f, g = oracle.fgrad(m.nrows, m.ncols, m.row_ptr, m.col, m.val, x, p, w)
    for mode in (oracle.EXPECTED, oracle.WORST_CASE):
        F, G, fs, arg = oracle.robust_quadratic([(m.nrows, m.ncols, m.row_ptr, m.col, m.val)], x, p, w, mode)
        assert F == f and np.array_equal(G, g)


def test_robust_expected_is_the_stacked_quadratic():
    """sum_s pi_s f(A_s x) is one quadratic over the row-stacked matrix with
    voxel weights pi_s w: an independent construction of the same value."""
    ms = _scenarios(4)
    prob = np.array([0.1, 0.2, 0.3, 0.4])
    x = dosegen.spot_weights_f64(ms[0].ncols, 6)
    p = np.where(np.arange(ms[0].nrows) % 5 == 0, 60.0, 0.0)
    w = np.where(p > 0, 10.0, 1.0)
    F, G, fs, arg = oracle.robust_quadratic([(m.nrows, m.ncols, m.row_ptr, m.col, m.val) for m in ms],
                                            x, p, w, oracle.EXPECTED, prob)
    st = sp.vstack([sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(m.nrows, m.ncols)) for m in ms]).tocsr()
    st.sort_indices()
    P = np.tile(p, 4)
    W = np.concatenate([pr * w for pr in prob])
    f2, g2 = oracle.fgrad(st.shape[0], st.shape[1], st.indptr.astype(np.uint32), st.indices.astype(np.uint32),
                          st.data, x, P, W)
    assert abs(F - f2) <= 1e-13 * f2 and np.allclose(G, g2, rtol=1e-12, atol=1e-12 * np.abs(g2).max())
    assert arg == -1


def test_robust_worst_case_picks_the_largest_and_its_gradient():
    """Scaled copies A_s = c_s A: the worst case is the scenario with the largest
    f_s (first on ties), its gradient is c_s* A^T r_s*, and away from ties the
    max is locally that quadratic, so central differences are exact."""
    m = _scenarios(1)[0]
    x = dosegen.spot_weights_f64(m.ncols, 7)
    p = np.where(np.arange(m.nrows) % 7 == 0, 60.0, 0.0)
    w = np.where(p > 0, 10.0, 1.0)
    cs = [1.0, 3.0, 0.5, 3.0]     # f grows with c here (doses far above p): scenario 1 wins, 3 ties it
    scen = [(m.nrows, m.ncols, m.row_ptr, m.col, c * m.val) for c in cs]
    F, G, fs, arg = oracle.robust_quadratic(scen, x * 50, p, w, oracle.WORST_CASE)
    assert arg == 1 and fs[1] == fs[3] and F == fs[1] == fs.max()
    f1, g1 = oracle.fgrad(m.nrows, m.ncols, m.row_ptr, m.col, 3.0 * m.val, x * 50, p, w)
    assert F == f1 and np.array_equal(G, g1)
    cs = [1.0, 3.0, 0.5]
    scen = [(m.nrows, m.ncols, m.row_ptr, m.col, c * m.val) for c in cs]
    xs = x * 50
    F, G, fs, arg = oracle.robust_quadratic(scen, xs, p, w, oracle.WORST_CASE)
    h = 1e-3
    for j in (0, 7, m.ncols - 1):
        e = np.zeros(m.ncols)
        e[j] = h
        Fp = oracle.robust_quadratic(scen, xs + e, p, w, oracle.WORST_CASE)[0]
        Fm = oracle.robust_quadratic(scen, xs - e, p, w, oracle.WORST_CASE)[0]
        assert abs((Fp - Fm) / (2 * h) - G[j]) <= 1e-6 * max(1.0, abs(G[j]))


# ------------------------------------------------------------------ formats

def test_fp8_e4m3_code_table():
    vals = np.array([oracle.fp8_e4m3_value(c) for c in range(256)])
    assert vals[0x7E] == 448.0 and vals[0xFE] == -448.0           # largest finite
    assert vals[0x38] == 1.0 and vals[0x08] == 2.0 ** -6           # one, smallest normal
    assert vals[0x01] == 2.0 ** -9 and vals[0x07] == 7 * 2.0 ** -9  # subnormals
    assert math.isnan(vals[0x7F]) and math.isnan(vals[0xFF])        # the only NaNs
    assert np.sum(np.isnan(vals)) == 2 and not np.any(np.isinf(vals))
    assert np.all(np.diff(vals[:0x7F]) > 0)                         # monotone in the code
    # Library routine: torch's float8_e4m3fn has the same 254 finite values.
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    tv = codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()
    fin = ~np.isnan(vals)
    assert np.array_equal(tv[fin], vals[fin]) and np.all(np.isnan(tv[~fin]))


def test_fp8_nearest_matches_torch_rne():
    rng = np.random.default_rng(8)
    t = np.concatenate([rng.uniform(0, 448, 4000), rng.uniform(0, 0.02, 1000),
                        [0.0, 448.0, 2.0 ** -10, 3 * 2.0 ** -11, 1.0625, 1.1875, 17.0, 19.0]])
    t = t.astype(np.float32)   # exactly representable: one rounding on both sides
    ours = np.array([oracle.fp8_e4m3_nearest(float(v)) for v in t], dtype=np.uint8)
    ref = torch.from_numpy(t).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)
    assert oracle.fp8_e4m3_nearest(1e6) == 0x7E            # saturates at 448


def test_bf16_round_matches_torch_and_neighbour_search():
    rng = np.random.default_rng(9)
    f32 = np.concatenate([rng.uniform(0, 1, 3000), rng.uniform(0, 1e-3, 500),
                          [1.0, 1.00390625, 1.01171875, 2.0 ** -130]]).astype(np.float32)
    ours = np.array([oracle.bf16_round(float(v)) for v in f32], dtype=np.uint16)
    ref = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    # FP64 inputs (no exact FP32 form): the code is a nearest bf16, ties to even.
    for v in rng.uniform(1e-3, 1.0, 500):
        c = oracle.bf16_round(float(v))
        err = abs(oracle.bf16_value(c) - v)
        for nb in (c - 1, c + 1):
            e2 = abs(oracle.bf16_value(nb) - v)
            assert err < e2 or (err == e2 and c % 2 == 0)


def test_f16_code_table_matches_numpy():
    """Every binary16 bit pattern decodes to numpy's float16 value."""
    vals = np.array([oracle.f16_value(c) for c in range(65536)])
    ref = np.arange(65536, dtype=np.uint32).astype(np.uint16).view(np.float16).astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(vals), nan) and np.array_equal(vals[~nan], ref[~nan])
    assert np.signbit(vals[0x8000]) and not np.signbit(vals[0])
    assert vals[0x3C00] == 1.0 and vals[0x7BFF] == 65504.0 and vals[0x0001] == 2.0 ** -24
    assert vals[0x0400] == 2.0 ** -14 and vals[0x03FF] == 1023 * 2.0 ** -24


def test_f16_round_matches_numpy_rne():
    rng = np.random.default_rng(17)
    mids = []   # exact halfway points between neighbouring finite halves: ties
    for c in list(range(0, 0x7BFF, 97)) + [0x03FF, 0x0400, 0x3BFF, 0x3C00, 0x7BFE]:
        a = np.uint16(c).view(np.float16).astype(np.float64)
        b = np.uint16(c + 1).view(np.float16).astype(np.float64)
        mids.append((a + b) / 2)
    v = np.concatenate([rng.uniform(0, 1, 3000), rng.uniform(0, 1e-4, 1000), rng.uniform(0, 7e4, 500),
                        -rng.uniform(0, 10, 200), mids,
                        [0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e9, 2.0 ** -25, 3 * 2.0 ** -26,
                         2.0 ** -26, 2.0 ** -14 - 2.0 ** -25]])
    ours = np.array([oracle.f16_round(float(t)) for t in v], dtype=np.uint16)
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16).view(np.uint16)   # numpy rounds FP64 to half directly, ties to even
    assert np.array_equal(ours, ref)
    assert oracle.f16_round(65520.0) == 0x7C00 and oracle.f16_round(-1e9) == 0xFC00


def test_f16_encoding_error_bound():
    A = dosegen.random_csr(60, 30, seed=18, density=0.3)
    enc = oracle.encode(A, oracle.F16)
    assert enc.scales is None and enc.values.dtype == np.uint16
    assert np.array_equal(enc.values, A.val.astype(np.float16).view(np.uint16))
    normal = A.val >= 2.0 ** -14
    # 11 significant bits: unit roundoff 2^-11 for normal values, 2^-25 absolute below
    assert np.all(np.abs(enc.decoded - A.val)[normal] <= 2.0 ** -11 * A.val[normal])
    assert np.all(np.abs(enc.decoded - A.val)[~normal] <= 2.0 ** -25)


def test_f32_encoding_matches_numpy_rne():
    """FP32 storage (the paper's Single): numpy's FP64 -> FP32 rounding, including
    exact halfway points between neighbouring floats."""
    rng = np.random.default_rng(19)
    f = rng.uniform(0, 1, 200).astype(np.float32)
    mids = (f.astype(np.float64) + np.nextafter(f, np.float32(2)).astype(np.float64)) / 2
    v = np.concatenate([rng.uniform(0, 1, 3000), rng.uniform(0, 1e-30, 200), mids, [0.0, 1e-45, 3.4e38]])
    A = dosegen.CSR(1, v.size, np.array([0, v.size], dtype=np.uint32), np.arange(v.size, dtype=np.uint32), v)
    enc = oracle.encode(A, oracle.F32)
    assert enc.scales is None and enc.values.dtype == np.uint32
    assert np.array_equal(enc.values, v.astype(np.float32).view(np.uint32))
    assert np.array_equal(enc.decoded, v.astype(np.float32).astype(np.float64))
    # ties went to the even neighbour
    even = np.where(f.view(np.uint32) % 2 == 0, f, np.nextafter(f, np.float32(2)))
    assert np.array_equal(enc.values[3200:3400], even.view(np.uint32))


def test_u16_encoding_nearest_code():
    A = dosegen.random_csr(100, 50, seed=14, density=0.3)
    enc = oracle.encode(A, oracle.U16_SCALE)
    s = float(enc.scales[0])
    assert s == float(np.float32(A.val.max() / 65535.0))
    t = A.val / s
    q = enc.values.astype(np.float64)
    assert np.all(np.abs(q - np.minimum(t, 65535.0)) <= 0.5)
    ties = np.abs(q - t) == 0.5
    assert np.all(q[ties] % 2 == 0)
    assert np.array_equal(enc.decoded, s * q)
    # Exact ties and the clamp, constructed by hand.
    B = dosegen.CSR(1, 4, np.array([0, 4], dtype=np.uint32), np.arange(4, dtype=np.uint32),
                    np.array([65535.0, 2.5, 3.5, 65534.5]) * 2.0 ** -10)
    eb = oracle.encode(B, oracle.U16_SCALE)
    assert eb.scales[0] == np.float32(2.0 ** -10)
    assert list(eb.values) == [65535, 2, 4, 65534]


def test_fp8_rowscale_encoding():
    A = dosegen.random_csr(60, 30, seed=15, density=0.3, empty_frac=0.2)
    enc = oracle.encode(A, oracle.FP8E4M3_ROWSCALE)
    L = A.row_lengths()
    for i in range(A.nrows):
        k0, k1 = A.row_ptr[i], A.row_ptr[i + 1]
        if L[i] == 0:
            assert enc.scales[i] == 1.0
            continue
        s = enc.scales[i]
        assert s == np.float32(A.val[k0:k1].max() / 448.0)
        t = (A.val[k0:k1] / float(s)).astype(np.float32)
        ref = torch.from_numpy(t).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
        exact32 = A.val[k0:k1] / float(s) == t.astype(np.float64)
        assert np.array_equal(enc.values[k0:k1][exact32], ref[exact32])
        # relative error of a normal E4M3 code is at most 2^-4
        dec = enc.decoded[k0:k1]
        normal = dec >= float(s) * 2.0 ** -6
        assert np.all(np.abs(dec - A.val[k0:k1])[normal] <= 2.0 ** -4 * A.val[k0:k1][normal])


def test_bf16_encoding_error_bound():
    A = dosegen.random_csr(60, 30, seed=16, density=0.3)
    enc = oracle.encode(A, oracle.BF16)
    # 8 significant bits: unit roundoff 2^-8
    assert np.all(np.abs(enc.decoded - A.val) <= 2.0 ** -8 * A.val)


# ---------------------------------------------- printed values of the paper

def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_dimensions.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, nr, nc, nnz, ratio, size = line.split()
            rows.append((name, float(nr), float(nc), float(nnz), ratio, size))
    return rows


def _interval(printed: str):
    """Rounding interval of a printed decimal (e.g. '8.880' -> [8.8795, 8.8805])."""
    mant = printed.lower().split("e")[0]
    dec = len(mant.split(".")[1]) if "." in mant else 0
    exp = int(printed.lower().split("e")[1]) if "e" in printed.lower() else 0
    half = 0.5 * 10.0 ** (exp - dec)
    v = float(printed)
    return v - half, v + half


def test_operational_intensity_liver1_is_0332():
    with open(os.path.join(GOLDEN, "operational_intensity.txt")) as f:
        line = [ln for ln in f if not ln.startswith("#") and ln.strip()][0]
    name, printed, digits = line.split()
    t1 = {r[0]: r for r in _table1()}
    _, nr, nc, nnz, _, _ = t1[name]
    oi = oracle.paper_operational_intensity(nnz, nr, nc)
    assert round(oi, int(digits)) == float(printed)
    # A dropped row term or a 4-byte value width moves the third digit.
    assert round(2 * nnz / (6 * nnz + 8 * nc), 3) != float(printed)
    assert round(2 * nnz / (8 * nnz + 12 * nr + 8 * nc), 3) != float(printed)


def test_table1_sizes_and_ratios_follow_csr_widths():
    for name, nr, nc, nnz, ratio, size in _table1():
        # printed nnz is rounded to 3 digits: the size must fall inside the model's range
        n_lo, n_hi = _interval(f"{nnz:.2e}")
        s_lo, s_hi = _interval(size)
        m_lo = oracle.csr_storage_bytes(n_lo, nr) / 1e9
        m_hi = oracle.csr_storage_bytes(n_hi, nr) / 1e9
        assert m_lo <= s_hi and m_hi >= s_lo, name
        # 4-byte values (FP32) would not fit any row
        assert oracle.csr_storage_bytes(n_lo, nr, value_bytes=4) / 1e9 > s_hi, name
        r_lo, r_hi = _interval(ratio)
        dens = 100.0 * nnz / (nr * nc)
        assert r_lo * 0.995 <= dens <= r_hi * 1.005, name
