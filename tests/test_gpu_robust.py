"""Multi-beam plans and robust scenario objectives against the FP64 oracle.

Multi-beam: the merged handle's dose with x = [x_1; ...; x_B] equals the sum of
the beams' doses (per-row relative error <= 1e-5, as every forward test), and
its adjoint gives every beam's gradient.  Robust objective: each scenario's
f_s equals the single-matrix fused pass bitwise; the worst case copies g_s*
bitwise; the expected value combines in FP64 (checked to one FP32 rounding);
end to end F is within 1e-4 of the oracle's and g within 1e-4 (|A|^T |r|) of
it, the bounds of the single-scenario fused tests.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import OFMT, adj_check, fwd_check

pytestmark = pytest.mark.gpu

BEAM = replace(dosegen.TINY, grid=(24, 20, 16), lattice=(10, 8), spacing=(2.0, 2.0))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    dose.build()
    dose.load()


def _to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _merge(beams):
    """Horizontal concatenation [A_1 A_2 ...] (test-side construction)."""
    nrows = beams[0].nrows
    offs = np.cumsum([0] + [b.ncols for b in beams])
    rps = [b.row_ptr.astype(np.int64) for b in beams]
    lens = sum(np.diff(rp) for rp in rps)
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.empty(int(rp[-1]), dtype=np.uint32)
    val = np.empty(int(rp[-1]))
    for i in range(nrows):
        k = rp[i]
        for b, o, brp in zip(beams, offs, rps):
            a, e = brp[i], brp[i + 1]
            col[k:k + e - a] = b.col[a:e] + o
            val[k:k + e - a] = b.val[a:e]
            k += e - a
    return dosegen.CSR(nrows, int(offs[-1]), rp.astype(np.uint32), col, val)


def _plan(shift=(0.0, 0.0)):
    return [dosegen.generate_along(replace(BEAM, seed=BEAM.seed + 11 * k, shift=shift), ax)
            for k, ax in enumerate(dosegen.ROBUST_AXES)]


@pytest.fixture(scope="module")
def plan():
    return _plan()


@pytest.mark.parametrize("fmt", ["f16", "bf16", "f32"])
def test_multibeam_from_codes_is_the_sum_of_beam_doses(plan, fmt):
    encs = [oracle.encode(b, OFMT[fmt]) for b in plan]
    A = dose.DoseMatrix.from_multibeam([(e.row_ptr, e.col, e.ncols, e.values, None) for e in encs], fmt=fmt)
    assert A.ncols == sum(b.ncols for b in plan) and A.nnz == sum(b.nnz for b in plan)
    xs = [dosegen.spot_weights(b.ncols, 40 + k) for k, b in enumerate(plan)]
    d = A.spmv(_to(np.concatenate(xs))).cpu().numpy()
    ref = oracle.multibeam_spmv([(e.nrows, e.row_ptr, e.col, e.decoded) for e in encs], xs)
    fwd_check(d, ref)
    # the adjoint of the plan is every beam's adjoint, stacked
    r = np.random.default_rng(5).normal(size=A.nrows).astype(np.float32)
    g = A.adjoint(_to(r)).cpu().numpy()
    g_ref = np.concatenate([oracle.spmv_t(e.nrows, e.ncols, e.row_ptr, e.col, e.decoded, r) for e in encs])
    g_abs = np.concatenate([oracle.abs_spmv_t(e.nrows, e.ncols, e.row_ptr, e.col, e.decoded, r) for e in encs])
    adj_check(g, g_ref, g_abs)
    A.device_status()


def test_multibeam_from_fp64_values_encodes_the_merged_matrix(plan):
    A = dose.DoseMatrix.from_multibeam([(b.row_ptr, b.col, b.ncols, b.val) for b in plan], fmt="u16", index16=True)
    merged = _merge(plan)
    enc = oracle.encode(merged, oracle.U16_SCALE)   # one scale for the whole plan
    assert A.info()["scale"] == float(enc.scales[0])
    x = np.concatenate([dosegen.spot_weights(b.ncols, 50 + k) for k, b in enumerate(plan)])
    fwd_check(A.spmv(_to(x)).cpu().numpy(), oracle.spmv(merged.nrows, enc.row_ptr, enc.col, enc.decoded, x))
    A.device_status()


def test_multibeam_rejects_unmergeable_codes(plan):
    e8 = [oracle.encode(b, oracle.FP8E4M3_ROWSCALE) for b in plan]
    with pytest.raises(dose.DoseError):
        dose.DoseMatrix.from_multibeam([(e.row_ptr, e.col, e.ncols, e.values, e.scales) for e in e8], fmt="fp8")
    e16 = [oracle.encode(b, oracle.U16_SCALE) for b in plan]   # a scale per beam
    with pytest.raises(dose.DoseError):
        dose.DoseMatrix.from_multibeam([(e.row_ptr, e.col, e.ncols, e.values, e.scales) for e in e16], fmt="u16")
    short = replace(BEAM, grid=(24, 20, 15))
    b2 = dosegen.generate(short)
    with pytest.raises(dose.DoseError):
        dose.DoseMatrix.from_multibeam([(plan[0].row_ptr, plan[0].col, plan[0].ncols, plan[0].val),
                                        (b2.row_ptr, b2.col, b2.ncols, b2.val)], fmt="u16")


@pytest.fixture(scope="module")
def scenarios():
    """Four setup shifts of the three-beam plan, each merged into one F16 handle."""
    out = []
    for sh in ((0.0, 0.0), (-3.0, 0.0), (3.0, 3.0), (0.0, -3.0)):
        beams = _plan(sh)
        encs = [oracle.encode(b, oracle.F16) for b in beams]
        A = dose.DoseMatrix.from_multibeam([(e.row_ptr, e.col, e.ncols, e.values, None) for e in encs], fmt="f16")
        out.append((A, encs))
    nx, ny, nz = BEAM.grid
    target = replace(BEAM, grid=(nx, ny, nz))
    p, w = dosegen.ellipsoid_target(target, semi_axes=(5.0, 4.0, 3.0), depth_frac=0.5)
    x = np.concatenate([dosegen.spot_weights(b.ncols, 60 + k) for k, b in enumerate(_plan())]) * 4.0
    return out, p, w, x


def _oracle_scen(encs):
    """One scenario for the oracle: the merged decoded matrix."""
    m = _merge([dosegen.CSR(e.nrows, e.ncols, e.row_ptr, e.col, e.decoded) for e in encs])
    return (m.nrows, m.ncols, m.row_ptr, m.col, m.val)


@pytest.mark.parametrize("mode", ["expected", "worst"])
def test_robust_objective_and_gradient(scenarios, mode):
    scen, p, w, x = scenarios
    mats = [A for A, _ in scen]
    prob = np.array([0.4, 0.3, 0.2, 0.1])
    S = dose.ScenarioSet(mats, prob)
    f_scen = torch.empty(len(mats), dtype=torch.float64, device="cuda")
    F, G, _ = S.robust_quadratic(_to(x), _to(p), _to(w), mode=mode, f_scen=f_scen)
    F, G, fs = float(F.item()), G.cpu().numpy(), f_scen.cpu().numpy()
    # each scenario's f_s and g_s are the single-matrix fused pass, bitwise
    gs = []
    for k, A in enumerate(mats):
        f1, g1 = A.fwd_adj_quadratic(_to(x), _to(p), _to(w))
        assert float(f1.item()) == fs[k]
        gs.append(g1.cpu().numpy())
    if mode == "expected":
        assert abs(F - float(np.dot(prob, fs))) <= 4e-15 * F
        G_own = (prob[:, None] * np.array(gs, dtype=np.float64)).sum(0).astype(np.float32)
        assert np.all(np.abs(G - G_own) <= np.spacing(np.abs(G_own)))
    else:
        best = int(np.argmax(fs))
        assert F == fs[best] and np.array_equal(G, gs[best])
    # end to end against the oracle
    oscen = [_oracle_scen(encs) for _, encs in scen]
    omode = oracle.EXPECTED if mode == "expected" else oracle.WORST_CASE
    F_ref, G_ref, fs_ref, arg = oracle.robust_quadratic(oscen, x, p, w, omode, prob)
    assert abs(F - F_ref) <= 1e-4 * F_ref
    assert np.all(np.abs(fs - fs_ref) <= 1e-4 * fs_ref)
    if mode == "worst":
        top = np.sort(fs_ref)[::-1]
        if top[0] - top[1] > 1e-3 * top[0]:
            assert int(np.argmax(fs)) == arg
    # gradient bound: sum over the scenarios that enter, of prob_s |A_s|^T |r_s|
    bound = np.zeros(len(G))
    for k, (nr, nc, rp, col, a) in enumerate(oscen):
        if mode == "worst" and k != arg:
            continue
        _, r = oracle.objective(oracle.spmv(nr, rp, col, a, x), p, w)
        bound += (prob[k] if mode == "expected" else 1.0) * oracle.abs_spmv_t(nr, nc, rp, col, a, r)
    adj_check(G, G_ref, bound, rtol=1e-4)
    # bitwise repeatable
    F2, G2 = S.robust_quadratic(_to(x), _to(p), _to(w), mode=mode)
    assert float(F2.item()) == F and np.array_equal(G2.cpu().numpy(), G)
    S.close()


@pytest.mark.parametrize("mode", ["expected", "worst"])
def test_robust_pg_step_updates_x_from_the_gradient(scenarios, mode):
    scen, p, w, x = scenarios
    S = dose.ScenarioSet([A for A, _ in scen])      # uniform probabilities
    F, G = S.robust_quadratic(_to(x), _to(p), _to(w), mode=mode)
    G = G.cpu().numpy()
    eta = np.float32(1e-6)
    xt = _to(x.astype(np.float32))
    g_out = torch.empty_like(xt)
    F2 = S.pg_step(xt, _to(p), _to(w), float(eta), mode=mode, g=g_out)
    assert float(F2.item()) == float(F.item())
    assert np.array_equal(g_out.cpu().numpy(), G)
    expect = np.maximum(np.float32(0), x.astype(np.float32) - eta * G.astype(np.float32))
    assert np.array_equal(xt.cpu().numpy(), expect)
    S.close()


def test_scenario_set_rejects_mismatched_shapes(scenarios, plan):
    scen, _, _, _ = scenarios
    other = dose.DoseMatrix.from_multibeam([(b.row_ptr, b.col, b.ncols, b.val) for b in plan[:2]], fmt="u16")
    with pytest.raises(dose.DoseError):
        dose.ScenarioSet([scen[0][0], other])
    with pytest.raises(dose.DoseError):
        dose.ScenarioSet([scen[0][0], scen[1][0]], prob=[0.7, 0.7])


@pytest.mark.parametrize("nan_at", [0, 1, 2])
def test_worst_case_reports_a_diverged_scenario(nan_at):
    """Three scenarios of one shape; in scenario nan_at one row reaches spot 0 with
    weight 0, and x_0 = 1e30 makes that row's dose overflow in (d - p)^2, so
    w (d - p)^2 = 0 * inf is NaN there: the worst case must be that scenario
    (F NaN, its g copied) wherever it sits among the scenarios."""
    nrows, ncols = 64, 32
    rng = np.random.default_rng(51)
    mats = []
    for s in range(3):
        # columns 1 .. ncols-1 only; the NaN scenario's row 5 also reaches column 0
        base = dosegen.random_csr(nrows, ncols - 1, seed=60 + s, lengths=rng.integers(1, 6, nrows))
        rp, cols, vals = [0], [], []
        brp = base.row_ptr.astype(np.int64)
        for i in range(nrows):
            c = list(base.col[brp[i]:brp[i + 1]] + 1)
            v = list(base.val[brp[i]:brp[i + 1]])
            if s == nan_at and i == 5:
                c, v = [0] + c, [0.5] + v
            cols += c
            vals += v
            rp.append(len(cols))
        mats.append(dose.DoseMatrix.from_csr(np.asarray(rp, dtype=np.uint32), np.asarray(cols, dtype=np.uint32),
                                             ncols=ncols, fmt="f32",
                                             values=np.asarray(vals, dtype=np.float32).view(np.uint32)))
    x = np.full(ncols, 0.5, dtype=np.float32)
    x[0] = 1e30
    p = np.zeros(nrows, dtype=np.float32)
    w = np.ones(nrows, dtype=np.float32)
    w[5] = 0.0
    S = dose.ScenarioSet(mats)
    f_scen = torch.empty(3, dtype=torch.float64, device="cuda")
    F, G, fs = S.robust_quadratic(_to(x), _to(p), _to(w), mode="worst", f_scen=f_scen)
    fs = fs.cpu().numpy()
    assert np.isnan(fs[nan_at]) and np.all(np.isfinite(np.delete(fs, nan_at)))
    assert np.isnan(float(F.item()))
    _, g_alone = mats[nan_at].fwd_adj_quadratic(_to(x), _to(p), _to(w))
    assert np.array_equal(G.cpu().numpy().view(np.uint32), g_alone.cpu().numpy().view(np.uint32))
    S.close()
