"""The row-group layout of the adjoint and fused passes against the FP64 oracle.

Up to four consecutive non-empty rows share one list of the union of their
columns, with the rows' stored values side by side (stored zeros where a row
has no entry).  The layout changes which instructions add which terms, never
which terms are added: forward rows within 1e-5 relative, f within 1e-12 of
the oracle's f of the GPU's own dose, g componentwise within 1e-5 (|A|^T |r|)_j,
every result bitwise repeatable, and the CSR layout on the same handle inputs
held to the same bounds.
"""
import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import adj_check, edge_case_matrices, fwd_check, make

pytestmark = pytest.mark.gpu

FORMATS = ["u16", "bf16", "fp8", "f16", "f32"]
SMALL_TILES = dict(rg_tile_union=320, rg_tile_rows=256, rg_stages=2, rg_warps=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    dose.build()
    dose.load()


def _to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def tiny():
    return dosegen.generate(dosegen.TINY)


def _objective_inputs(csr, seed=5):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, csr.ncols).astype(np.float32)
    p = np.where(rng.uniform(size=csr.nrows) < 0.3, 60.0, 0.0).astype(np.float32)
    w = np.where(p > 0, 10.0, 1.0).astype(np.float32)
    return x, p, w


def _check_fused_and_adjoint(A, enc, csr, seed=5):
    """Fused pass (d, f, g) and the adjoint on the handle, against the oracle;
    a second call gives the same bits."""
    x, p, w = _objective_inputs(csr, seed)
    f, g, d = A.fwd_adj_quadratic(_to(x), _to(p), _to(w), want_d=True)
    f, g, d = float(f.item()), g.cpu().numpy(), d.cpu().numpy()
    d_ref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x)
    fwd_check(d, d_ref)
    f_own, r_own = oracle.objective(d.astype(np.float64), p, w)
    assert abs(f - f_own) <= 1e-12 * max(f_own, 1e-300)
    g_ref = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r_own)
    gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r_own)
    adj_check(g, g_ref, gabs)
    f2, g2, d2 = A.fwd_adj_quadratic(_to(x), _to(p), _to(w), want_d=True)
    assert float(f2.item()) == f
    assert np.array_equal(g2.cpu().numpy().view(np.uint32), g.view(np.uint32))
    assert np.array_equal(d2.cpu().numpy().view(np.uint32), d.view(np.uint32))
    r = np.random.default_rng(seed + 1).normal(size=csr.nrows).astype(np.float32)
    ga = A.adjoint(_to(r)).cpu().numpy()
    adj_check(ga, oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r),
              oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r))
    assert np.array_equal(A.adjoint(_to(r)).cpu().numpy().view(np.uint32), ga.view(np.uint32))
    A.device_status()


@pytest.mark.parametrize("fmt", FORMATS)
def test_row_groups_tiny_beam_every_format(tiny, fmt):
    A, enc = make(tiny, fmt, tuning=dict(adj_layout=2))
    info = A.info()
    assert info["adj_layout_fused"] == 2 and info["adj_layout_adjoint"] == 2
    assert info["rg_index_bytes"] == 2 and info["rg_groups"] > 0
    # every entry is in its group's union; groups of up to four rows
    assert info["rg_union_entries"] >= tiny.nnz / 4
    _check_fused_and_adjoint(A, enc, tiny)


@pytest.mark.parametrize("fmt", ["u16", "fp8"])
def test_row_groups_small_tiles_and_warps(tiny, fmt):
    """Stages of at most 320 union columns and 256 rows, a two-deep ring and three
    workers: many stages per CTA, groups spread over few warps."""
    A, enc = make(tiny, fmt, tuning=dict(adj_layout=2, **SMALL_TILES))
    assert A.info()["rg_warps_fused"] == 3
    _check_fused_and_adjoint(A, enc, tiny)


def test_row_groups_and_csr_layout_agree(tiny):
    """The same matrix on both layouts: both within the oracle's bounds, and
    switching layouts on one handle works."""
    A, enc = make(tiny, "u16")
    assert A.info()["adj_layout_fused"] == 2          # the default where row groups apply
    _check_fused_and_adjoint(A, enc, tiny)
    A.set_tuning(adj_layout=1)
    assert A.info()["adj_layout_fused"] == 1 and A.info()["adj_layout_adjoint"] == 1
    _check_fused_and_adjoint(A, enc, tiny)
    A.set_tuning(adj_layout=2)
    assert A.info()["adj_layout_fused"] == 2
    C, enc_c = make(tiny, "u16", tuning=dict(adj_layout=1))
    assert C.info()["rg_groups"] == 0 and C.info()["adj_layout_fused"] == 1
    with pytest.raises(dose.DoseError):
        C.set_tuning(adj_layout=2)


@pytest.mark.parametrize("name", ["one_by_one", "empty_matrix", "one_row", "ragged_small_nc"])
def test_row_groups_edge_cases(name):
    """One entry; no entries; one row of 257 entries (a group past the
    registers, summed in two passes over the stage); 3003 ragged rows over 64
    columns."""
    csr = edge_case_matrices()[name]
    for tuning in (dict(adj_layout=2), dict(adj_layout=2, **SMALL_TILES)):
        A, enc = make(csr, "u16", tuning=tuning)
        _check_fused_and_adjoint(A, enc, csr)


def test_row_groups_long_rows_past_registers():
    """Rows of 200-600 entries over 3000 columns: unions of more than 256
    columns take the two-pass path; neighbouring rows merge only while their
    union stays small."""
    rng = np.random.default_rng(12)
    lens = rng.integers(200, 600, 900)
    lens[::7] = 0
    csr = dosegen.random_csr(900, 3000, seed=13, lengths=lens)
    for fmt in ("u16", "f32"):
        A, enc = make(csr, fmt, tuning=dict(adj_layout=2))
        _check_fused_and_adjoint(A, enc, csr)


def test_row_groups_uncorrelated_rows():
    """Random rows share few columns: most groups hold one row, stored four
    values wide."""
    csr = dosegen.random_csr(5000, 700, seed=14, density=0.05, empty_frac=0.5)
    A, enc = make(csr, "bf16", tuning=dict(adj_layout=2))
    inf = A.info()
    assert inf["rg_groups"] >= 0.5 * np.count_nonzero(csr.row_lengths())
    _check_fused_and_adjoint(A, enc, csr)


def test_row_groups_32bit_union_indices():
    """More than 65536 spots: the union columns are stored as 32-bit indices;
    a banded matrix keeps each CTA's window narrow."""
    nrows, ncols, span = 20000, 70000, 150
    rng = np.random.default_rng(15)
    rp, cols = [0], []
    for i in range(nrows):
        start = (i * (ncols - span)) // nrows
        n = int(rng.integers(0, 40)) if i % 5 else 0
        c = start + np.sort(rng.choice(span, size=n, replace=False))
        cols.append(c)
        rp.append(rp[-1] + n)
    col = np.concatenate(cols).astype(np.uint32)
    csr = dosegen.CSR(nrows, ncols, np.asarray(rp, dtype=np.uint32), col, rng.uniform(0.01, 1.0, col.size))
    A, enc = make(csr, "u16", tuning=dict(adj_layout=2))
    info = A.info()
    assert info["rg_index_bytes"] == 4
    assert info["rg_window"] < ncols // 4
    _check_fused_and_adjoint(A, enc, csr)


def test_row_groups_ragged_vector_tails():
    """nrows not a multiple of 4: the last rows of p, w and r come from the
    producer's plain loads."""
    csr = dosegen.random_csr(4099, 90, seed=16, density=0.2, empty_frac=0.2)
    A, enc = make(csr, "fp8", tuning=dict(adj_layout=2, **SMALL_TILES))
    _check_fused_and_adjoint(A, enc, csr)


def test_row_groups_refused_for_rows_past_a_stage():
    """adj_layout = 2 on a matrix with a 5000-entry row: unsupported; the default
    layout falls back to CSR for it."""
    lens = [3, 5000, 7, 0]
    csr = dosegen.random_csr(4, 6000, seed=17, lengths=lens)
    with pytest.raises(dose.DoseError) as ei:
        make(csr, "u16", tuning=dict(adj_layout=2))
    assert ei.value.status == 4
    A, enc = make(csr, "u16")
    assert A.info()["rg_groups"] == 0 and A.info()["adj_layout_adjoint"] == 1
    r = np.random.default_rng(1).normal(size=csr.nrows).astype(np.float32)
    adj_check(A.adjoint(_to(r)).cpu().numpy(), oracle.spmv_t(4, 6000, enc.row_ptr, enc.col, enc.decoded, r),
              oracle.abs_spmv_t(4, 6000, enc.row_ptr, enc.col, enc.decoded, r))


def test_row_groups_pg_graph_matches_eager(tiny):
    """100 projected-gradient steps in one CUDA graph on the row-group layout,
    against the oracle's iterates, and bitwise equal to eager replay."""
    p, w = dosegen.ellipsoid_target(dosegen.TINY)
    x0 = dosegen.spot_weights(tiny.ncols, dosegen.weight_seed(dosegen.TINY))
    A, enc = make(tiny, "u16", tuning=dict(adj_layout=2))
    eta = oracle.pg_step_size(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, w)
    x_ref, f_ref = oracle.pg(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, x0, p, w, eta, 100)
    xg = _to(x0.copy())
    fh = dose.PGSolver(A, xg, _to(p), _to(w), eta, 100, use_graph=True).run().cpu().numpy()
    assert np.all(np.abs(fh - f_ref) <= 1e-4 * f_ref)
    xe = _to(x0.copy())
    fe = dose.PGSolver(A, xe, _to(p), _to(w), eta, 100, use_graph=False).run().cpu().numpy()
    assert np.array_equal(fe.view(np.uint64), fh.view(np.uint64))
    assert np.array_equal(xe.cpu().numpy().view(np.uint32), xg.cpu().numpy().view(np.uint32))


def test_pg_solver_resumes_from_a_checkpoint(tiny, tmp_path):
    """Run 50 graph-captured projected-gradient steps, checkpoint, then resume in
    a new solver (its own graph, x overwritten in place under the captured
    pointer) for 50 more: the final x and the f history of the second half are
    bitwise those of 100 uninterrupted steps."""
    p, w = dosegen.ellipsoid_target(dosegen.TINY)
    x0 = dosegen.spot_weights(tiny.ncols, dosegen.weight_seed(dosegen.TINY))
    A, enc = make(tiny, "u16")
    eta = oracle.pg_step_size(tiny.nrows, tiny.ncols, enc.row_ptr, enc.col, enc.decoded, w)
    pt, wt = _to(p), _to(w)
    x_full = _to(x0.copy())
    full = dose.PGSolver(A, x_full, pt, wt, eta, 50, use_graph=True)
    f_first = full.run().cpu().numpy().copy()
    f_second = full.run().cpu().numpy().copy()
    x_a = _to(x0.copy())
    first = dose.PGSolver(A, x_a, pt, wt, eta, 50, use_graph=True)
    assert np.array_equal(first.run().cpu().numpy().view(np.uint64), f_first.view(np.uint64))
    path = str(tmp_path / "pg50.npz")
    first.checkpoint(path)
    x_b = _to(np.zeros_like(x0))
    second = dose.PGSolver(A, x_b, pt, wt, eta, 50, use_graph=True)  # captured before the state is loaded
    assert second.resume(path) == 50
    f_b = second.run().cpu().numpy()
    assert np.array_equal(f_b.view(np.uint64), f_second.view(np.uint64))
    assert np.array_equal(x_b.cpu().numpy().view(np.uint32), x_full.cpu().numpy().view(np.uint32))
    assert second.steps_done == 100


def _beam_batch(n=4):
    from dataclasses import replace
    b2 = replace(dosegen.TINY, grid=(40, 36, 24), lattice=(30, 24), spacing=(40 / 30, 36 / 24),
                 seed=dosegen.SEED0 + 50)
    out = []
    for base in (dosegen.TINY, b2):
        for sh in ((-3.0, 0.0), (3.0, 3.0)):
            out.append(dosegen.generate(replace(base, shift=sh)))
    return out[:n]


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("nvec", [1, 3, 8, 13, 16])
def test_row_group_batched_spmm(fmt, nvec):
    """dose_spmv_batched on matrices of one format that all have the row-group
    layout: each D against the oracle's SpMM (per element, FP32 bound), rows
    without entries exactly 0 although D held garbage, the tail past each D
    untouched, bitwise repeatable, and within the bound of the same batch on
    CSR-layout handles."""
    mats = _beam_batch()
    handles, csr_handles, encs, Xs, bufs, Ds = [], [], [], [], [], []
    for i, m in enumerate(mats):
        A, enc = make(m, fmt)
        assert A.info()["rg_groups"] > 0
        C, _ = make(m, fmt, tuning=dict(adj_layout=1))
        handles.append(A)
        csr_handles.append(C)
        encs.append(enc)
        Xs.append(_to(dosegen.spot_weights(m.ncols, 400 + i, nvec=nvec).reshape(m.ncols, nvec)))
        buf = torch.full((m.nrows * nvec + 37,), -7.0, dtype=torch.float32, device="cuda")
        bufs.append(buf)
        Ds.append(buf[:m.nrows * nvec].view(m.nrows, nvec))
    assert dose.spmv_batched_plan(handles, nvec) == (2, 1)
    assert dose.spmv_batched_plan(csr_handles, nvec) == (1, 1)
    dose.spmv_batched(handles, Xs, Ds)
    first = [D.clone() for D in Ds]
    for m, enc, X, D, buf in zip(mats, encs, Xs, Ds, bufs):
        ref = oracle.spmm(m.nrows, enc.row_ptr, enc.col, enc.decoded, X.cpu().numpy().astype(np.float64))
        fwd_check(D.cpu().numpy().reshape(-1), ref.reshape(-1))
        assert torch.all(buf[m.nrows * nvec:] == -7.0)
    dose.spmv_batched(handles, Xs, Ds)
    for D, F in zip(Ds, first):
        assert torch.equal(D, F)
    Dc = dose.spmv_batched(csr_handles, Xs)
    for m, enc, X, D, C in zip(mats, encs, Xs, Ds, Dc):
        ref = oracle.spmm(m.nrows, enc.row_ptr, enc.col, enc.decoded, X.cpu().numpy().astype(np.float64))
        fwd_check(C.cpu().numpy().reshape(-1), ref.reshape(-1))


def test_row_group_batched_spmm_in_a_graph():
    """The row-group batch captured in a CUDA graph: the replay gives the same
    bits as the eager call; small stage tiles spread each matrix over many
    stages and the ring runs on across the matrices."""
    mats = _beam_batch()
    handles, Xs = [], []
    for i, m in enumerate(mats):
        A, _ = make(m, "u16", tuning=dict(rg_tile_union=320, rg_tile_rows=256))
        handles.append(A)
        Xs.append(_to(dosegen.spot_weights(m.ncols, 500 + i, nvec=16).reshape(m.ncols, 16)))
    eager = [D.clone() for D in dose.spmv_batched(handles, Xs)]
    Ds = [torch.empty_like(D) for D in eager]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        dose.spmv_batched(handles, Xs, Ds, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        dose.spmv_batched(handles, Xs, Ds, stream=s)
    for D in Ds:
        D.fill_(3.0)
    graph.replay()
    torch.cuda.synchronize()
    for D, E in zip(Ds, eager):
        assert torch.equal(D, E)
    for A in handles:
        A.device_status()


# ------------------------------------------------------------ dose_spmv on row groups

def _check_spmv_rg(A, enc, csr, seed=21):
    """dose_spmv on the row-group layout: every row against the oracle (per-row
    FP32 bound), rows without entries exactly 0 although d held garbage, the
    tail past d untouched, bitwise repeatable; unit vectors give the stored
    values bit-exactly."""
    assert A.info()["spmv_layout"] == 2
    x = np.random.default_rng(seed).uniform(0, 1, csr.ncols).astype(np.float32)
    buf = torch.full((csr.nrows + 33,), -5.0, dtype=torch.float32, device="cuda")
    d = buf[:csr.nrows]
    A.spmv(_to(x), d)
    ref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x)
    got = d.cpu().numpy()
    fwd_check(got, ref)
    empty = np.diff(enc.row_ptr.astype(np.int64)) == 0
    assert np.all(got[empty] == 0.0)
    assert torch.all(buf[csr.nrows:] == -5.0)
    assert np.array_equal(A.spmv(_to(x)).cpu().numpy().view(np.uint32), got.view(np.uint32))
    if csr.ncols:
        rows_of = np.repeat(np.arange(csr.nrows), np.diff(enc.row_ptr.astype(np.int64)))
        for j in np.random.default_rng(seed + 1).choice(csr.ncols, min(4, csr.ncols), replace=False):
            e = np.zeros(csr.ncols, dtype=np.float32)
            e[j] = 1.0
            expect = np.zeros(csr.nrows, dtype=np.float32)
            sel = enc.col == j
            expect[rows_of[sel]] = enc.decoded[sel].astype(np.float32)
            assert np.array_equal(A.spmv(_to(e)).cpu().numpy().view(np.uint32), expect.view(np.uint32)), j
    A.device_status()
    return got


@pytest.mark.parametrize("fmt", FORMATS)
def test_spmv_on_row_groups_every_format(tiny, fmt):
    """The default dose_spmv runs on the row-group layout; the CSR form
    (fwd_layout = 1) on the same handle meets the same bound; switching back
    gives the same bits as before."""
    A, enc = make(tiny, fmt)
    d_rg = _check_spmv_rg(A, enc, tiny)
    A.set_tuning(fwd_layout=1)
    assert A.info()["spmv_layout"] == 1 and A.info()["rg_spmv_bytes"] == 0
    x = np.random.default_rng(21).uniform(0, 1, tiny.ncols).astype(np.float32)
    fwd_check(A.spmv(_to(x)).cpu().numpy(), oracle.spmv(tiny.nrows, enc.row_ptr, enc.col, enc.decoded, x))
    A.set_tuning(fwd_layout=2)
    assert np.array_equal(A.spmv(_to(x)).cpu().numpy().view(np.uint32), d_rg.view(np.uint32))
    assert A.info()["rg_spmv_bytes"] > 0


@pytest.mark.parametrize("fmt", ["u16", "fp8"])
def test_spmv_on_row_groups_small_tiles(tiny, fmt):
    A, enc = make(tiny, fmt, tuning=SMALL_TILES)
    _check_spmv_rg(A, enc, tiny)


@pytest.mark.parametrize("name", ["one_by_one", "empty_matrix", "one_row", "ragged_small_nc"])
def test_spmv_on_row_groups_edge_cases(name):
    csr = edge_case_matrices()[name]
    for tuning in (dict(fwd_layout=2), dict(fwd_layout=2, **SMALL_TILES)):
        A, enc = make(csr, "u16", tuning=tuning)
        _check_spmv_rg(A, enc, csr)


def test_spmv_on_row_groups_wide_and_ragged():
    """Rows of 200-600 entries (unions past 256 columns), 32-bit union indices
    over 70000 spots, and nrows not a multiple of 32."""
    rng = np.random.default_rng(12)
    lens = rng.integers(200, 600, 901)
    lens[::7] = 0
    csr = dosegen.random_csr(901, 3000, seed=13, lengths=lens)
    for fmt in ("u16", "f32", "fp8"):
        A, enc = make(csr, fmt, tuning=dict(fwd_layout=2))
        _check_spmv_rg(A, enc, csr)
    nrows, ncols, span = 20003, 70000, 150
    rp, cols = [0], []
    for i in range(nrows):
        start = (i * (ncols - span)) // nrows
        n = int(rng.integers(0, 40)) if i % 5 else 0
        cols.append(start + np.sort(rng.choice(span, size=n, replace=False)))
        rp.append(rp[-1] + n)
    col = np.concatenate(cols).astype(np.uint32)
    csr = dosegen.CSR(nrows, ncols, np.asarray(rp, dtype=np.uint32), col, rng.uniform(0.01, 1.0, col.size))
    A, enc = make(csr, "u16")
    assert A.info()["rg_index_bytes"] == 4
    _check_spmv_rg(A, enc, csr)


def test_spmv_layout_fallbacks_and_refusals():
    """Compensated handles and rows past 4096 entries keep dose_spmv on CSR;
    fwd_layout = 2 is refused where the row-group form cannot run."""
    csr = dosegen.generate(dosegen.TINY)
    A, enc = make(csr, "u16", compensated=True)
    assert A.info()["spmv_layout"] == 1
    with pytest.raises(dose.DoseError) as ei:
        make(csr, "u16", compensated=True, tuning=dict(fwd_layout=2))
    assert ei.value.status == 4
    with pytest.raises(dose.DoseError):
        A.set_tuning(fwd_layout=2)
    long = dosegen.random_csr(4, 6000, seed=17, lengths=[3, 5000, 7, 0])
    B, encb = make(long, "u16")
    assert B.info()["spmv_layout"] == 1
    x = np.random.default_rng(3).uniform(0, 1, long.ncols).astype(np.float32)
    fwd_check(B.spmv(_to(x)).cpu().numpy(), oracle.spmv(4, encb.row_ptr, encb.col, encb.decoded, x))
    S, _ = make(csr, "u16", sell=True)
    assert S.info()["spmv_layout"] == 3


def test_spmv_on_row_groups_in_a_graph(tiny):
    """Captured in a CUDA graph: the replay gives the eager bits."""
    A, enc = make(tiny, "u16", tuning=SMALL_TILES)
    x = _to(np.random.default_rng(8).uniform(0, 1, tiny.ncols).astype(np.float32))
    eager = A.spmv(x).clone()
    d = torch.empty_like(eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        A.spmv(x, d, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        A.spmv(x, d, stream=s)
    d.fill_(7.0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(d, eager)
