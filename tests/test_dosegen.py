"""The synthetic pencil-beam inputs have the structure the paper describes.

Sec. II-A/II-B: rows = voxels, columns = spots, rows far outnumber columns,
most rows are empty (about 70 % in Fig. 2) and row lengths are very uneven;
the non-zero ratio of the paper's matrices is 0.6-2 %.
"""
import numpy as np
import pytest

import dosegen


def test_tiny_beam_shape_and_nnz_target():
    A = dosegen.generate(dosegen.TINY)
    assert (A.nrows, A.ncols) == (20480, 500)
    assert abs(A.nnz - dosegen.NNZ_TARGETS["tiny"]) <= 0.05 * dosegen.NNZ_TARGETS["tiny"]
    assert 0.015 <= A.nnz / (A.nrows * A.ncols) <= 0.025       # ~2 % density
    rp = A.row_ptr.astype(np.int64)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == A.nnz
    for i in range(A.nrows):
        c = A.col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c.astype(np.int64)) > 0)         # ascending, unique
    assert A.col.max() < A.ncols
    assert A.val.min() >= dosegen.TINY.tau and A.val.max() <= 1.0


def test_clinical_beam_counts_and_row_length_profile():
    n, rl = dosegen.count_nnz(dosegen.CLINICAL, row_lengths=True)
    assert rl.size == 256 * 256 * 160
    assert abs(n - dosegen.NNZ_TARGETS["clinical"]) <= 0.05 * dosegen.NNZ_TARGETS["clinical"]
    empty = np.mean(rl == 0)
    assert 0.7 <= empty <= 0.95                                 # mostly empty rows
    assert 200 <= rl.max() <= 450                               # 0 to ~400 entries per row
    assert rl.size / dosegen.CLINICAL.ncols > 40                # rows >> columns


def test_liver1_shaped_beam_counts():
    """The paper-shaped matrix: Table I's liver beam 1 dimensions and nnz within
    1 %, about 70 % empty rows (Fig. 2), rows of thousands of entries."""
    b = dosegen.LIVER1_SHAPED
    n, rl = dosegen.count_nnz(b, row_lengths=True)
    assert b.nrows == 2_970_000 and b.ncols == 68_000
    assert abs(n - dosegen.NNZ_TARGETS["liver1"]) <= 0.01 * dosegen.NNZ_TARGETS["liver1"]
    assert 0.65 <= np.mean(rl == 0) <= 0.8
    assert rl.max() > 4000 and np.mean(rl[rl > 0] > 1024) > 0.5


def test_generation_is_deterministic():
    a = dosegen.generate(dosegen.TINY)
    b = dosegen.generate(dosegen.TINY)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.val, b.val)
    x1 = dosegen.spot_weights(500, 123)
    x2 = dosegen.spot_weights(500, 123)
    assert x1.dtype == np.float32 and np.array_equal(x1, x2)
    assert x1.min() >= 0.0 and x1.max() < 1.0
    assert not np.array_equal(x1, dosegen.spot_weights(500, 124))


def test_batched_scenarios_are_shifted_beams():
    beams = dosegen.batched_beams()
    assert len(beams) == 27
    assert len({b.shift for b in beams}) == 9
    assert sorted({b.ncols for b in beams}) == [1000, 2500, 4000]
    for b in beams:
        assert 2_000_000 <= b.nrows <= 8_000_000


def test_ellipsoid_target():
    p, w = dosegen.ellipsoid_target(dosegen.TINY)
    inside = p == 60.0
    assert inside.sum() > 0 and np.all(w[inside] == 10.0) and np.all(w[~inside] == 1.0)
    # semi-axes (8, 8, 4): volume ~ 4/3 pi 256 voxels
    assert abs(inside.sum() - 4.0 / 3.0 * np.pi * 256) < 0.15 * 4.0 / 3.0 * np.pi * 256


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_generate_along_permutes_rows_to_patient_order(axis):
    """Row (z*ny + y)*nx + x of a beam entering along `axis` is the generator's
    row at the permuted coordinates (depth axis = entry axis)."""
    from dataclasses import replace
    beam = replace(dosegen.TINY, grid=(12, 10, 8), lattice=(6, 5), spacing=(2.0, 2.0))
    nx, ny, nz = beam.grid
    pat = dosegen.generate_along(beam, axis)
    if axis == "z":
        g, gcoord = beam, lambda x, y, z: (x, y, z)
    elif axis == "x":
        g, gcoord = replace(beam, grid=(ny, nz, nx)), lambda x, y, z: (y, z, x)
    else:
        g, gcoord = replace(beam, grid=(nz, nx, ny)), lambda x, y, z: (z, x, y)
    gen = dosegen.generate(g)
    gnx, gny, _ = g.grid
    assert pat.nnz == gen.nnz and pat.nrows == gen.nrows
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                r = (z * ny + y) * nx + x
                gx, gy, gz = gcoord(x, y, z)
                q = (gz * gny + gy) * gnx + gx
                a = slice(pat.row_ptr[r], pat.row_ptr[r + 1])
                b = slice(gen.row_ptr[q], gen.row_ptr[q + 1])
                assert np.array_equal(pat.col[a], gen.col[b]) and np.array_equal(pat.val[a], gen.val[b])


def test_robust_plan_shapes():
    plan = dosegen.robust_plan()
    assert len(plan) == 9 and all(len(s) == 3 for s in plan)
    assert {ax for _, ax in plan[0]} == {"x", "y", "z"}
    assert len({b.shift for b, _ in (s[0] for s in plan)}) == 9
    assert all(b.grid == dosegen.ROBUST_GRID for s in plan for b, _ in s)
