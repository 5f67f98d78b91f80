"""The C-ABI library loads on a CPU-only host, exports every entry point that
include/dose.h declares, and its host-side logic (argument validation, value
encoders) behaves as specified -- no GPU and no kernel launch needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import dosegen
import oracle
import paper_2103_09683_gb300 as dose

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    dose.build()
    return dose.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "dose.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dose_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "dose_spmv" in names and "dose_create_matrix" in names and len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in dose.EXPORTS, f"binding does not wrap {n}"
    assert lib.dose_version().startswith(b"libdose")


@pytest.mark.parametrize("fmt,ofmt", [("u16", oracle.U16_SCALE), ("bf16", oracle.BF16),
                                      ("fp8", oracle.FP8E4M3_ROWSCALE), ("f16", oracle.F16),
                                      ("f32", oracle.F32)])
def test_library_encoder_matches_oracle_bit_exact(lib, fmt, ofmt):
    A = dosegen.generate(dosegen.TINY)
    rng = np.random.default_rng(1)
    # add ties and awkward values: exact midpoints between codes, tiny and large entries
    val = A.val.copy()
    val[:50] = rng.uniform(0, 1e-6, 50)
    codes, scales = dose.encode_host(fmt, A.row_ptr, val)
    ref = oracle.encode(dosegen.CSR(A.nrows, A.ncols, A.row_ptr, A.col, val), ofmt)
    assert np.array_equal(codes, ref.values)
    if fmt not in ("bf16", "f16", "f32"):
        assert np.array_equal(scales, ref.scales)


def test_f16_encoder_on_ties_subnormals_and_overflow(lib):
    """Every halfway point between neighbouring finite halves, the subnormal
    range and the overflow threshold, against the oracle's encoder."""
    codes = np.arange(0, 0x7BFF, dtype=np.uint32).astype(np.uint16)
    lo = codes.view(np.float16).astype(np.float64)
    hi = (codes + 1).view(np.float16).astype(np.float64)
    v = np.concatenate([lo, 0.5 * (lo + hi), [65504.0, 65519.99, 65520.0, 1e6, 2.0 ** -25, 2.0 ** -26, 1e-300]])
    rp = np.array([0, v.size], dtype=np.uint32)
    got, scales = dose.encode_host("f16", rp, v)
    assert scales is None
    ref = np.array([oracle.f16_round(float(t)) for t in v], dtype=np.uint16)
    assert np.array_equal(got, ref)


def test_fp8_encoder_on_exact_ties(lib):
    # one row whose max is 448 * s with s = 1: every E4M3 midpoint in (0, 448]
    mids = []
    vals = sorted({oracle.fp8_e4m3_value(c) for c in range(0x7F)})
    for a, b in zip(vals[:-1], vals[1:]):
        mids += [a, 0.5 * (a + b)]
    mids.append(448.0)
    v = np.array(mids, dtype=np.float64)
    rp = np.array([0, v.size], dtype=np.uint32)
    codes, scales = dose.encode_host("fp8", rp, v)
    assert scales[0] == 1.0
    ref = [oracle.fp8_e4m3_nearest(t) for t in v]
    assert list(codes) == ref


def _desc(**kw):
    d = dose._Desc()
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_create_rejects_invalid_csr_on_host(lib):
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    out = ctypes.c_void_p()
    v = np.full(3, 0.5)
    cases = {
        "row_ptr[0]": dict(nrows=2, ncols=3, nnz=3, row_ptr=arr([1, 2, 3], np.uint32),
                           col_idx=arr([0, 1, 2], np.uint32)),
        "row_ptr[nrows]": dict(nrows=2, ncols=3, nnz=3, row_ptr=arr([0, 1, 2], np.uint32),
                               col_idx=arr([0, 1, 2], np.uint32)),
        "non-decreasing": dict(nrows=2, ncols=3, nnz=3, row_ptr=arr([0, 4, 3], np.uint32),
                               col_idx=arr([0, 1, 2], np.uint32)),
        ">= ncols": dict(nrows=2, ncols=3, nnz=3, row_ptr=arr([0, 2, 3], np.uint32),
                         col_idx=arr([0, 3, 2], np.uint32)),
        "duplicate": dict(nrows=2, ncols=3, nnz=3, row_ptr=arr([0, 2, 3], np.uint32),
                          col_idx=arr([1, 1, 2], np.uint32)),
    }
    for needle, kw in cases.items():
        d = _desc(fmt=0, values_f64=arr(v, np.float64), **kw)
        st = lib.dose_create_matrix(ctypes.byref(d), 0, None, None, ctypes.byref(out))
        assert st == 1, needle
        assert needle in lib.dose_last_error().decode(), (needle, lib.dose_last_error())
    # negative value for the encoder, NULL arguments, unknown flags
    d = _desc(nrows=1, ncols=3, nnz=3, row_ptr=arr([0, 3], np.uint32), col_idx=arr([0, 1, 2], np.uint32),
              fmt=0, values_f64=arr([0.5, -1.0, 0.2], np.float64))
    assert lib.dose_create_matrix(ctypes.byref(d), 0, None, None, ctypes.byref(out)) == 1
    assert lib.dose_create_matrix(None, 0, None, None, ctypes.byref(out)) == 1
    assert lib.dose_create_matrix(ctypes.byref(d), 0x80, None, None, ctypes.byref(out)) == 1
    # 16-bit column indices need ncols <= 65536
    d = _desc(nrows=1, ncols=70000, nnz=3, row_ptr=arr([0, 3], np.uint32), col_idx=arr([0, 1, 69999], np.uint32),
              fmt=0, values_f64=arr([0.5, 1.0, 0.2], np.float64))
    assert lib.dose_create_matrix(ctypes.byref(d), dose.CREATE_U16_INDEX, None, None, ctypes.byref(out)) == 1
    assert "65536" in lib.dose_last_error().decode()
    assert lib.dose_destroy(None) == 0
    assert lib.dose_spmv(None, None, None, None) == 1
    assert lib.dose_spmv_batched(None, -1, None, None, 16, None) == 1
    lay, nl = ctypes.c_int(7), ctypes.c_int(7)
    assert lib.dose_spmv_batched_plan(None, 0, 16, ctypes.byref(lay), ctypes.byref(nl)) == 0
    assert (lay.value, nl.value) == (0, 0)
    assert lib.dose_spmv_batched_plan(None, 0, 17, ctypes.byref(lay), ctypes.byref(nl)) == 1
    assert lib.dose_spmv_batched_plan(None, 1, 16, ctypes.byref(lay), ctypes.byref(nl)) == 1
    assert lib.dose_spmv_batched_plan(None, 0, 16, None, ctypes.byref(nl)) == 1


def test_create_rejects_bad_descriptors_and_codes_on_host(lib):
    """Every create-time check that needs no device: sizes, missing arrays,
    flags, and non-finite codes or scales in each stored format."""
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    out = ctypes.c_void_p()
    rp, col = arr([0, 2, 3], np.uint32), arr([0, 2, 1], np.uint32)
    v64 = arr([0.5, 0.25, 1.0], np.float64)
    base = dict(nrows=2, ncols=3, nnz=3, row_ptr=rp, col_idx=col)

    def rejects(needle, flags=0, tuning=None, **kw):
        d = _desc(**{**base, **kw})
        st = lib.dose_create_matrix(ctypes.byref(d), flags, ctypes.byref(tuning) if tuning else None, None,
                                    ctypes.byref(out))
        msg = lib.dose_last_error().decode()
        assert st == 1 and needle in msg, (needle, st, msg)
        assert out.value is None

    rejects("nnz must be < 2^32", nnz=1 << 32, fmt=0, values_f64=v64)
    rejects("nrows must be < 2^32 - 1", nrows=0xFFFFFFFF, fmt=0, values_f64=v64)
    rejects("row_ptr is NULL", row_ptr=None, fmt=0, values_f64=v64)
    rejects("col_idx is NULL", col_idx=None, fmt=0, values_f64=v64)
    rejects("values_f64 must be host memory", on_device=1, fmt=0, values_f64=v64)
    rejects("neither values nor values_f64", fmt=0)
    rejects("unknown format", fmt=9, values_f64=v64)
    rejects("scales are NULL", fmt=0, values=arr([1, 2, 3], np.uint16))
    rejects("scales are NULL", fmt=2, values=arr([1, 2, 3], np.uint8))
    t = dose.Tuning(sell_sigma=(1 << 24) + 1)
    rejects("sell_sigma", flags=dose.CREATE_SELL, tuning=t, fmt=0, values_f64=v64)
    for bad in (0.0, -1.0, np.inf, np.nan):
        rejects("scales must be finite and positive", fmt=0, values=arr([1, 2, 3], np.uint16),
                scales=arr([bad], np.float32))
        rejects("scales must be finite and positive", fmt=2, values=arr([1, 2, 3], np.uint8),
                scales=arr([1.0, bad], np.float32))
    rejects("FP8 code is NaN at entry 1", fmt=2, values=arr([0x38, 0xFF, 0x10], np.uint8),
            scales=arr([1.0, 1.0], np.float32))
    rejects("F16 value is infinite or NaN at entry 2", fmt=3, values=arr([0x3C00, 0x3800, 0x7C00], np.uint16))
    rejects("BF16 value is infinite or NaN at entry 0", fmt=1, values=arr([0x7FC0, 0x3F80, 0x3F00], np.uint16))
    rejects("BF16 value is infinite or NaN at entry 1", fmt=1, values=arr([0x3F80, 0xFF80, 0x3F00], np.uint16))
    rejects("F32 value is infinite or NaN at entry 1", fmt=4,
            values=arr(np.array([1.0, np.inf, 0.5], np.float32).view(np.uint32), np.uint32))
    # the FP64-value path rejects what its encoders cannot represent
    rejects("", fmt=0, values_f64=arr([0.5, np.nan, 1.0], np.float64))


def test_multibeam_and_scenarios_reject_bad_arguments_on_host(lib):
    """dose_create_multibeam validates every beam on the host before merging;
    dose_create_scenarios rejects empty sets before touching a device."""
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    out = ctypes.c_void_p()
    ok = dict(nrows=2, ncols=3, nnz=3, row_ptr=arr([0, 2, 3], np.uint32), col_idx=arr([0, 1, 2], np.uint32),
              fmt=0, values_f64=arr([0.5, 0.25, 1.0], np.float64))
    cases = {
        "same voxel grid": [ok, dict(ok, nrows=1, row_ptr=arr([0, 3], np.uint32))],
        "same format": [ok, dict(ok, fmt=1)],
        "col_idx out of range": [ok, dict(ok, col_idx=arr([0, 3, 2], np.uint32))],
        "row_ptr must run from 0 to nnz": [ok, dict(ok, row_ptr=arr([0, 2, 2], np.uint32))],
        "host CSR arrays": [ok, dict(ok, on_device=1)],
    }
    for needle, beams in cases.items():
        descs = (dose._Desc * len(beams))(*[_desc(**b) for b in beams])
        st = lib.dose_create_multibeam(descs, len(beams), 0, None, None, ctypes.byref(out))
        assert st == 1, needle
        assert needle in lib.dose_last_error().decode(), (needle, lib.dose_last_error())
    assert lib.dose_create_multibeam(None, 0, 0, None, None, ctypes.byref(out)) == 1
    assert lib.dose_create_scenarios(None, 0, None, ctypes.byref(out)) == 1
    assert lib.dose_robust_quadratic(None, 0, None, None, None, None, None, None, None) == 1
    assert lib.dose_robust_pg_step(None, 0, None, None, None, ctypes.c_float(-1.0), None, None, None) == 1


def test_binding_has_no_cpu_path(lib, monkeypatch):
    """Host tensors are refused before any library call, and a missing
    libdose.so is an error: nothing computes on the CPU."""
    import torch

    A = dose.DoseMatrix(0, 8, 4, 0, "u16")  # a null handle: no call may reach the library
    x, v8 = torch.zeros(4), torch.zeros(8)
    calls = [lambda: A.spmv(x), lambda: A.spmv_f64(x.double()), lambda: A.adjoint(v8),
             lambda: A.fwd_adj_quadratic(x, v8, v8), lambda: A.pg_step(x, v8, v8, 0.1),
             lambda: dose.spmv_batched([A], [x.reshape(4, 1)])]
    for call in calls:
        with pytest.raises(TypeError, match="CUDA tensor"):
            call()
    A.close()
    monkeypatch.setattr(dose, "_lib", None)
    monkeypatch.setattr(dose._build, "LIB", "/nonexistent/libdose.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dose.load()
