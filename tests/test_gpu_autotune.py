"""The autotuner with its cache on the GPU: a sweep stores the chosen knobs
under the matrix fingerprint and the GPU name; a second handle of the same
matrix takes them from the cache without timing and computes the same bits;
the knobs keep parity with the FP64 oracle for dose_spmv, the fused objective
pass and the 16-vector batched SpMM; the DOSE_AUTOTUNE environment switch
tunes handles at create."""
import json

import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import adj_check, fwd_check, make

pytestmark = pytest.mark.gpu

ALL = ("forward", "fused", "batched")
KNOB_KEYS = [name for name, _ in dose.Tuning._fields_]


def _to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def tiny():
    return dosegen.generate(dosegen.TINY)


@pytest.fixture(scope="module")
def inputs(tiny):
    p, w = dosegen.ellipsoid_target(dosegen.TINY)
    x = dosegen.spot_weights(tiny.ncols, dosegen.weight_seed(dosegen.TINY))
    return p, w, x


def _knobs(r):
    return {k: r[k] for k in KNOB_KEYS}


def _check_parity(A, enc, csr, p, w, x):
    d = A.spmv(_to(x)).cpu().numpy()
    fwd_check(d, oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x))
    f, g = A.fwd_adj_quadratic(_to(x), _to(p), _to(w))
    f_ref, g_ref = oracle.fgrad(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, x, p, w)
    assert abs(float(f.item()) - f_ref) <= 1e-5 * f_ref
    _, r = oracle.objective(oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x), p, w)
    gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
    adj_check(g.cpu().numpy(), g_ref, gabs, rtol=1e-5)
    X = dosegen.spot_weights(csr.ncols, 77, nvec=16).reshape(csr.ncols, 16)
    (D,) = dose.spmv_batched([A], [_to(X)])
    ref = oracle.spmm(csr.nrows, enc.row_ptr, enc.col, enc.decoded, X.astype(np.float64))
    fwd_check(D.cpu().numpy().reshape(-1), ref.reshape(-1))
    A.device_status()
    return d, f, g, D


def test_sweep_stores_and_cache_applies_with_parity(tmp_path, tiny, inputs):
    p, w, x = inputs
    cache = str(tmp_path / "autotune.json")
    A, enc = make(tiny, "u16")
    fp = A.info()["fingerprint"]
    assert fp == dose.fingerprint_host(enc.row_ptr, enc.col, ncols=tiny.ncols)
    r1 = A.autotune(_to(x), mode="cached", purposes=ALL, cache=cache)
    assert r1["source"] == "sweep" and r1["fingerprint"] == fp
    assert r1["ms_forward"] > 0 and r1["ms_fused"] > 0 and r1["ms_batched"] > 0
    assert _knobs(r1) == A.info()["tuning"]
    doc = json.load(open(cache))
    (e,) = doc["entries"]
    assert e["gpu"] == dose.gpu_name(0) and e["fingerprint"] == f"{fp:016x}" and e["purposes"] == 7
    assert e["tuning"] == A.info()["tuning"]
    out_a = _check_parity(A, enc, tiny, p, w, x)

    # a second handle of the same matrix: knobs from the cache, no timing, same bits
    B, _ = make(tiny, "u16")
    r2 = B.autotune(mode="cached", purposes=ALL, cache=cache)
    assert r2["source"] == "cache" and _knobs(r2) == _knobs(r1)
    assert (r2["ms_forward"], r2["ms_fused"], r2["ms_batched"]) == pytest.approx(
        (r1["ms_forward"], r1["ms_fused"], r1["ms_batched"]))
    assert B.info()["tuning"] == A.info()["tuning"]
    out_b = _check_parity(B, enc, tiny, p, w, x)
    for a, b in zip(out_a, out_b):
        assert torch.equal(torch.as_tensor(a), torch.as_tensor(b))

    # another purpose set is another entry; "full" re-sweeps and replaces
    r3 = B.autotune(mode="cached", purposes=("forward",), cache=cache)
    assert r3["source"] == "sweep" and r3["ms_fused"] == 0 and r3["ms_batched"] == 0
    r4 = B.autotune(mode="full", purposes=ALL, cache=cache)
    assert r4["source"] == "sweep"
    assert len(json.load(open(cache))["entries"]) == 2
    _check_parity(B, enc, tiny, p, w, x)

    # "off" changes nothing
    before = B.info()["tuning"]
    r5 = B.autotune(mode="off", cache=cache)
    assert r5["source"] == "off" and B.info()["tuning"] == before


def test_other_format_is_another_key(tmp_path, tiny, inputs):
    p, w, x = inputs
    cache = str(tmp_path / "autotune.json")
    A, _ = make(tiny, "u16")
    A.autotune(mode="cached", purposes=("forward", "fused"), cache=cache)
    B, enc = make(tiny, "fp8")
    assert B.info()["fingerprint"] != A.info()["fingerprint"]
    rb = B.autotune(mode="cached", purposes=("forward", "fused"), cache=cache)
    assert rb["source"] == "sweep"
    assert len(json.load(open(cache))["entries"]) == 2
    _check_parity(B, enc, tiny, p, w, x)


def test_environment_switch_tunes_at_create(tmp_path, monkeypatch, tiny, inputs):
    p, w, x = inputs
    cache = str(tmp_path / "env.json")
    monkeypatch.setenv("DOSE_AUTOTUNE_CACHE", cache)
    monkeypatch.setenv("DOSE_AUTOTUNE", "cached")
    A, enc = make(tiny, "u16")
    (e,) = json.load(open(cache))["entries"]
    assert e["purposes"] == 3 and e["tuning"] == A.info()["tuning"]
    B, _ = make(tiny, "u16")  # from the cache
    assert B.info()["tuning"] == A.info()["tuning"]
    assert len(json.load(open(cache))["entries"]) == 1
    _check_parity(B, enc, tiny, p, w, x)
    # explicit knobs at create win over the environment
    C, _ = make(tiny, "u16", tuning=dict(tile_nnz=2048))
    assert C.info()["tuning"]["tile_nnz"] == 2048
    monkeypatch.setenv("DOSE_AUTOTUNE", "sometimes")
    with pytest.raises(dose.DoseError, match="DOSE_AUTOTUNE must be"):
        make(tiny, "u16")
    monkeypatch.setenv("DOSE_AUTOTUNE", "off")
    D, _ = make(tiny, "u16")
    assert D.info()["tuning"]["tile_nnz"] != 0


def test_foreign_cache_file_is_refused_and_kept(tmp_path, tiny):
    cache = tmp_path / "foreign.json"
    cache.write_text('{"not": "a cache"}')
    A, _ = make(tiny, "u16")
    before = A.info()["tuning"]
    with pytest.raises(dose.DoseError, match="DOSE_ERR_IO"):
        A.autotune(mode="cached", cache=str(cache))
    assert cache.read_text() == '{"not": "a cache"}'
    assert A.info()["tuning"] == before
