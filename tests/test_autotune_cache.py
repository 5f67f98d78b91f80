"""The autotuner's cache on the host (no GPU): the structure fingerprint that
keys it, the JSON file's round trip through the library's reader and writer,
misses on every part of the key, replacement of an entry, and refusal to
overwrite a file that is not such a cache."""
import json
import os

import numpy as np
import pytest

import dosegen
import paper_2103_09683_gb300 as dose

GPU = "NVIDIA GB300 (152 SMs, sm_103)"
FWD, FUSED, BATCHED = dose.TUNE_FORWARD, dose.TUNE_FUSED, dose.TUNE_BATCHED


@pytest.fixture(scope="module")
def tiny():
    return dosegen.generate(dosegen.TINY)


def test_fingerprint_depends_on_structure_format_and_flags_only(tiny):
    rp, col = tiny.row_ptr, tiny.col
    fp = dose.fingerprint_host(rp, col, ncols=tiny.ncols)
    assert fp == dose.fingerprint_host(rp.copy(), col.copy(), ncols=tiny.ncols)
    assert fp != dose.fingerprint_host(rp, col, ncols=tiny.ncols, fmt="bf16")
    assert fp != dose.fingerprint_host(rp, col, ncols=tiny.ncols, flags=dose.CREATE_U16_INDEX)
    assert fp != dose.fingerprint_host(rp, col, ncols=tiny.ncols + 1)
    # one row's highest column moves up by one: a different key
    lens = np.diff(rp.astype(np.int64))
    i = next(r for r in np.flatnonzero(lens >= 3) if int(col[rp[r]:rp[r + 1]].max()) + 1 < tiny.ncols)
    i = int(i)
    c2 = col.copy()
    seg = c2[rp[i]:rp[i + 1]]
    seg[int(np.argmax(seg))] += 1
    assert fp != dose.fingerprint_host(rp, c2, ncols=tiny.ncols)
    # an entry moved to another row (same nnz): a different key
    rp2 = rp.copy()
    j = int(np.flatnonzero(np.diff(rp.astype(np.int64)) >= 1)[0])
    rp2[j + 1] -= 1
    assert fp != dose.fingerprint_host(rp2, col, ncols=tiny.ncols)
    # interior columns of a row do not enter (only its extent does)
    c3 = col.copy()
    seg = c3[rp[i]:rp[i + 1]]
    if len(seg) >= 3:
        order = np.argsort(seg)
        mid = rp[i] + order[1]
        if seg[order[1]] + 1 < seg[order[2]]:
            c3[mid] += 1
            assert fp == dose.fingerprint_host(rp, c3, ncols=tiny.ncols)


def test_fingerprint_rejects_bad_row_pointers():
    with pytest.raises(dose.DoseError, match="row_ptr"):
        dose.fingerprint_host(np.array([0, 2, 1], np.uint32), np.array([0], np.uint32), ncols=3)


def _tuning(seed):
    rng = np.random.default_rng(seed)
    return {name: int(rng.integers(1, 9000)) for name, _ in dose.Tuning._fields_}


def test_cache_round_trip_and_misses(tmp_path):
    path = str(tmp_path / "sub" / "dir" / "autotune.json")
    assert dose.autotune_cache_lookup(path, GPU, 123, FWD | FUSED) is None
    assert not os.path.exists(path)  # a lookup creates nothing
    t1, t2 = _tuning(1), _tuning(2)
    dose.autotune_cache_store(path, GPU, 0xDEADBEEF00112233, FWD | FUSED, t1, (0.15, 0.18, 0.0))
    dose.autotune_cache_store(path, GPU, 0xDEADBEEF00112233, BATCHED, t2, (0.0, 0.0, 0.28))
    got, ms = dose.autotune_cache_lookup(path, GPU, 0xDEADBEEF00112233, FWD | FUSED)
    assert got == t1 and ms == pytest.approx([0.15, 0.18, 0.0])
    got2, ms2 = dose.autotune_cache_lookup(path, GPU, 0xDEADBEEF00112233, BATCHED)
    assert got2 == t2 and ms2[2] == pytest.approx(0.28)
    # every part of the key misses on its own
    assert dose.autotune_cache_lookup(path, GPU, 0xDEADBEEF00112234, FWD | FUSED) is None
    assert dose.autotune_cache_lookup(path, "NVIDIA B200 (148 SMs, sm_100)", 0xDEADBEEF00112233, FWD | FUSED) is None
    assert dose.autotune_cache_lookup(path, GPU, 0xDEADBEEF00112233, FWD) is None
    # the file is plain JSON in the documented layout
    doc = json.load(open(path))
    assert doc["format"] == "dose-autotune-1" and len(doc["entries"]) == 2
    e = doc["entries"][0]
    assert e["gpu"] == GPU and e["fingerprint"] == "deadbeef00112233" and e["purposes"] == FWD | FUSED
    assert e["tuning"] == t1
    # storing the same key replaces the entry
    t3 = _tuning(3)
    dose.autotune_cache_store(path, GPU, 0xDEADBEEF00112233, FWD | FUSED, t3)
    assert len(json.load(open(path))["entries"]) == 2
    assert dose.autotune_cache_lookup(path, GPU, 0xDEADBEEF00112233, FWD | FUSED)[0] == t3
    assert not [f for f in os.listdir(os.path.dirname(path)) if ".tmp." in f]


def test_cache_reads_entries_written_by_hand(tmp_path):
    """Fields missing from an entry read as 0 (library default); entries
    without a key are skipped; escapes in the GPU name are honoured."""
    path = str(tmp_path / "hand.json")
    gpu = 'GPU "x"\\y'
    doc = {"format": "dose-autotune-1", "entries": [
        {"gpu": gpu, "fingerprint": "00000000000000ff", "purposes": 3, "tuning": {"tile_nnz": 4096}},
        {"fingerprint": "00000000000000ff", "purposes": 3, "tuning": {}},
    ]}
    with open(path, "w") as f:
        json.dump(doc, f)
    got, ms = dose.autotune_cache_lookup(path, gpu, 0xFF, 3)
    assert got["tile_nnz"] == 4096 and all(v == 0 for k, v in got.items() if k != "tile_nnz")
    assert ms == [0.0, 0.0, 0.0]


@pytest.mark.parametrize("text", ["not json", '{"format": "other", "entries": []}', '[1, 2]',
                                  '{"format": "dose-autotune-1", "entries": {}}', '{"format": "dose-autotune-1",'])
def test_cache_refuses_foreign_files_and_leaves_them(tmp_path, text):
    path = str(tmp_path / "foreign.json")
    with open(path, "w") as f:
        f.write(text)
    with pytest.raises(dose.DoseError, match="DOSE_ERR_IO"):
        dose.autotune_cache_lookup(path, GPU, 1, 3)
    with pytest.raises(dose.DoseError, match="DOSE_ERR_IO"):
        dose.autotune_cache_store(path, GPU, 1, 3, _tuning(4))
    assert open(path).read() == text


def test_cache_entry_with_bad_knob_is_skipped(tmp_path):
    path = str(tmp_path / "bad.json")
    doc = {"format": "dose-autotune-1", "entries": [
        {"gpu": GPU, "fingerprint": "0000000000000001", "purposes": 3, "tuning": {"tile_nnz": -5}},
        {"gpu": GPU, "fingerprint": "0000000000000002", "purposes": 3, "tuning": {"tile_nnz": 1.5}},
        {"gpu": GPU, "fingerprint": "0000000000000003", "purposes": 3, "tuning": {"tile_nnz": "8192"}},
    ]}
    with open(path, "w") as f:
        json.dump(doc, f)
    for fp in (1, 2, 3):
        assert dose.autotune_cache_lookup(path, GPU, fp, 3) is None
