"""Out-of-memory paths, injected on the host: with DOSE_TEST_ALLOC_LIMIT set,
every device allocation of the library larger than the limit fails as out of
memory without reaching the driver.  No GPU fault is involved: the failing
calls return DOSE_ERR_OOM, release what they had allocated, and the same
process then creates and runs matrices normally."""
import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import fwd_check, make

pytestmark = pytest.mark.gpu

OOM = 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    dose.build()
    dose.load()


def _wide():
    """1 M entries over 8192 spots: the per-CTA gradient partials (152 CTAs x
    8192 columns x 4 B, ~5 MB) are the largest allocation, larger than the
    column indices (4 MB) and values (2 MB) allocated before them."""
    lens = np.full(4096, 256)
    return dosegen.random_csr(4096, 8192, seed=77, lengths=lens)


def test_create_fails_cleanly_past_its_large_arrays(monkeypatch):
    csr = _wide()
    enc = oracle.encode(csr, oracle.U16_SCALE)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    partials = sm * 8192 * 4
    assert partials > 4 * csr.nnz + 64  # the partials come after col and values and are larger
    monkeypatch.setenv("DOSE_TEST_ALLOC_LIMIT", str(partials - 1))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        with pytest.raises(dose.DoseError) as ei:
            dose.DoseMatrix.from_csr(enc.row_ptr, enc.col, ncols=csr.ncols, fmt="u16", values=enc.values,
                                     scales=enc.scales)
        assert ei.value.status == OOM
        assert "adjoint partials: out of device memory" in str(ei.value)
    torch.cuda.synchronize()
    # 20 failed creates that had allocated ~6 MB each: nothing left behind
    assert torch.cuda.mem_get_info()[0] >= free0 - (32 << 20)
    monkeypatch.delenv("DOSE_TEST_ALLOC_LIMIT")
    A, enc2 = make(csr, "u16")
    x = dosegen.spot_weights(csr.ncols, 78)
    fwd_check(A.spmv(torch.from_numpy(x).cuda()).cpu().numpy(),
              oracle.spmv(csr.nrows, enc2.row_ptr, enc2.col, enc2.decoded, x))
    A.device_status()


def test_create_reports_the_array_that_did_not_fit(monkeypatch):
    csr = _wide()
    enc = oracle.encode(csr, oracle.U16_SCALE)
    monkeypatch.setenv("DOSE_TEST_ALLOC_LIMIT", str(4 * csr.nnz - 1))  # the column indices no longer fit
    with pytest.raises(dose.DoseError) as ei:
        dose.DoseMatrix.from_csr(enc.row_ptr, enc.col, ncols=csr.ncols, fmt="u16", values=enc.values,
                                 scales=enc.scales)
    assert ei.value.status == OOM and "col_idx: out of device memory" in str(ei.value)
    # the library-encoding path (FP64 values in) takes the same exit
    with pytest.raises(dose.DoseError) as ei:
        dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="bf16", values_f64=csr.val)
    assert ei.value.status == OOM


def test_sell_copy_and_scenario_set_report_oom(monkeypatch):
    # SELL: the padded column array is the one allocation above the CSR's own
    lens = np.random.default_rng(79).integers(1, 200, 4096)
    csr = dosegen.random_csr(4096, 1000, seed=79, lengths=lens)
    enc = oracle.encode(csr, oracle.U16_SCALE)
    col_bytes = 4 * ((csr.nnz + 3) // 4 * 4 + 16)
    monkeypatch.setenv("DOSE_TEST_ALLOC_LIMIT", str(col_bytes))
    with pytest.raises(dose.DoseError) as ei:
        dose.DoseMatrix.from_csr(enc.row_ptr, enc.col, ncols=csr.ncols, fmt="u16", values=enc.values,
                                 scales=enc.scales, sell=True)
    assert ei.value.status == OOM and "SELL copy: out of device memory" in str(ei.value)
    # a scenario set's per-scenario gradients (S x ncols floats) above the limit
    A, _ = make(csr, "u16")  # every allocation of a plain handle fits
    monkeypatch.setenv("DOSE_TEST_ALLOC_LIMIT", str(8 * csr.ncols - 1))
    with pytest.raises(dose.DoseError) as ei:
        dose.ScenarioSet([A, A])
    assert ei.value.status == OOM
    # autotune's scratch (a dose vector of nrows floats) above the limit
    monkeypatch.setenv("DOSE_TEST_ALLOC_LIMIT", str(4 * csr.nrows - 1))
    with pytest.raises(dose.DoseError) as ei:
        A.autotune(torch.zeros(csr.ncols, device="cuda"))
    assert ei.value.status == OOM and "out of device memory" in str(ei.value)
    monkeypatch.delenv("DOSE_TEST_ALLOC_LIMIT")
    S = dose.ScenarioSet([A, A])
    S.close()
    A.device_status()


def test_row_group_layout_past_the_limit_falls_back_to_csr(monkeypatch):
    """The row-group arrays (union values: 4 stored values per union column) are
    larger than the CSR column indices; with the limit between the two, the
    default layout keeps the CSR passes and still matches the oracle, while an
    explicit adj_layout = 2 reports the out-of-memory failure."""
    lens = np.random.default_rng(81).integers(1, 200, 4096)
    csr = dosegen.random_csr(4096, 600, seed=81, lengths=lens)
    enc = oracle.encode(csr, oracle.U16_SCALE)
    col_bytes = 4 * ((csr.nnz + 3) // 4 * 4 + 16)
    monkeypatch.setenv("DOSE_TEST_ALLOC_LIMIT", str(col_bytes))
    with pytest.raises(dose.DoseError) as ei:
        make(csr, "u16", tuning=dict(adj_layout=2))
    assert ei.value.status == OOM and "row-group layout" in str(ei.value)
    A, enc = make(csr, "u16")
    monkeypatch.delenv("DOSE_TEST_ALLOC_LIMIT")
    inf = A.info()
    assert inf["rg_groups"] == 0 and inf["adj_layout_fused"] == 1
    r = np.random.default_rng(82).normal(size=csr.nrows).astype(np.float32)
    g = A.adjoint(torch.from_numpy(r).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
    gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
    assert np.all(np.abs(g - ref) <= 1e-5 * gabs + 1e-30)
    A.device_status()
