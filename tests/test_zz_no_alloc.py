"""dose_adjoint_noalloc: the adjoint for callers that cannot allocate device
memory (their device memory is owned by another runtime or a fixed arena, or
allocation is forbidden once they are running).  They hold A as device CSR
arrays and cannot create a handle; this entry point keeps its scratch in a
static device array.  Checked through the C ABI against the handle-based
dose_adjoint, with the adjoint tolerance used everywhere else
(|g - g_ref| <= 1e-5 (|A|^T |r|)_j), on two calls in a row -- the second call
reuses the static scratch the first one left behind -- for every stored
format; a warm call leaves the device's free memory unchanged and still works
when every library allocation would fail.

Collected last (file name) so that a stopping run has already run the rest.
"""
import os

import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import adj_check, make

pytestmark = pytest.mark.gpu

_VIEW = {"fp8": np.uint8, "f32": np.int32}  # stored-value bits as the binding takes them (else int16)


def _device_csr(enc, fmt, dev):
    row_ptr = torch.from_numpy(enc.row_ptr.view(np.int32)).to(dev)
    col = torch.from_numpy(enc.col.view(np.int32)).to(dev)
    values = torch.from_numpy(np.ascontiguousarray(enc.values).view(_VIEW.get(fmt, np.int16))).to(dev)
    row_scales = torch.from_numpy(enc.scales).to(dev) if fmt == "fp8" else None
    scale = float(enc.scales[0]) if fmt == "u16" else 1.0
    return row_ptr, col, values, row_scales, scale


@pytest.mark.parametrize("fmt", ["u16", "bf16", "fp8", "f16", "f32"])
def test_noalloc_adjoint_matches_handle_adjoint_twice(fmt):
    dose.build()
    csr = dosegen.generate(dosegen.TINY)
    A, enc = make(csr, fmt)
    dev = torch.device("cuda")
    row_ptr, col, values, row_scales, scale = _device_csr(enc, fmt, dev)
    for seed in (21, 22):
        r = np.random.default_rng(seed).normal(size=csr.nrows).astype(np.float32)
        rt = torch.from_numpy(r).to(dev)
        g_ref = A.adjoint(rt).cpu().numpy().astype(np.float64)
        g = dose.adjoint_noalloc(row_ptr, col, values, rt, ncols=csr.ncols, fmt=fmt, scale=scale,
                                 row_scales=row_scales)
        torch.cuda.synchronize()
        g = g.cpu().numpy()
        gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        adj_check(g, g_ref, gabs)
        adj_check(g, oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r), gabs)


def test_noalloc_adjoint_allocates_nothing():
    """A warm call with its output already allocated: the device's free memory is
    the same before and after, and the call still succeeds while every device
    allocation of the library would fail (DOSE_TEST_ALLOC_LIMIT=1)."""
    dose.build()
    csr = dosegen.generate(dosegen.TINY)
    A, enc = make(csr, "u16")
    dev = torch.device("cuda")
    row_ptr, col, values, row_scales, scale = _device_csr(enc, "u16", dev)
    r = torch.from_numpy(np.random.default_rng(5).normal(size=csr.nrows).astype(np.float32)).to(dev)
    g = torch.empty(csr.ncols, dtype=torch.float32, device=dev)
    dose.adjoint_noalloc(row_ptr, col, values, r, ncols=csr.ncols, scale=scale, g=g)  # first call: address lookup
    torch.cuda.synchronize()
    old = os.environ.get("DOSE_TEST_ALLOC_LIMIT")
    os.environ["DOSE_TEST_ALLOC_LIMIT"] = "1"
    try:
        with pytest.raises(dose.DoseError) as ei:  # the limit is in force: a create fails as out of memory
            make(csr, "u16")
        assert ei.value.status == 2
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        dose.adjoint_noalloc(row_ptr, col, values, r, ncols=csr.ncols, scale=scale, g=g)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    finally:
        if old is None:
            del os.environ["DOSE_TEST_ALLOC_LIMIT"]
        else:
            os.environ["DOSE_TEST_ALLOC_LIMIT"] = old
    assert free1 == free0
    gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r.cpu().numpy())
    adj_check(g.cpu().numpy(), A.adjoint(r).cpu().numpy().astype(np.float64), gabs)


def test_noalloc_adjoint_long_row_and_wide_accumulator():
    """One row of 16000 entries among short rows, with ncols close to the most
    columns one shared-memory accumulator holds: against the FP64 oracle."""
    dose.build()
    max_smem = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin", 227 * 1024)
    ncols = max_smem // 4 - 64
    lens = [3, 0, 16000, 7, 1, 0, 250]
    csr = dosegen.random_csr(len(lens), ncols, seed=41, lengths=lens)
    enc = oracle.encode(csr, oracle.U16_SCALE)
    dev = torch.device("cuda")
    row_ptr, col, values, row_scales, scale = _device_csr(enc, "u16", dev)
    r = np.random.default_rng(42).normal(size=csr.nrows).astype(np.float32)
    g = dose.adjoint_noalloc(row_ptr, col, values, torch.from_numpy(r).to(dev), ncols=ncols, scale=scale)
    torch.cuda.synchronize()
    adj_check(g.cpu().numpy(), oracle.spmv_t(csr.nrows, ncols, enc.row_ptr, enc.col, enc.decoded, r),
              oracle.abs_spmv_t(csr.nrows, ncols, enc.row_ptr, enc.col, enc.decoded, r))


def test_noalloc_adjoint_rejects_oversized_ncols():
    dose.build()
    dev = torch.device("cuda")
    row_ptr = torch.zeros(2, dtype=torch.int32, device=dev)
    col = torch.zeros(0, dtype=torch.int32, device=dev)
    values = torch.zeros(0, dtype=torch.int16, device=dev)
    r = torch.zeros(1, device=dev)
    with pytest.raises(dose.DoseError, match="exceeds the static scratch"):
        dose.adjoint_noalloc(row_ptr, col, values, r, ncols=(1 << 20) + 1, g=torch.zeros((1 << 20) + 1, device=dev))
