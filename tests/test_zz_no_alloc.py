"""dose_adjoint_noalloc: the adjoint for callers that cannot allocate device
memory (their device memory is owned by another runtime or a fixed arena, or
allocation is forbidden once they are running).  They hold A as device CSR
arrays and cannot create a handle; this entry point keeps its scratch in a
static device array.  Checked through the C ABI against the handle-based
dose_adjoint, with the adjoint tolerance used everywhere else
(|g - g_ref| <= 1e-5 (|A|^T |r|)_j), on two calls in a row -- the second call
reuses the static scratch the first one left behind.

Collected last (file name) so that a stopping run has already run the rest.
"""
import numpy as np
import pytest
import torch

import dosegen
import oracle
import paper_2103_09683_gb300 as dose
from gpu_helpers import adj_check, make

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fmt", ["u16", "fp8"])
def test_noalloc_adjoint_matches_handle_adjoint_twice(fmt):
    dose.build()
    csr = dosegen.generate(dosegen.TINY)
    A, enc = make(csr, fmt)
    dev = torch.device("cuda")
    row_ptr = torch.from_numpy(enc.row_ptr.view(np.int32)).to(dev)
    col = torch.from_numpy(enc.col.view(np.int32)).to(dev)
    values = torch.from_numpy(enc.values.view(np.uint8 if fmt == "fp8" else np.int16)).to(dev)
    row_scales = torch.from_numpy(enc.scales).to(dev) if fmt == "fp8" else None
    scale = float(enc.scales[0]) if fmt == "u16" else 1.0
    gabs_cache = {}
    for call, seed in enumerate((21, 22)):
        r = np.random.default_rng(seed).normal(size=csr.nrows).astype(np.float32)
        rt = torch.from_numpy(r).to(dev)
        g_ref = A.adjoint(rt).cpu().numpy().astype(np.float64)
        g = dose.adjoint_noalloc(row_ptr, col, values, rt, ncols=csr.ncols, fmt=fmt, scale=scale,
                                 row_scales=row_scales)
        torch.cuda.synchronize()
        g = g.cpu().numpy()
        gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        gabs_cache[call] = gabs
        adj_check(g, g_ref, gabs)
        exact = oracle.spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
        adj_check(g, exact, gabs)


def test_noalloc_adjoint_rejects_oversized_ncols():
    dose.build()
    dev = torch.device("cuda")
    row_ptr = torch.zeros(2, dtype=torch.int32, device=dev)
    col = torch.zeros(0, dtype=torch.int32, device=dev)
    values = torch.zeros(0, dtype=torch.int16, device=dev)
    r = torch.zeros(1, device=dev)
    g = torch.zeros(1, device=dev)
    with pytest.raises(dose.DoseError, match="exceeds the static scratch"):
        dose.adjoint_noalloc(row_ptr, col, values, r, ncols=(1 << 20) + 1, g=torch.zeros((1 << 20) + 1, device=dev))
