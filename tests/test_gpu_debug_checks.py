"""The debug-checked build (libdose_debug.so, DOSE_DEBUG_CHECKS): its
row-group kernels check every group record against its stage and every union
column against the CTA's window before they touch memory, and record
DOSE_ERR_BOUNDS instead of an out-of-bounds access.  On valid matrices it
computes the release build's bits and records nothing: the cases here (every
format on the tiny beam, small stage tiles, the edge-case matrices, 32-bit
union indices) run in a child process on the debug library and are compared
bit for bit with the release library's results from this process."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import dosegen
import paper_2103_09683_gb300 as dose
from gpu_helpers import edge_case_matrices, make

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    tiny = dosegen.generate(dosegen.TINY)
    out = [(tiny, fmt, None) for fmt in ("u16", "bf16", "fp8", "f16", "f32")]
    out.append((tiny, "u16", dict(rg_tile_union=320, rg_tile_rows=256)))
    for name in ("one_by_one", "empty_matrix", "one_row", "ragged_small_nc"):
        out.append((edge_case_matrices()[name], "u16", None))
    rng = np.random.default_rng(15)
    nrows, ncols, span = 3000, 70000, 150
    rp, cols = [0], []
    for i in range(nrows):
        start = (i * (ncols - span)) // nrows
        n = int(rng.integers(0, 40)) if i % 5 else 0
        cols.append(start + np.sort(rng.choice(span, size=n, replace=False)))
        rp.append(rp[-1] + n)
    col = np.concatenate(cols).astype(np.uint32)
    out.append((dosegen.CSR(nrows, ncols, np.asarray(rp, dtype=np.uint32), col, rng.uniform(0.01, 1.0, col.size)),
                "u16", None))
    return out


def test_debug_build_matches_release_bits_and_records_nothing(tmp_path):
    dose.build(debug=True)  # compiled here, loaded by the child
    data = {}
    cases = _cases()
    for k, (csr, fmt, tuning) in enumerate(cases):
        pre = f"c{k}_"
        A, enc = make(csr, fmt, tuning=tuning)
        assert A.info()["spmv_layout"] == 2 or csr.nrows == 0
        rng = np.random.default_rng(k)
        x = rng.uniform(0, 1, csr.ncols).astype(np.float32)
        p = np.where(rng.uniform(size=csr.nrows) < 0.3, 60.0, 0.0).astype(np.float32)
        w = np.where(p > 0, 10.0, 1.0).astype(np.float32)
        r = rng.normal(size=csr.nrows).astype(np.float32)
        X = rng.uniform(0, 1, (csr.ncols, 16)).astype(np.float32)
        xt, pt, wt, rt, Xt = (torch.from_numpy(a).cuda() for a in (x, p, w, r, X))
        f, g, d2 = A.fwd_adj_quadratic(xt, pt, wt, want_d=True)
        res = dict(d=A.spmv(xt), f=f, g=g, d2=d2, ga=A.adjoint(rt), D=dose.spmv_batched([A], [Xt])[0])
        A.device_status()
        data.update({pre + "fmt": np.array(fmt), pre + "rp": enc.row_ptr, pre + "col": enc.col,
                     pre + "ncols": np.array(csr.ncols), pre + "values": enc.values,
                     pre + "x": x, pre + "p": p, pre + "w": w, pre + "r": r, pre + "X": X})
        if enc.scales is not None:
            data[pre + "scales"] = np.asarray(enc.scales)
        for name, t in res.items():
            data[pre + name] = t.cpu().numpy()
        if tuning:
            data[pre + "tuning_keys"] = np.array(list(tuning))
            data[pre + "tuning_values"] = np.array(list(tuning.values()), dtype=np.int64)
    data["ncase"] = np.array(len(cases))
    path = str(tmp_path / "cases.npz")
    np.savez(path, **data)
    env = dict(os.environ, DOSE_DEBUG_CHECKS="1", PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    res = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_checks_child.py"), path],
                         capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    assert f"DEBUG CHECKS OK {len(cases)}" in res.stdout
