"""Child process of tests/test_gpu_debug_checks.py: loads the debug-checked
library (DOSE_DEBUG_CHECKS=1 in its environment), recomputes the saved cases
and checks that every result equals the release library's bits and that no
kernel recorded an out-of-bounds index."""
import sys

import numpy as np
import torch

import paper_2103_09683_gb300 as dose


def main(path):
    assert dose.debug_checks(), "DOSE_DEBUG_CHECKS is not set"
    dose.build()
    lib = dose.load()
    import os
    assert os.path.basename(dose._build.LIB_DEBUG) in str(lib._name)
    z = np.load(path)
    ncase = int(z["ncase"])
    for k in range(ncase):
        pre = f"c{k}_"
        fmt = str(z[pre + "fmt"])
        tuning = None
        if pre + "tuning_keys" in z:
            tuning = {str(k): int(v) for k, v in zip(z[pre + "tuning_keys"], z[pre + "tuning_values"])}
        A = dose.DoseMatrix.from_csr(z[pre + "rp"], z[pre + "col"], ncols=int(z[pre + "ncols"]), fmt=fmt,
                                     values=z[pre + "values"], scales=z[pre + "scales"] if pre + "scales" in z else None,
                                     tuning=tuning)
        x, p, w, r = (torch.from_numpy(z[pre + n]).cuda() for n in ("x", "p", "w", "r"))
        X = torch.from_numpy(z[pre + "X"]).cuda()
        got = {"d": A.spmv(x)}
        f, g, d2 = A.fwd_adj_quadratic(x, p, w, want_d=True)
        got.update(f=f, g=g, d2=d2, ga=A.adjoint(r), D=dose.spmv_batched([A], [X])[0])
        A.device_status()  # DOSE_ERR_BOUNDS would raise here
        for name, t in got.items():
            ref = z[pre + name]
            a = t.cpu().numpy().reshape(ref.shape)
            assert np.array_equal(a.view(np.uint8), ref.view(np.uint8)), (k, name)
    print("DEBUG CHECKS OK", ncase)


if __name__ == "__main__":
    main(sys.argv[1])
