"""The debug-checked variant of the library (DOSE_DEBUG_CHECKS) builds for
sm_103a, exports the same C ABI as the release library and is the one loaded
under DOSE_DEBUG_CHECKS=1 (host-side calls only here; its kernels run in
tests/test_gpu_debug_checks.py)."""
import os
import shutil
import subprocess
import sys

import pytest

import paper_2103_09683_gb300 as dose

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _exports(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    return sorted(line.split()[-1] for line in out.splitlines() if line.split()[-1].startswith("dose_"))


@pytest.mark.skipif(not shutil.which("nm"), reason="nm not available")
def test_debug_library_builds_and_exports_the_same_abi():
    rel = dose.build(debug=False)
    dbg = dose.build(debug=True)
    assert os.path.basename(dbg) == "libdose_debug.so" and dbg != rel
    assert _exports(dbg) == _exports(rel)
    assert len(_exports(rel)) >= 25


def test_environment_selects_the_debug_library():
    dose.build(debug=True)
    code = ("import paper_2103_09683_gb300 as d; lib = d.load(); "
            "print(lib._name); print(d.load().dose_version().decode())")
    env = dict(os.environ, DOSE_DEBUG_CHECKS="1", PYTHONPATH=ROOT)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, env=env)
    assert res.returncode == 0, res.stderr
    assert "libdose_debug.so" in res.stdout and "libdose" in res.stdout.splitlines()[-1]
