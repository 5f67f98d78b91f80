"""A C program compiled against include/dose.h and linked to libdose.so (no
GPU): the header's struct layouts equal the Python binding's ctypes
declarations field by field, and the host-side calls behave as the header
documents (encoder values, host-side rejections with a message, NULL handling)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2103_09683_gb300 as dose

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client_output(tmp_path_factory):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    lib = dose.build()
    out = tmp_path_factory.mktemp("cabi")
    exe = str(out / "c_abi_client")
    libdir = os.path.dirname(lib)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-O1",
                           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_client.c"),
                           "-o", exe, lib, f"-Wl,-rpath,{libdir}"])
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    return res


def _layout(text):
    sizes, offs = {}, {}
    for line in text.splitlines():
        parts = line.split()
        if len(parts) == 3 and parts[0] == "sizeof":
            sizes[parts[1]] = int(parts[2])
        elif len(parts) == 3 and parts[0] == "offset":
            offs[parts[1]] = int(parts[2])
    return sizes, offs


def test_c_client_passes_its_checks(client_output):
    assert client_output.returncode == 0, client_output.stdout + client_output.stderr
    assert "ALL OK" in client_output.stdout
    assert client_output.stdout.count("rejected ") == 14


def test_header_layouts_match_the_binding(client_output):
    sizes, offs = _layout(client_output.stdout)
    structs = {"dose_csr_desc": dose._Desc, "dose_tuning": dose.Tuning, "dose_info": dose._Info}
    for cname, ctype in structs.items():
        assert sizes[cname] == ctypes.sizeof(ctype), cname
    checked = 0
    for key, off in offs.items():
        cname, field = key.split(".")
        assert getattr(structs[cname], field).offset == off, key
        checked += 1
    assert checked >= 30
