"""The boundary from plain C: tests/c_abi_smoke.c includes include/hj.h,
links libhj_gb300.so with gcc and runs.  On the CPU, grid creation must fail
loudly (no device) and the device-free compile check must pass."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_compiles_and_links_as_c():
    from paper_2101_05916_gb300 import build
    so = build.build()
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    try:
        import torch
        gpu = torch.cuda.is_available()
    except Exception:
        gpu = False
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "c_abi_smoke")
        libdir = os.path.dirname(so)
        subprocess.check_call([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                               os.path.join(ROOT, "tests", "c_abi_smoke.c"), "-o", exe, "-L", libdir,
                               "-l:" + os.path.basename(so), "-Wl,-rpath," + libdir])
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    out = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    assert out["jit_check"] == "0"
    assert out["jit_check_bad"].startswith("1 ")   # HJ_ERR_ARG
    if not gpu:
        assert not out["grid_create"].startswith("0")
