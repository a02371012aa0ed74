"""The C ABI library builds, loads and exports every entry point that
include/hj.h declares; the Python binding mirrors them.  No compute calls:
these run without a GPU."""
import os
import re
import subprocess

import pytest

from paper_2101_05916_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(hj_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    return build_mod.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hj_grid_create", "hj_set_dynamics", "hj_set_constraint",
              "hj_set_disturbance_bound", "hj_solve", "hj_solve_batch", "hj_prolong",
              "hj_query_value", "hj_query_gradient", "hj_get_value", "hj_set_value"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, missing


def test_binding_loads_and_mirrors_names(libpath):
    from paper_2101_05916_gb300 import hj
    L = hj.lib()
    for n in declared_functions():
        assert hasattr(L, n)
        assert n in hj.SIGNATURES, n
        assert hasattr(hj, n) or n in ("hj_grid_points",), n


def test_no_device_fails_loudly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2101_05916_gb300 import hj
    with pytest.raises(hj.HJError) as e:
        hj.hj_grid_create([5, 5], [0.0, 0.0], [1.0, 1.0])
    assert e.value.status == hj.HJ_ERR_CUDA


def test_default_opts(libpath):
    from paper_2101_05916_gb300 import hj
    o = hj.hj_default_opts()
    assert o.scheme == hj.HJ_WENO5 and o.cfl == 0.5 and o.tol == 1e-4 and o.check_dt == 0.1
    assert o.use_graph == 1


def test_allocator_hook_arguments(libpath):
    """hj_set_allocator needs both functions or neither; no device needed."""
    import ctypes
    L = ctypes.CDLL(libpath)
    L.hj_set_allocator.restype = ctypes.c_int
    L.hj_set_allocator.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert L.hj_set_allocator(None, None, None) == 0
    fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)(
        lambda n, d, u: None)
    assert L.hj_set_allocator(ctypes.cast(fn, ctypes.c_void_p), None, None) == 1  # HJ_ERR_ARG
    assert L.hj_set_allocator(None, None, None) == 0
