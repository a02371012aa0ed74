"""Builds libhj_gb300.so in-tree with nvcc for sm_103a.

Each .cu translation unit compiles in its own nvcc process (in parallel),
then one link step produces the shared library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libhj_gb300.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["hj_kernels.cu", "hj_api.cu", "hj_batch.cu", "hj_server.cu", "hj_static.cu",
           "hj_filter.cu", "hj_jit.cu"]
# device headers that hj_jit.cu hands to NVRTC as text
JIT_HEADERS = ["hj_device.cuh", "hj_stage.cuh", "hj_group.cuh"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-ftz=true",
         "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC, "-I" + BUILD]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _cuda_lib64(cc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")


def _write_jit_sources() -> None:
    """hj_jit_sources.inc: the device headers as raw string literals."""
    names, bodies = [], []
    for h in JIT_HEADERS:
        text = open(os.path.join(CSRC, h)).read()
        if ")HJSRC\"" in text:
            raise RuntimeError("%s holds the raw-string delimiter" % h)
        names.append('"%s"' % h)
        bodies.append('R"HJSRC(%s)HJSRC"' % text)
    out = ("// generated by build.py from " + ", ".join(JIT_HEADERS) + "\n"
           "static const char* const kJitHeaderNames[] = {" + ", ".join(names) + "};\n"
           "static const char* const kJitHeaders[] = {\n" + ",\n".join(bodies) + "};\n")
    path = os.path.join(BUILD, "hj_jit_sources.inc")
    if not os.path.exists(path) or open(path).read() != out:
        with open(path, "w") as f:
            f.write(out)


def _deps_mtime() -> float:
    m = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= _deps_mtime():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    _write_jit_sources()
    defs = ['-DHJ_CUDA_LIB64="%s"' % _cuda_lib64(cc)]

    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(one, srcs))
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
