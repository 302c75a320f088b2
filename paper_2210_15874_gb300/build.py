"""Build libqnoise.so in-tree with nvcc for sm_103a (GB300).

Usage: python -m paper_2210_15874_gb300.build [--force]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libqnoise.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["qn_api.cpp", "qn_kernels.cu", "qn_noalloc.cu", "qn_tc.cu"]
HEADERS = [os.path.join(CSRC, "qn_internal.h"), os.path.join(INCLUDE, "qn.h")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel, link, and atomically replace libqnoise.so."""
    if not force and not _stale():
        return LIB
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
    with tempfile.TemporaryDirectory(prefix="qnbuild") as tmp:
        procs, objs = [], []
        for src in SOURCES:
            obj = os.path.join(tmp, src + ".o")
            cmd = [cc, *common, *ARCH, "-lineinfo", "-c", os.path.join(CSRC, src), "-o", obj]
            if src.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), cmd))
            objs.append(obj)
        for p, cmd in procs:
            out, _ = p.communicate()
            if p.returncode != 0 or verbose:
                sys.stderr.write(out.decode(errors="replace"))
            if p.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
        tmp_lib = os.path.join(tmp, "libqnoise.so")
        subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp_lib, *objs, "-lcudart"])
        shutil.copyfile(tmp_lib, LIB + ".tmp")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
