"""Builds libosbpd.so (the CUDA library behind include/osbpd.h) for sm_103a, in-tree.

Each translation unit is compiled by its own nvcc process in parallel, then linked into
``paper_2309_11273_gb300/_build/libosbpd.so``.  The family-build unit is compiled with
``--fmad=false`` so that its horizon and crack decisions round each product separately.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libosbpd.so")
ROOT = os.path.dirname(HERE)
UNITS = {"pd_build.cu": ["--fmad=false"], "pd_step.cu": [], "pd_api.cu": [], "pd_noalloc.cu": []}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _sources():
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    deps.append(os.path.join(ROOT, "include", "osbpd.h"))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _sources())


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libosbpd.so if any source is newer than it; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    exe = nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I" + os.path.join(ROOT, "include"), "-Xptxas", "-v" if verbose else "-O3"]

    def compile_unit(item):
        name, extra = item
        obj = os.path.join(OUT, name.replace(".cu", ".o"))
        cmd = [exe, "-c", os.path.join(SRC, name), "-o", obj] + common + extra
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS.items()))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [exe, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
