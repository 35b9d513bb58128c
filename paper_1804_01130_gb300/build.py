"""Builds libgfm.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel; gfm_assemble.cu is compiled with
--fmad=false so the FP64 assembly rounds every operation as written.
Usage: python -m paper_1804_01130_gb300.build [--force] [-v]
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(HERE, f"libgfm_{platform.machine()}.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
UNITS = {
    "gfm_api.cu": [],
    "gfm_assemble.cu": ["--fmad=false"],
    "gfm_solve.cu": ["-Xptxas", "-v"],
    "gfm_coarse.cu": [],
    "gfm_setup.cpp": [],
    "gfm_noalloc.cu": ["-Xptxas", "-v"],
    "gfm_shard.cpp": [],
    "gfm_gradient.cu": [],
    "gfm_iso.cu": [],
}
HEADERS = ["gfm_internal.h", "gfm_setup.h"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: libgfm needs the CUDA toolkit to build")


def _newest_input() -> float:
    paths = [os.path.join(CSRC, u) for u in UNITS] + [os.path.join(CSRC, h) for h in HEADERS]
    paths.append(os.path.join(INCLUDE, "gfm.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit and link libgfm; returns the .so path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, unit + ".o")
        objs.append(obj)
        flags = COMMON + extra
        if unit.endswith(".cu"):
            flags = ARCH + flags
        cmd = [cc, *flags, "-c", src, "-o", obj]
        procs.append((unit, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for unit, cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(f"[libgfm] {unit}:\n{out}")
        if p.returncode != 0:
            failed.append(unit)
    if failed:
        raise RuntimeError(f"libgfm: compilation failed for {failed}")
    tmp = LIB + ".tmp"
    link = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"libgfm: link failed:\n{r.stdout}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
