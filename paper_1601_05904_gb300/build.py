"""Builds the CUDA library ``libaidw.so`` in-tree for sm_103a (GB300).

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``), then linked into one shared
library next to this file.  A content hash of the sources and flags names
the build, so an unchanged tree is not rebuilt.

``build(checked=True)`` builds the same sources with -DAIDW_BOUNDS_CHECK
into ``libaidw_checked.so``: the kernels test the indices they compute
against their arrays and count failures (``aidw_bounds_report``), the
stand-in for a GPU memory checker.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libaidw.so")
LIB_CHECKED = os.path.join(PKG, "libaidw_checked.so")
CHECKED_FLAGS = ["-DAIDW_BOUNDS_CHECK"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--ftz=true", "--prec-div=true",
              "--prec-sqrt=true", "--fmad=true", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fno-strict-aliasing", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _tag(extra_flags=()) -> str:
    h = hashlib.sha1()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra_flags)).encode())
    return h.hexdigest()[:16]


def _compile(src: str, obj: str, extra: list[str]) -> tuple[str, int, str]:
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, r.returncode, r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checked: bool = False) -> str:
    """Compile and link libaidw.so (libaidw_checked.so if checked); returns
    its path."""
    flags = CHECKED_FLAGS if checked else []
    lib = LIB_CHECKED if checked else LIB
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    tag = _tag(flags)
    stamp = os.path.join(bdir, "stamp")
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == tag:
                return lib
    os.makedirs(bdir, exist_ok=True)
    extra = flags + (["-Xptxas", "-v"] if ptxas_info else [])
    objs = []
    jobs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        for src in _sources():
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            jobs.append(ex.submit(_compile, src, obj, extra))
        errors = []
        for fut in jobs:
            src, rc, out = fut.result()
            if verbose or ptxas_info or rc:
                print(f"== {os.path.basename(src)}\n{out}", end="")
            if rc:
                errors.append(src)
    if errors:
        raise RuntimeError("nvcc failed for " + ", ".join(os.path.basename(e) for e in errors))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(tag + "\n")
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
