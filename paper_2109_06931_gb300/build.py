"""Build libhpa.so (the C-ABI library) from csrc/ with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into
paper_2109_06931_gb300/_build/libhpa.so.  Run `python -m
paper_2109_06931_gb300.build` or call build().  build(checked=True) makes
the bounds-checked flavour _build/libhpa_checked.so (-DHPA_CHECKED: an
out-of-range index computed on the device skips its access and makes the
call fail with HPA_E_INTERNAL and the site's number, never a trap).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhpa.so")
LIB_CHECKED = os.path.join(OUT, "libhpa_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhpa")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "hpa.h")]


def lib_path(checked: bool = False) -> str:
    return LIB_CHECKED if checked else LIB


def up_to_date(checked: bool = False) -> bool:
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    lib = lib_path(checked)
    if not force and up_to_date(checked):
        return lib
    objdir = os.path.join(OUT, "checked") if checked else OUT
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
                    "-I" + CSRC] + (["-DHPA_CHECKED"] if checked else []) + list(extra)
    objs = []

    def one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc()] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(one, _sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
