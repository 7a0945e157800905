"""Build ``libmpcd.so`` (the C-ABI library of include/mpcd.h) for sm_103a.

The translation units are compiled in parallel with nvcc and linked
into ``paper_2604_14307_gb300/_build/libmpcd.so`` (in-tree).  The rigid-body
unit is compiled without fused multiply-add so that the FP64 body and
site-position arithmetic rounds exactly as written; host code never fuses.
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
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmpcd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "mpcd_api.cu": [],
    "kernels_solvent.cu": [],
    "kernels_bodies.cu": ["-fmad=false"],
    "static_collide.cu": [],
    "kernels_sort.cu": [],
    "kernels_angular.cu": [],
    "kernels_slab.cu": [],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmpcd.so")


def _sources():
    srcs = [os.path.join(CSRC, f) for f in UNITS]
    deps = srcs + [os.path.join(CSRC, "mpcd_internal.cuh"), os.path.join(ROOT, "include", "mpcd.h")]
    return srcs, deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    _, deps = _sources()
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", os.path.join(ROOT, "include")] + (extra or [])
    objs = []

    def one(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(OUT_DIR, name.replace(".cu", f".{os.getpid()}.o"))
        cmd = [cc, "-c", src, "-o", obj] + common + UNITS[name]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr[-6000:]}")
        if verbose and r.stderr.strip():
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([cc, "-shared", "-o", tmp] + objs + ARCH, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
