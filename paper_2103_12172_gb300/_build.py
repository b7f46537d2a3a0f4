"""In-tree build of libmdp.so for sm_103a with nvcc (no cmake, no torch extension machinery).

The translation units are compiled in parallel into ``_build/`` at the repository root and
linked into ``paper_2103_12172_gb300/libmdp.so``. Host code is compiled with
``-ffp-contract=off`` so that the floating-point comparisons that select grid sets are
plain IEEE operations on every host architecture.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libmdp.so")
LIB_CHECKED = os.path.join(PKG, "libmdp_checked.so")   # MDP_CHECKED=1: bounds-checked kernels
SOURCES = ["plan.cpp", "kernels.cu", "kernels_adj.cu", "kernels_tc.cu", "factor.cu", "qr.cu", "api.cu", "probe.cu",
           "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags():
    return ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                   "-Xcompiler", "-fcx-fortran-rules",
                   "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False, both: bool = False) -> str:
    """Compile (if needed) and return the path of libmdp.so, or of the bounds-checked
    libmdp_checked.so (checked=True: every translation unit with -DMDP_CHECKED=1). both=True
    builds the two libraries (the translation units of both in one parallel pass)."""
    variants = [False, True] if both else [checked]
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "mdp.h"))
    jobs, links = [], []
    for chk in variants:
        bdir = os.path.join(BUILD, "checked") if chk else BUILD
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in SOURCES:
            path = os.path.join(CSRC, src)
            obj = os.path.join(bdir, src + ".o")
            objs.append(obj)
            if force or _stale(obj, [path] + headers):
                jobs.append([_nvcc()] + _flags() + (["-DMDP_CHECKED=1"] if chk else []) + ["-c", path, "-o", obj])
        links.append((LIB_CHECKED if chk else LIB, objs))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    for lib, objs in links:
        if force or _stale(lib, objs):
            run([_nvcc()] + ARCH + ["-shared", "-o", lib] + objs + ["-lcudart"])
    return links[-1][0]


if __name__ == "__main__":
    print(build(force=True, verbose=True))
