"""Build libsmg.so in-tree with nvcc for sm_103a (GB300).

Every translation unit is compiled in parallel (the plane-relaxation unit once per x-line
chunk size K), then linked into ``paper_1212_6680_gb300/libsmg.so``.  No cmake.
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
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libsmg.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
KS = (1, 2, 3, 4, 6, 8, 16)
SOURCES = ["api.cpp", "hierarchy.cpp", "cycle.cu", "krylov_kernels.cu", "lobpcg.cu", "noalloc.cu", "batched.cu", "net.cu",
           "net_api.cpp", "conv_tc.cu", "gram_tc.cu"]
WKS = (8, 16)  # rows per lane of the wide-line kernel's segments (plane_wide.cu, one unit each)


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include")]


def _units():
    units = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, os.path.splitext(s)[0] + ".o")
        lang = ["-x", "cu"] if s.endswith(".cu") else ["-x", "c++"]
        units.append((src, obj, lang, []))
    for w in WKS:
        units.append((os.path.join(CSRC, "plane_wide.cu"), os.path.join(BUILD, f"plane_wide_w{w}.o"), ["-x", "cu"],
                      [f"-DSMG_WK={w}"]))
    for k in (1, 2, 3, 4):
        src = os.path.join(CSRC, "batched_inst.cu")
        units.append((src, os.path.join(BUILD, f"batched_k{k}.o"), ["-x", "cu"], [f"-DSMG_K={k}"]))
    for k in KS:
        for prec in (0, 1, 2):
            src = os.path.join(CSRC, "plane_relax_inst.cu")
            obj = os.path.join(BUILD, f"plane_relax_k{k}_p{prec}.o")
            units.append((src, obj, ["-x", "cu"], [f"-DSMG_K={k}", f"-DSMG_PREC={prec}"]))
    return units


def _deps_mtime():
    t = 0.0
    for f in os.listdir(CSRC):
        t = max(t, os.path.getmtime(os.path.join(CSRC, f)))
    t = max(t, os.path.getmtime(os.path.join(ROOT, "include", "smg.h")))
    return t


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link libsmg.so; returns its path.  Skips work when the library is newer
    than every source (set force=True to rebuild)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = _flags()
    deps = _deps_mtime()

    def compile_one(u):
        src, obj, lang, extra = u
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= deps:
            return obj, ""
        cmd = [cc] + lang + flags + extra + ["-c", src, "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)} {' '.join(extra)}:\n{p.stderr}")
        return obj, p.stderr

    units = _units()
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(units), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, units))
    if verbose:
        for obj, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [r[0] for r in results] + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
