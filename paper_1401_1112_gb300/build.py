"""Build the sm_103a level-solve library in-tree (paper_1401_1112_gb300/_build/libats.so).

nvcc compiles each translation unit in parallel for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``) and links one shared library
against the static CUDA runtime.  No cmake, no torch extension machinery.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libats.so")
# the bounds-checked build (ATS_BOUNDS_CHECK=1): same sources, every gathered
# index range-checked on the device; made on request, not by default
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libats.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["kernels.cu", "runtime.cpp", "layout.cpp", "hierarchy.cpp", "server.cpp", "noalloc.cu", "loop.cu",
           "coef_models.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _defines(checked=False):
    # ATS_NVCC_DEFINES: optional extra -D definitions (e.g. the register caps
    # ATS_MINB_OP / ATS_MINB_UPD of the FP32 tick kernels) for tuning sweeps
    return os.environ.get("ATS_NVCC_DEFINES", "").split() + (["-DATS_BOUNDS_CHECK=1"] if checked else [])


def _flags(extra=(), checked=False):
    defines = _defines(checked)
    return [
        "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
        "-I", INCLUDE, "-I", CSRC, *defines, *extra,
    ]


def _needs_build(lib=LIB, checked=False) -> bool:
    if not os.path.exists(lib):
        return True
    stamp = lib + ".defines"
    if (open(stamp).read() if os.path.exists(stamp) else "") != " ".join(_defines(checked)):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, checked: bool = False) -> str:
    out_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    if not force and not _needs_build(lib, checked):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *_flags(extra, checked), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(lib + ".defines", "w") as f:
        f.write(" ".join(_defines(checked)))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
