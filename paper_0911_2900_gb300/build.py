"""Builds libfastgb.so in-tree with nvcc for sm_103a (GB300).

Every translation unit is compiled in parallel (one nvcc per file, one
-gencode), then linked into ``paper_0911_2900_gb300/lib/libfastgb.so``.  The
build is skipped when the library is newer than every source and header.
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
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libfastgb.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libfastgb_checked.so")  # debug build: index checks
OBJ_DIR = os.path.join(HERE, "_build")

SOURCES = ["plan.cu", "plan_v1.cu", "plan_v2.cu", "plan_v3.cu", "plan_v4.cu", "plan_v5.cu",
           "move.cu", "aux.cu", "noalloc.cu", "api.cpp", "floor_field.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
             if f.endswith((".cu", ".cuh", ".cpp", ".h"))]
    files.append(os.path.join(INCLUDE, "fastgb.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          checked: bool = False) -> str:
    """Builds the release library, or with checked=True the debug build in
    which kernels check the indices they derive from data (FASTGB_CHECKED)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    nvcc = _nvcc()
    obj_dir = OBJ_DIR + ("_checked" if checked else "")
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    # host code: no fused multiply-add contraction (the exact floor field's
    # doubles are fl(a + fl(b * sqrt2)) on every host, x86 and Arm alike)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]
    if checked:
        common.append("-DFASTGB_CHECKED")

    def compile_one(src):
        obj = os.path.join(obj_dir, src + ".o")
        path = os.path.join(CSRC, src)
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, *common, "-rdc=false", "-c", path, "-o", obj]
            if ptxas_v:
                cmd += ["-Xptxas", "-v"]
        else:
            cmd = [nvcc, *common, "-x", "c++", "-c", path, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_v:
        for obj, log in results:
            if log.strip():
                print(f"== {os.path.basename(obj)}\n{log}", file=sys.stderr)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv)
    print(LIB)
