"""Compile libnursd for sm_103a in-tree (no cmake): one nvcc per .cu in parallel, then link.

The shared library lands at ``paper_2501_05244_gb300/_lib/libnursd.so``;
objects go to ``paper_2501_05244_gb300/_build/``.  Both are git-ignored.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libnursd.so")
LIB_CHECKED = os.path.join(LIBDIR, "libnursd_checked.so")  # -DNURSD_CHECKED: bounds checks into the status word
SOURCES = ["api.cu", "fft.cu", "fft_reg.cu", "temporal_tc.cu", "temporal_umma.cu", "points.cu", "spread.cu", "contract.cu", "contract_umma.cu", "contract_tc.cu", "gtf.cu", "interp.cu", "illum.cu", "srsd_interp.cu", "resample.cu", "nursd3d.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnursd")


def _deps_mtime() -> float:
    paths = ([os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
             + [os.path.abspath(__file__)])
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    """Build (if stale) and return the path of libnursd.so, or of libnursd_checked.so when `checked`
    (every data-dependent index check compiled in, failures reported through the status word)."""
    lib = LIB_CHECKED if checked else LIB
    build_dir = os.path.join(BUILD, "checked") if checked else BUILD
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(build_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = nvcc_path()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DNURSD_CHECKED"] if checked else [])

    def compile_one(src: str):
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(SRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
