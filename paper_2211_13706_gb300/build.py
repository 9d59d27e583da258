"""Builds libmz.so (the C ABI of include/mz.h) in-tree for sm_103a.

Five translation units compiled in parallel, then linked with the CUDA
runtime statically. Output: paper_2211_13706_gb300/_build/libmz.so.

The debug variant, libmz_debug.so, is the same sources compiled with MZ_DEBUG:
every index a kernel takes from the niv map or a plan table is checked before
use (a failure is reported by mz_check as MZ_ERR_BOUNDS, never by a trap), and
workspaces and outputs are filled with a poison pattern before each transform.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmz.so")
LIB_DEBUG = os.path.join(OUT, "libmz_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["mz_host.cpp", "mz_plan_io.cpp", "mz_kernels.cu", "mz_build.cu", "mz_abi.cu"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, verbose_ptxas: bool, debug: bool = False) -> tuple[str, str]:
    path = os.path.join(CSRC, src)
    obj = os.path.join(OUT, src + (".dbg.o" if debug else ".o"))
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "-I", os.path.join(HERE, "..", "include"), "-c", path, "-o", obj]
    if debug:
        cmd.insert(1, "-DMZ_DEBUG")
    if verbose_ptxas and src.endswith(".cu"):
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "mz.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _link(lib: str, objs: list[str]) -> None:
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose_ptxas: bool = False, debug: bool = False, both: bool = False) -> str:
    """Builds libmz.so (libmz_debug.so with debug; both libraries at once with both) when
    a source is newer than the library, or always with force. Returns the library path
    (the release one with both)."""
    variants = [False, True] if both else [debug]
    libs = {d: (LIB_DEBUG if d else LIB) for d in variants}
    todo = [d for d in variants if force or _stale(libs[d])]
    if todo:
        os.makedirs(OUT, exist_ok=True)
        jobs = [(src, d) for d in todo for src in SOURCES]
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda j: _compile(j[0], verbose_ptxas, j[1]), jobs))
        if verbose_ptxas:
            for _, log in results:
                sys.stderr.write(log)
        for d in todo:
            _link(libs[d], [o for (src, dd), (o, _) in zip(jobs, results) if dd == d])
    return libs[variants[0]]


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, debug="--debug" in sys.argv,
                both="--both" in sys.argv))
