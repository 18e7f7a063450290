"""Builds the CUDA shared library libmdgb300.so in-tree with nvcc for sm_103a.

    python -m paper_0912_3824_gb300.build        (or build() from Python)

The translation units compile in parallel; the result is linked against the
shared CUDA runtime.  Build products live next to this file and are ignored by
git.  build(checked=True) makes libmdgb300_checked.so instead: the same library
with every index that the kernels read from device memory tested against its
array (MD_CHECK_BOUNDS; a violation is reported as MD_E_BOUNDS), for the
bounds-checked test run; load it with MDGB300_LIB=<path>.
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
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmdgb300.so")
OUT_DIR_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libmdgb300_checked.so")
SOURCES = ["md_api.cu", "md_kernels_mixed.cu", "md_kernels_fp64.cu", "md_kernels_fp32.cu", "md_noalloc.cu",
           "md_peak.cu"]
HEADERS = ["md_common.cuh", "md_kernels.cuh", "md_tables.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose_ptxas: bool = False, checked: bool = False) -> list[str]:
    f = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
         "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    if checked:
        f += ["-DMD_CHECK_BOUNDS=1"]
    return f


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + \
        [os.path.join(INCLUDE, h) for h in ("md.h", "md_bench.h")] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    """Compile (if sources changed) and return the path of libmdgb300.so
    (libmdgb300_checked.so with checked=True)."""
    lib, out_dir = (LIB_CHECKED, OUT_DIR_CHECKED) if checked else (LIB, OUT_DIR)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    objs = [os.path.join(out_dir, s.replace(".cu", ".o")) for s in SOURCES]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [cc, *_flags(verbose_ptxas, checked), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(compile_one, zip(SOURCES, objs)))
    if verbose_ptxas:
        sys.stderr.write("".join(logs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checked="--checked" in sys.argv))
