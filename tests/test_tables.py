"""The chunk tables of the force and step kernels (host logic of
csrc/md_tables.h), checked on the CPU by a small C++ program."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_0912_3824_gb300", "csrc")


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "vector_types.h")):
            return os.path.join(cand, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "vector_types.h")):
            return inc
    return None


def test_chunk_tables(tmp_path):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("g++ or the CUDA headers not found")
    exe = tmp_path / "tables_unit"
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", inc, os.path.join(HERE, "tables_unit.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout
