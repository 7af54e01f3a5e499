"""A plain C program (tests/c_abi/oz2_c_example.c) drives the emulated DGEMM
through include/oz2.h and liboz2.so alone: no Python, no torch on its path.
On the CPU it must compile warning-free and link against the library; on the
GPU it must run and pass its own checks (exact integer product at N = 5, the
normwise target under the bound rule, argument errors before any launch)."""
import os
import shutil
import subprocess

import pytest

from paper_2602_02549_b300.build import LIB, build

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c_abi", "oz2_c_example.c")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


def _cuda_home():
    nvcc = shutil.which("nvcc")
    if nvcc is None:
        pytest.fail("nvcc not on PATH: the CUDA toolkit is needed to build liboz2")
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _compile(out_dir):
    build()
    cuda = _cuda_home()
    exe = os.path.join(out_dir, "oz2_c_example")
    libdir = os.path.dirname(LIB)
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", INCLUDE,
           "-I", os.path.join(cuda, "include"), SRC, "-o", exe, "-L", libdir, "-loz2",
           "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lm", f"-Wl,-rpath,{libdir}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_example_compiles_and_links(tmp_path):
    exe = _compile(str(tmp_path))
    out = subprocess.run(["nm", "-u", exe], capture_output=True, text=True, check=True).stdout
    used = {line.split()[-1] for line in out.splitlines()}
    assert {"oz2_gemm", "oz2_gemm_ex", "oz2_sync", "oz2_workspace_size", "oz2_status_str"} <= used


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    exe = _compile(str(tmp_path))
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok:" in r.stdout
