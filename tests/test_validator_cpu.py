"""Fault injection on the host: corrupted block descriptors of an apply program are refused.

Compiles tests/validator_harness.cpp against the library's internal header, links libvie.so
and runs it: a valid two-stage program is accepted, and each of fifteen corruptions of one
field (matrix offset or buffer size, leading dimension, block shape, input or output slice,
vector space, coefficient count) is refused with VIE_EINVAL.  No device memory is touched."""
import os
import shutil
import subprocess

import pytest

import paper_2111_01730_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_validator_refuses_corrupted_block_descriptors(tmp_path):
    cxx = shutil.which("g++")
    lib64 = os.path.join(CUDA, "lib64")
    if cxx is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")) or not (
            os.path.isdir(lib64) and any(f.startswith("libcudart.so") for f in os.listdir(lib64))):
        pytest.skip("needs g++, the CUDA headers and libcudart")
    pkg.load_library()  # the library must be built (raises otherwise)
    libdir = os.path.dirname(pkg.LIB_PATH)
    exe = str(tmp_path / "validator_harness")
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2111_01730_gb300", "csrc"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "validator_harness.cpp"), pkg.LIB_PATH,
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", f"-Wl,-rpath,{libdir}",
           f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok 15", r.stdout + r.stderr
