"""Host logic of the apply programs, checked through the library itself (no GPU).

Each harness under tests/ is compiled against the library's internal header, linked with
libvie.so and run; no device memory is touched.
* validator_harness.cpp, fault injection: a valid two-stage program is accepted, and each of
  fifteen corruptions of one field (matrix offset or buffer size, leading dimension, block
  shape, input or output slice, vector space, coefficient count) is refused with VIE_EINVAL;
* tiles_harness.cpp: the warp tiling of seeded random stages, for the default and all nine
  tile-budget x vector-count candidates, covers every output row exactly once with whole
  passes of 32/g rows, within the tile budget."""
import os
import shutil
import subprocess

import pytest

import paper_2111_01730_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _run_harness(tmp_path, name):
    cxx = shutil.which("g++")
    lib64 = os.path.join(CUDA, "lib64")
    if cxx is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")) or not (
            os.path.isdir(lib64) and any(f.startswith("libcudart.so") for f in os.listdir(lib64))):
        pytest.skip("needs g++, the CUDA headers and libcudart")
    pkg.load_library()  # the library must be built (raises otherwise)
    libdir = os.path.dirname(pkg.LIB_PATH)
    exe = str(tmp_path / name)
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2111_01730_gb300", "csrc"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", name + ".cpp"), pkg.LIB_PATH,
           "-L", lib64, "-lcudart", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{lib64}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout.strip()


def test_validator_refuses_corrupted_block_descriptors(tmp_path):
    assert _run_harness(tmp_path, "validator_harness") == "ok 15"


def test_warp_tiles_cover_every_output_row_once(tmp_path):
    assert _run_harness(tmp_path, "tiles_harness") == "ok 2000"
