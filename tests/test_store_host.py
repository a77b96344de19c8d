"""Host code of the batched and serving solvers, checked on the CPU by two
C++ harnesses compiled here and linked to libadmm.so: the device store's
range allocator against a per-cell occupancy model
(tests/range_alloc_check.cpp) and the validation and FP32 packing of an
instance (tests/stage_check.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.path.dirname(os.path.dirname(shutil.which("nvcc") or "")),
                 "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


@pytest.fixture(scope="module")
def compile_harness(tmp_path_factory):
    cxx, inc = shutil.which("g++"), _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    from paper_1903_10041_gb300 import build
    so = build.build()
    out = tmp_path_factory.mktemp("harness")

    def make(name):
        exe = out / name
        subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_1903_10041_gb300", "csrc"), "-I", inc,
                        os.path.join(ROOT, "tests", name + ".cpp"), so, "-Wl,-rpath," + os.path.dirname(so),
                        "-o", str(exe)], check=True)
        return exe
    return make


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_range_allocator_is_first_fit_and_coalesces(compile_harness, seed):
    exe = compile_harness("range_alloc_check")
    r = subprocess.run([str(exe), str(seed)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "range allocator ok" in r.stdout


def test_instance_staging_packs_and_validates(compile_harness):
    exe = compile_harness("stage_check")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "staging ok" in r.stdout
