"""The scalar device helpers of the CUDA library (the thread -> edge binary search of
Algorithm 3 line 2, the chunk-index / tile-descriptor writers, the packed append counter)
compiled as plain host C++ and checked against the C++ standard library on random and
adversarial degree sequences (CPU only; see tests/host_units/device_helpers.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def test_device_helpers_on_host(tmp_path):
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "device_helpers"
    units = os.path.join(ROOT, "tests", "host_units")
    subprocess.run([cxx, "-std=c++17", "-O1", "-x", "c++", "-I", CUDA_INC,
                    "-I", os.path.join(ROOT, "paper_1408_1605_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-include", os.path.join(units, "cuda_shim.h"), os.path.join(units, "device_helpers.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout[-2000:]
