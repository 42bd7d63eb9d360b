"""Device helpers of the CUDA library compiled as plain host C++ (CPU only):
  * the scalar ones (the thread -> edge binary search of Algorithm 3, the chunk-index
    and tile-descriptor writers, the packed append counter) against the C++ standard
    library on random and adversarial degree sequences (tests/host_units/device_helpers.cpp);
  * the warp- and block-collective ones (warp and block scans, the warp-cooperative
    descriptor writers for hub rows) on a small SIMT emulator, one OS thread per GPU thread,
    against the standard library and the scalar writers (tests/host_units/warp_helpers.cpp);
  * the two block-level passes that rebuild an ordered wave level's frontier in vertex order
    (over the 64-bit root masks, over the byte marks) on the same emulator, against the
    marked set, the degree scan and the binary search of Algorithm 3 written out in the
    test (tests/host_units/batch_order.cpp);
  * the warp and CTA appends of a wave's next frontier (batch_warp_flush, batch_flush) on the
    emulator, several flushes on top of an earlier reservation: contiguous in-order ranges,
    the degree scan carried on, column bases and tile descriptors
    (tests/host_units/batch_append.cpp);
  * where a batched wave's claims go (record_claim: at once, event slot, dense row, overflow
    list), on one thread and on racing emulated threads: every claimed (root, vertex) pair
    found exactly once with its parent and level (tests/host_units/claim_records.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.mark.parametrize("unit,prelude", [("device_helpers", "cuda_shim.h"), ("warp_helpers", "simt_emu.h"),
                                          ("batch_order", "simt_emu.h"), ("batch_append", "simt_emu.h"),
                                          ("claim_records", "simt_emu.h")])
def test_device_helpers_on_host(tmp_path, unit, prelude):
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / unit
    units = os.path.join(ROOT, "tests", "host_units")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-x", "c++", "-I", CUDA_INC,
                    "-I", os.path.join(ROOT, "paper_1408_1605_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-include", os.path.join(units, prelude), os.path.join(units, unit + ".cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout[-2000:]
