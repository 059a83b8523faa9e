"""The kernels' index arithmetic, checked on the CPU (no GPU): site_index
(own and neighbour colour-split indices, Philox site numbers) over every site
of lattices L = 4 ... 96, 128, 256 and samples of L = 1624, and the pool
kernels' multiply-shift division for every divisor they use.  The same
host/device functions the kernels call, compiled for the host by nvcc."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_index_arithmetic_on_the_host():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "index_check")
        subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1006_2566_gb300", "csrc"),
                        "-o", exe, os.path.join(ROOT, "tests", "native", "index_check.cu")], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout
