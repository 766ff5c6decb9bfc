"""CPU check of the fused transform's division by a runtime divisor
(FastDiv, `fastdiv.cuh`): compiled for the host with nvcc, it must equal
integer division for every divisor up to 4096 and the dividends of
`tests/host/fastdiv_host_check.cu`."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return os.path.join(c, "bin", "nvcc")
    return shutil.which("nvcc")


def test_fastdiv_equals_division(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "fastdiv_host_check")
    src = os.path.join(ROOT, "tests", "host", "fastdiv_host_check.cu")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-I",
                        os.path.join(ROOT, "paper_1605_01244_gb300", "csrc"), src, "-o", exe],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
    assert r.stdout.split()[-1] == "0"
