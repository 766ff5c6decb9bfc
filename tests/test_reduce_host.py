"""CPU check of set_points' fixed-point coordinate reduction: the integer
path of `reduce.cuh`, compiled for the host, against FP64 round-to-nearest
steps (exit status and counts of `tests/host/reduce_host_check.cu`).  The
GPU tests check the same path on the device (`test_reduce_gpu.py`)."""
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


def test_fixed_point_reduction_matches_fp64_steps(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "reduce_host_check")
    src = os.path.join(ROOT, "tests", "host", "reduce_host_check.cu")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-Xcompiler",
           "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(ROOT, "paper_1605_01244_gb300", "csrc"), src, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe, "300000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
    counts = dict(zip(r.stdout.split()[0::2], map(int, r.stdout.split()[1::2])))
    assert counts["mismatches"] == 0
    assert counts["fixed"] > 0.8 * counts["cases"]
