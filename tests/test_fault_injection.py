"""Failure detection without a GPU fault: host-side fault injection
(GBNFFT_FAULT=alloc | fft_plan makes the plan's allocation / cuFFT-plan
wrapper fail) and argument errors surface as status codes, never as crashes.
The alloc fault is taken before any device allocation, so it runs on CPU."""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import ctypes, sys
sys.path.insert(0, %r)
from paper_1605_01244_gb300 import _lib, build
build.build()
lib = _lib.lib()
h = ctypes.c_void_p()
code = lib.nfft3d_plan(ctypes.byref(h), 8, 8, 8, 10, 4, 2.0, 0.0, None)
print(code, int(bool(h.value)))
'''


def _run(env_value):
    env = dict(os.environ)
    env["GBNFFT_FAULT"] = env_value
    r = subprocess.run([sys.executable, "-c", SCRIPT % ROOT], capture_output=True, text=True, env=env,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    code, has = r.stdout.split()
    return int(code), int(has)


def test_injected_allocation_failure_returns_err_alloc():
    from paper_1605_01244_gb300 import _lib
    code, has = _run("alloc")
    assert code == _lib.NFFT3_ERR_ALLOC and has == 0


@pytest.mark.gpu
def test_injected_fft_plan_failure_returns_err_cufft():
    from paper_1605_01244_gb300 import _lib
    code, has = _run("fft_plan")
    assert code == _lib.NFFT3_ERR_CUFFT and has == 0


@pytest.mark.gpu
def test_plan_survives_bad_calls():
    """Bad arguments and a failed set_points leave the plan usable."""
    import numpy as np
    import torch
    import oracle
    from paper_1605_01244_gb300 import Plan, workloads as wl
    from paper_1605_01244_gb300._lib import NFFTError
    plan = Plan((8, 8, 8), 50, m=5)
    with pytest.raises(TypeError):
        plan.eval(torch.zeros((8, 8, 8), dtype=torch.complex64, device="cuda"))
    x = wl.uniform_points(50, seed=3)
    bad = x.copy()
    bad[7, 1] = np.inf
    with pytest.raises(NFFTError):
        plan.set_points(torch.from_numpy(bad).cuda())
    plan.set_points(torch.from_numpy(x).cuda())
    c = wl.gaussian_coeffs((8, 8, 8), 3.0, seed=4)
    f = plan.eval(torch.from_numpy(c).cuda()).cpu().numpy()
    fd = oracle.forward(c, x)
    assert np.linalg.norm(f - fd) / np.linalg.norm(fd) <= 1e-9   # m = 5 window error


@pytest.mark.gpu
def test_tile_staged_gather_bounded_wait_reports_error(monkeypatch):
    """The tile-staged gather's mbarrier waits are bounded.  With the first
    wait's limit set to zero polls (GBNFFT_TMA_FIRST_WAIT=0) every block gives
    up at once: it records the error bit, waits (bounded) for the copies it
    issued, and returns; nfft3_sync reports NFFT3_ERR_CUDA and the context
    stays usable for the next plan."""
    import numpy as np
    import torch
    import oracle
    from paper_1605_01244_gb300 import Plan, workloads as wl
    from paper_1605_01244_gb300._lib import NFFTError, NFFT3_ERR_CUDA
    c = wl.gaussian_coeffs((16, 16, 16), 4.0, seed=5)
    x = wl.mixed_points(3000, 0.05, seed=6)
    monkeypatch.setenv("GBNFFT_GATHER", "tma")
    monkeypatch.setenv("GBNFFT_TMA_FIRST_WAIT", "0")
    plan = Plan((16, 16, 16), len(x), m=3, precision="f32")
    plan.set_points(torch.from_numpy(x).cuda())
    plan.eval(torch.from_numpy(c).to(torch.complex64).cuda())
    with pytest.raises(NFFTError) as e:
        plan.sync()
    assert e.value.code == NFFT3_ERR_CUDA
    plan.close()
    monkeypatch.delenv("GBNFFT_TMA_FIRST_WAIT")
    p2 = Plan((16, 16, 16), len(x), m=3, precision="f32")
    p2.set_points(torch.from_numpy(x).cuda())
    f = p2.eval(torch.from_numpy(c).to(torch.complex64).cuda()).cpu().numpy().astype(np.complex128)
    p2.sync()
    fd = oracle.forward(c, x)
    assert np.linalg.norm(f - fd) / np.linalg.norm(fd) <= 2e-6
