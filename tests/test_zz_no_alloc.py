"""The allocation-free gradient entry point (nfft3d_eval_grad_noalloc).

Callers that cannot call cudaMalloc at evaluation time (device memory held by
another allocator's pool, or a loop that cannot take cudaMalloc's implicit
synchronisation) use this variant of nfft3d_eval_grad; its four oversampled
grids live in a fixed 16 MiB device array inside the library.  This file
checks, through the C ABI, that two calls in a row give the same f and grad
as nfft3d_eval_grad, and that plans too large for the array are refused.
It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1605_01244_gb300 import build, workloads as wl
from paper_1605_01244_gb300 import _lib

pytestmark = pytest.mark.gpu


def _max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_noalloc_matches_eval_grad_twice():
    build.build()
    from paper_1605_01244_gb300 import Plan
    N = (16, 12, 20)
    c = torch.from_numpy(wl.gaussian_coeffs(N, 1e9, seed=21)).cuda()
    x = torch.from_numpy(wl.mixed_points(700, 0.05, seed=22)).cuda()
    plan = Plan(N, 700, m=5, precision="f64")
    assert plan.n == (32, 24, 40)          # 4 * 30720 complex doubles < 16 MiB
    plan.set_points(x)
    f_ref, g_ref = plan.eval_grad(c)
    f_ref = f_ref.cpu().numpy()
    g_ref = g_ref.cpu().numpy()
    fn = _lib.lib().nfft3d_eval_grad_noalloc
    for _ in range(2):
        f = torch.full((700,), float("nan"), dtype=torch.complex128, device="cuda")
        g = torch.full((700, 3), float("nan"), dtype=torch.complex128, device="cuda")
        code = fn(plan._h, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                  ctypes.c_void_p(g.data_ptr()))
        assert code == 0, _lib.error_string(code)
        torch.cuda.synchronize()
        # the same kernels; four single FFTs instead of one batched FFT may round differently
        assert _max_rel(f.cpu().numpy(), f_ref) <= 1e-13
        assert _max_rel(g.cpu().numpy(), g_ref) <= 1e-13


def test_noalloc_refuses_grids_beyond_its_array():
    build.build()
    from paper_1605_01244_gb300 import Plan
    plan = Plan((64, 64, 64), 10, m=3, precision="f64")     # n = 128^3: 128 MiB of grids
    plan.set_points(torch.zeros((10, 3), dtype=torch.float64, device="cuda"))
    c = torch.zeros((64, 64, 64), dtype=torch.complex128, device="cuda")
    f = torch.empty(10, dtype=torch.complex128, device="cuda")
    g = torch.empty((10, 3), dtype=torch.complex128, device="cuda")
    code = _lib.lib().nfft3d_eval_grad_noalloc(plan._h, ctypes.c_void_p(c.data_ptr()),
                                               ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()))
    assert code == _lib.NFFT3_ERR_TOO_LARGE
