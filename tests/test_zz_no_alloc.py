"""The allocation-free gradient entry point (nfft3d_eval_grad_noalloc).

Callers that cannot call cudaMalloc at evaluation time (device memory held by
another allocator's pool, or a loop that cannot take cudaMalloc's implicit
synchronisation) use this variant of nfft3d_eval_grad; its four oversampled
grids live in a fixed 16 MiB device array inside the library, set up when
the FP64 plan is created.  This file checks, through the C ABI:
* on a fresh plan, the first call and the next leave the device's free
  memory unchanged, and both give the same f and grad as nfft3d_eval_grad
  and the FP64 direct sum;
* plans too large for the array, and mixed-family plans, are refused.
It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1605_01244_gb300 import build, workloads as wl
from paper_1605_01244_gb300 import _lib
from tests._util import rel_l2

pytestmark = pytest.mark.gpu


def _max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _call(plan, c, f, g):
    return _lib.lib().nfft3d_eval_grad_noalloc(plan._h, ctypes.c_void_p(c.data_ptr()),
                                               ctypes.c_void_p(f.data_ptr() if f is not None else 0),
                                               ctypes.c_void_p(g.data_ptr()))


def test_noalloc_fresh_plan_allocates_nothing_and_matches():
    build.build()
    from paper_1605_01244_gb300 import Plan
    N = (16, 12, 20)
    M = 700
    c_np = wl.gaussian_coeffs(N, 1e9, seed=21)
    x_np = wl.mixed_points(M, 0.05, seed=22)
    c = torch.from_numpy(c_np).cuda()
    x = torch.from_numpy(x_np).cuda()
    # the spectrum is flat: m = 7 keeps the window error (3e-14) below the gate
    plan = Plan(N, M, m=7, precision="f64")
    assert plan.n == (32, 24, 40)          # 4 * 30720 complex doubles < 16 MiB
    plan.set_points(x)
    outs = [(torch.full((M,), float("nan"), dtype=torch.complex128, device="cuda"),
             torch.full((M, 3), float("nan"), dtype=torch.complex128, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for f, g in outs:                       # the first call on this plan, then a second one
        code = _call(plan, c, f, g)
        assert code == 0, _lib.error_string(code)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    fd, gd = oracle.forward_grad(c_np, x_np)
    for f, g in outs:
        assert rel_l2(f.cpu().numpy(), fd) <= 1e-12
        assert rel_l2(g.cpu().numpy(), gd) <= 1e-11
    # the allocating entry point on the same plan; the same kernels up to the
    # transform (four single FFTs against the fused transform) and the gather
    f_ref, g_ref = plan.eval_grad(c)
    for f, g in outs:
        assert _max_rel(f.cpu().numpy(), f_ref.cpu().numpy()) <= 1e-12
        assert _max_rel(g.cpu().numpy(), g_ref.cpu().numpy()) <= 1e-12


def test_noalloc_refuses_grids_beyond_its_array_and_mixed_plans():
    build.build()
    from paper_1605_01244_gb300 import Plan
    plan = Plan((64, 64, 64), 10, m=3, precision="f64")     # n = 128^3: 128 MiB of grids
    plan.set_points(torch.zeros((10, 3), dtype=torch.float64, device="cuda"))
    c = torch.zeros((64, 64, 64), dtype=torch.complex128, device="cuda")
    f = torch.empty(10, dtype=torch.complex128, device="cuda")
    g = torch.empty((10, 3), dtype=torch.complex128, device="cuda")
    assert _call(plan, c, f, g) == _lib.NFFT3_ERR_TOO_LARGE
    p32 = Plan((8, 8, 8), 10, m=3, precision="f32")
    p32.set_points(torch.zeros((10, 3), dtype=torch.float64, device="cuda"))
    c32 = torch.zeros((8, 8, 8), dtype=torch.complex64, device="cuda")
    f32 = torch.empty(10, dtype=torch.complex64, device="cuda")
    g32 = torch.empty((10, 3), dtype=torch.complex64, device="cuda")
    assert _call(p32, c32, f32, g32) == _lib.NFFT3_ERR_ARG
