"""Differentiation of the NFFT.

CPU: the backward formulas (dL/dc = A^H G, dL/dx = Re(conj(G) grad f)) are
pinned by torch.autograd.gradcheck on an oracle-backed Function that uses
the same formulas with the FP64 direct sums.
GPU: the product's NFFTEval (CUDA adjoint + eval_grad) against that oracle
Function on the same inputs, and against central finite differences of the
CUDA forward.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_01244_gb300 import workloads as wl


class OracleEval(torch.autograd.Function):
    """f = A(x) c with the FP64 direct sums (test infrastructure)."""

    @staticmethod
    def forward(ctx, c, x):
        ctx.save_for_backward(c, x)
        return torch.from_numpy(oracle.forward(c.detach().numpy(), x.detach().numpy()))

    @staticmethod
    def backward(ctx, G):
        c, x = ctx.saved_tensors
        Gn = G.detach().numpy()
        gc = gx = None
        if ctx.needs_input_grad[0]:
            gc = torch.from_numpy(oracle.adjoint(Gn, x.detach().numpy(), c.shape))
        if ctx.needs_input_grad[1]:
            _, d = oracle.forward_grad(c.detach().numpy(), x.detach().numpy())
            gx = torch.from_numpy((np.conj(Gn)[:, None] * d).real)
        return gc, gx


def test_backward_convention_gradcheck_cpu():
    c = torch.from_numpy(wl.gaussian_coeffs((4, 4, 6), 2.0, seed=40)).requires_grad_()
    x = torch.from_numpy(wl.uniform_points(5, seed=41)).requires_grad_()
    assert torch.autograd.gradcheck(OracleEval.apply, (c, x), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_gradcheck_catches_a_wrong_convention():
    """The same check fails if the x-gradient is taken as Re(G * grad f)."""

    class Wrong(OracleEval):
        @staticmethod
        def backward(ctx, G):
            c, x = ctx.saved_tensors
            _, d = oracle.forward_grad(c.detach().numpy(), x.detach().numpy())
            return None, torch.from_numpy((G.detach().numpy()[:, None] * d).real)

    c = torch.from_numpy(wl.gaussian_coeffs((4, 4, 6), 2.0, seed=42))
    x = torch.from_numpy(wl.uniform_points(5, seed=43)).requires_grad_()
    assert not torch.autograd.gradcheck(lambda xx: Wrong.apply(c, xx), (x,), eps=1e-6, atol=1e-7,
                                        rtol=1e-6, raise_exception=False)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,m,tol", [("f64", 6, 1e-11), ("f32", 4, 5e-6)])
def test_nfft_eval_backward_matches_oracle(prec, m, tol):
    from paper_1605_01244_gb300 import Plan
    from paper_1605_01244_gb300.autograd import NFFTEval
    N = (12, 10, 16)
    M = 500
    cd = torch.complex128 if prec == "f64" else torch.complex64
    c_np = wl.gaussian_coeffs(N, 3.0, seed=44)
    x_np = wl.mixed_points(M, 0.05, seed=45)
    g = wl.rng(46)
    G_np = g.standard_normal(M) + 1j * g.standard_normal(M)
    # oracle gradients of L = Re(sum conj(G) f)  (dL/df-bar convention: grad_output = G)
    c0 = torch.from_numpy(c_np).requires_grad_()
    x0 = torch.from_numpy(x_np).requires_grad_()
    f0 = OracleEval.apply(c0, x0)
    f0.backward(torch.from_numpy(G_np))
    # CUDA
    plan = Plan(N, M, m=m, precision=prec)
    c1 = torch.from_numpy(c_np).to(cd).cuda().requires_grad_()
    x1 = torch.from_numpy(x_np).cuda().requires_grad_()
    f1 = NFFTEval.apply(c1, x1, plan)
    f1.backward(torch.from_numpy(G_np).to(cd).cuda())
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(f1.detach().cpu().numpy(), f0.detach().numpy()) <= (1e-12 if prec == "f64" else 1e-6)
    assert rel(c1.grad.cpu().numpy(), c0.grad.numpy()) <= tol
    assert rel(x1.grad.cpu().numpy(), x0.grad.numpy()) <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_chain_x_elementwise(prec):
    """nfft3*_chain_x against Re(conj(G) d) formed on the host in FP64, on a
    ragged point count (several blocks and a tail), and M = 0."""
    from paper_1605_01244_gb300 import Plan
    cd = torch.complex128 if prec == "f64" else torch.complex64
    M = 3 * 256 * 7 + 13
    g = wl.rng(50)
    G = torch.from_numpy(g.standard_normal(M) + 1j * g.standard_normal(M)).to(cd)
    d = torch.from_numpy(g.standard_normal((M, 3)) + 1j * g.standard_normal((M, 3))).to(cd)
    plan = Plan((8, 8, 8), M, m=3, precision=prec)
    got = plan.chain_x(G.cuda(), d.cuda()).cpu().numpy()
    Gn, dn = G.numpy().astype(np.complex128), d.numpy().astype(np.complex128)
    want = Gn.real[:, None] * dn.real + Gn.imag[:, None] * dn.imag
    assert np.max(np.abs(got - want)) <= 1e-15 * np.max(np.abs(want))
    empty = Plan((8, 8, 8), 0, m=3, precision=prec)
    assert empty.chain_x(torch.empty(0, dtype=cd, device="cuda"),
                         torch.empty((0, 3), dtype=cd, device="cuda")).shape == (0, 3)


@pytest.mark.gpu
def test_nfft_eval_x_gradient_finite_differences():
    """Central differences (h = 1e-6) of L(x) = Re(sum conj(G) f(x)) on the FP64 CUDA path."""
    from paper_1605_01244_gb300 import Plan
    from paper_1605_01244_gb300.autograd import NFFTEval
    N = (16, 16, 16)
    M = 300
    c = torch.from_numpy(wl.gaussian_coeffs(N, 4.0, seed=47)).cuda()
    x = torch.from_numpy(wl.uniform_points(M, seed=48)).cuda().requires_grad_()
    G = torch.from_numpy(wl.rng(49).standard_normal(M) + 0j).cuda()
    plan = Plan(N, M, m=7, precision="f64")
    f = NFFTEval.apply(c, x, plan)
    (G.conj() * f).real.sum().backward()
    h = 1e-6
    fd = torch.zeros_like(x)
    with torch.no_grad():
        for d in range(3):
            e = torch.zeros_like(x)
            e[:, d] = h
            plan.set_points((x + e).contiguous())
            fp = plan.eval(c)
            plan.set_points((x - e).contiguous())
            fm = plan.eval(c)
            fd[:, d] = (G.conj() * (fp - fm)).real / (2 * h)
    err = float((fd - x.grad).norm() / x.grad.norm())
    assert err <= 1e-6, err


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_differentiation_workload_sampled(prec, tol):
    """N = 128^3 two-vortex coefficients, M = 2^18 uniform points: eval_grad
    on the full set, checked against the oracle gradient on 200 sampled points."""
    from paper_1605_01244_gb300 import Plan
    cd = torch.complex128 if prec == "f64" else torch.complex64
    c_np = wl.gpe_coeffs((128, 128, 128), 8.0)
    x_np = wl.uniform_points(2 ** 18, seed=50)
    plan = Plan(c_np.shape, len(x_np), m=0, eps=1e-12 if prec == "f64" else 1e-6, precision=prec)
    plan.set_points(torch.from_numpy(x_np).cuda())
    f, g = plan.eval_grad(torch.from_numpy(c_np).to(cd).cuda())
    idx = wl.rng(51).choice(len(x_np), 200, replace=False)
    fo, go = oracle.forward_grad(c_np, x_np[idx])
    gs = g.cpu().numpy()[idx].astype(np.complex128)
    fs = f.cpu().numpy()[idx].astype(np.complex128)
    assert np.linalg.norm(fs - fo) / np.linalg.norm(fo) <= (1e-12 if prec == "f64" else 1e-6)
    assert np.linalg.norm(gs - go) / np.linalg.norm(go) <= tol
