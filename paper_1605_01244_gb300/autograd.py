"""torch.autograd Function for the NFFT: f = A(x) c, differentiable in c and x.

Forward: ``nfft3*_set_points`` + ``nfft3*_eval``.
Backward, with G = dL/d(Re f) + i dL/d(Im f) (PyTorch's convention for
complex tensors):

* dL/dc = A^H G, the type-1 adjoint (``nfft3*_adjoint``): f is linear in c,
  so d(Re f_j)/d(Re c_k) = Re A_jk, d(Im f_j)/d(Re c_k) = Im A_jk, ..., which
  sums to Re/Im of sum_j conj(A_jk) G_j;
* dL/dx_{j,d} = Re(conj(G_j) d_d f_j), with d_d f_j = sum_k 2 pi i k_d c_k
  e^{2 pi i k.x_j} from ``nfft3*_eval_grad`` (paper eq. (Lambda), torus
  units), contracted with G by ``nfft3*_chain_x``.

All arithmetic is in the CUDA library; this module only sequences the calls.
"""
from __future__ import annotations

import torch

from .nfft import Plan


class NFFTEval(torch.autograd.Function):
    """``NFFTEval.apply(c, x, plan) -> f``.

    c: (N1, N2, N3) complex CUDA tensor matching ``plan`` (complex128 for an
    FP64 plan, complex64 for a mixed plan); x: (M, 3) float64 CUDA tensor;
    plan: a :class:`Plan` of the same N and M (its points are reset from x in
    forward and again in backward, so one plan may serve several calls).
    """

    @staticmethod
    def forward(ctx, c: torch.Tensor, x: torch.Tensor, plan: Plan) -> torch.Tensor:
        c = c.detach().contiguous()
        x = x.detach().contiguous()
        plan.set_points(x)
        f = plan.eval(c)
        ctx.save_for_backward(c, x)
        ctx.plan = plan
        return f

    @staticmethod
    def backward(ctx, grad_f: torch.Tensor):
        c, x = ctx.saved_tensors
        plan: Plan = ctx.plan
        G = grad_f.detach().to(plan.cdtype).contiguous()
        plan.set_points(x)
        grad_c = grad_x = None
        if ctx.needs_input_grad[0]:
            grad_c = plan.adjoint(G)
        if ctx.needs_input_grad[1]:
            _, d = plan.eval_grad(c, want_f=False)          # d[j, dim] = d f_j / d x_dim
            grad_x = plan.chain_x(G, d)                      # Re(conj(G_j) d[j, dim])
        return grad_c, grad_x, None


def nfft_eval(c: torch.Tensor, x: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable f = A(x) c (see :class:`NFFTEval`)."""
    return NFFTEval.apply(c, x, plan)
