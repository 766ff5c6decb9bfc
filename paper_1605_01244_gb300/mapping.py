"""Physical domain <-> torus mapping of the paper's Fourier series (Sec. 2.2.1).

The paper writes the series on Omega = prod_d [a_d, b_d) with basis
E_k(xi) = prod_d exp(2 pi i kappa_d (xi_d - a_d)/(b_d - a_d)) / sqrt(b_d - a_d),
kappa_d = k_d - 1 - N_d/2 (1-based k_d), i.e. kappa_d in [-N_d/2, N_d/2).
With x_d = mod((xi_d - a_d)/(b_d - a_d), 1) - 1/2 in [-1/2, 1/2),
exp(2 pi i kappa (x + 1/2)) = (-1)^kappa exp(2 pi i kappa x), so

    psi(xi) = sum_k c_k exp(2 pi i kappa.x),   c_k = psihat_k (-1)^{sum kappa_d} / prod_d sqrt(b_d - a_d),

which is the torus series the library evaluates (the paper's NFFT mapping,
written for the + sign).  Derivatives: d/dxi_d = d/dx_d / (b_d - a_d).

These are elementwise input preparations (torch ops on the caller's device);
they are not steps of the transform.
"""
from __future__ import annotations

import torch


def torus_coefficients(psihat: torch.Tensor, a, b) -> torch.Tensor:
    """c_k = psihat_k (-1)^{kappa_1+kappa_2+kappa_3} / prod_d sqrt(b_d - a_d)."""
    N = psihat.shape
    dev = psihat.device
    scale = 1.0
    sign = torch.ones((), dtype=torch.float64, device=dev)
    for d in range(3):
        L = float(b[d]) - float(a[d])
        if not L > 0:
            raise ValueError("b_d must exceed a_d")
        scale /= L ** 0.5
        kappa = torch.arange(N[d], device=dev) - N[d] // 2
        s = 1.0 - 2.0 * (kappa.abs() % 2).to(torch.float64)
        shape = [1, 1, 1]
        shape[d] = N[d]
        sign = sign * s.reshape(shape)
    return (psihat * (sign * scale).to(psihat.dtype)).contiguous()


def torus_points(xi: torch.Tensor, a, b) -> torch.Tensor:
    """x_d = mod((xi_d - a_d)/(b_d - a_d), 1) - 1/2 (float64, shape (M, 3))."""
    xi = xi.to(torch.float64)
    lo = torch.tensor([float(v) for v in a], dtype=torch.float64, device=xi.device)
    hi = torch.tensor([float(v) for v in b], dtype=torch.float64, device=xi.device)
    y = (xi - lo) / (hi - lo)
    return (y - torch.floor(y) - 0.5).contiguous()


def physical_to_torus(psihat: torch.Tensor, a, b, Xi: torch.Tensor):
    """(c, x) for evaluating the physical series psihat at the physical points Xi (M, 3)."""
    return torus_coefficients(psihat, a, b), torus_points(Xi, a, b)


def gradient_to_physical(grad: torch.Tensor, a, b) -> torch.Tensor:
    """Torus-unit gradient (M, 3) -> physical-unit gradient: divide column d by b_d - a_d."""
    L = torch.tensor([float(bb) - float(aa) for aa, bb in zip(a, b)], dtype=torch.float64,
                     device=grad.device)
    return grad / L.to(grad.real.dtype if grad.is_complex() else grad.dtype)
