"""Physical <-> torus mapping (paper Sec. 2.2.1): the torus series with the mapped
coefficients and points equals the paper's physical series sum psihat_k E_k(xi),
E_k(xi) = prod_d exp(2 pi i kappa_d (xi_d - a_d)/(b_d - a_d)) / sqrt(b_d - a_d),
evaluated term by term."""
import numpy as np
import torch

import oracle
from paper_1605_01244_gb300 import workloads as wl
from paper_1605_01244_gb300.mapping import gradient_to_physical, physical_to_torus


def physical_series(psihat, a, b, Xi):
    N = psihat.shape
    out = np.zeros(len(Xi), np.complex128)
    kap = [np.arange(n) - n // 2 for n in N]
    for j, xi in enumerate(Xi):
        E = [np.exp(2j * np.pi * kap[d] * (xi[d] - a[d]) / (b[d] - a[d])) / np.sqrt(b[d] - a[d]) for d in range(3)]
        out[j] = np.einsum("abc,a,b,c->", psihat, E[0], E[1], E[2])
    return out


def test_mapping_reproduces_the_physical_series():
    a, b = (-20.0, -3.0, 1.0), (60.0, 5.0, 2.5)
    psihat = wl.gaussian_coeffs((6, 8, 4), 2.0, seed=60)
    Xi = np.stack([wl.rng(61).uniform(lo, hi, 40) for lo, hi in zip(a, b)], axis=1)
    Xi[0] = [a[0], b[1] - 1e-9, a[2]]                 # edges of the box
    c, x = physical_to_torus(torch.from_numpy(psihat), a, b, torch.from_numpy(Xi))
    assert float(x.min()) >= -0.5 and float(x.max()) < 0.5
    f = oracle.forward(c.numpy(), x.numpy())
    ref = physical_series(psihat, a, b, Xi)
    assert np.max(np.abs(f - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_gradient_units():
    a, b = (0.0, -1.0, 2.0), (4.0, 1.0, 10.0)
    psihat = wl.gaussian_coeffs((6, 4, 8), 2.0, seed=62)
    Xi = np.stack([wl.rng(63).uniform(lo, hi, 20) for lo, hi in zip(a, b)], axis=1)
    c, x = physical_to_torus(torch.from_numpy(psihat), a, b, torch.from_numpy(Xi))
    _, g = oracle.forward_grad(c.numpy(), x.numpy())
    gp = gradient_to_physical(torch.from_numpy(g), a, b).numpy()
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (physical_series(psihat, a, b, Xi + e) - physical_series(psihat, a, b, Xi - e)) / (2 * h)
        assert np.linalg.norm(fd - gp[:, d]) <= 1e-6 * np.linalg.norm(gp[:, d])
