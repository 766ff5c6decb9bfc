"""Vortex-core Newton locator.

Pins: the two-vortex ansatz psi = exp(-|x|^2/18)((x1 - a) + i x2)((x1 + a) - i x3)/(1 + |x|^2)
vanishes on the lines {x1 = a, x2 = 0} and {x1 = -a, x3 = 0}; with a on a
grid node its interpolating series vanishes there exactly (rounding level),
so converged points must lie on those lines.  The CUDA iteration is also
compared with the same iteration run on the FP64 oracle (CPU), and every
converged point is re-evaluated with the direct sum.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_01244_gb300 import workloads as wl

L = 8.0
A = 0.5


def line_distance(p):
    """Distance (torus units) from torus points p to the nearer analytic core line."""
    a = A / (2 * L)
    d1 = np.hypot(p[:, 0] - a, p[:, 1])
    d2 = np.hypot(p[:, 0] + a, p[:, 2])
    return np.minimum(d1, d2)


def seeds_near_lines(n, spread, seed):
    g = wl.rng(seed)
    t = g.uniform(-1.5, 1.5, n) / (2 * L)
    off = g.normal(0, spread, (n, 2))
    a = A / (2 * L)
    half = n // 2
    s1 = np.stack([a + off[:half, 0], off[:half, 1], t[:half]], 1)
    s2 = np.stack([-a + off[half:, 0], t[half:], off[half:, 1]], 1)
    return np.concatenate([s1, s2])


def oracle_newton(c, seeds, tol, max_iter, max_step):
    """The same minimum-norm Gauss-Newton iteration on the FP64 direct sums."""
    x = seeds.copy()
    status = np.zeros(len(x), int)
    for _ in range(max_iter):
        act = np.where(status == 0)[0]
        if len(act) == 0:
            break
        f, g = oracle.forward_grad(c, x[act])
        for i, j in enumerate(act):
            F = np.array([f[i].real, f[i].imag])
            if np.hypot(*F) < tol:
                status[j] = 1
                continue
            J = np.stack([g[i].real, g[i].imag])
            JJ = J @ J.T
            det = np.linalg.det(JJ)
            if not det > 1e-30 * (np.trace(JJ) ** 2):
                status[j] = 2
                continue
            dx = -J.T @ np.linalg.solve(JJ, F)
            if not np.linalg.norm(dx) <= max_step:
                status[j] = 3
                continue
            x[j] += dx
    return x, status


def test_oracle_newton_lands_on_the_analytic_lines():
    c = wl.gpe_coeffs((32, 32, 32), L, A)
    seeds = seeds_near_lines(16, 0.003, seed=70)
    x, status = oracle_newton(c, seeds, 1e-10, 30, 2.0 / 32)
    ok = status == 1
    assert ok.mean() >= 0.9
    assert np.max(line_distance(x[ok])) <= 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("gradient", ["window", "series"])
@pytest.mark.parametrize("prec,tol,dist", [("f64", 1e-10, 1e-9), ("f32", 1e-5, 1e-5)])
def test_cuda_newton_finds_the_cores(prec, tol, dist, gradient):
    from paper_1605_01244_gb300 import Plan
    from paper_1605_01244_gb300.newton import CONVERGED, dedupe, locate
    N = 64
    c = wl.gpe_coeffs((N, N, N), L, A)
    seeds = seeds_near_lines(4096, 0.004, seed=71)
    plan = Plan((N, N, N), len(seeds), m=0, eps=1e-12 if prec == "f64" else 1e-6, precision=prec)
    cd = torch.complex128 if prec == "f64" else torch.complex64
    res = locate(plan, torch.from_numpy(c).to(cd).cuda(), torch.from_numpy(seeds).cuda(), tol=tol,
                 gradient=gradient)
    x = res.x.cpu().numpy()
    st = res.status.cpu().numpy()
    ok = st == CONVERGED
    assert ok.mean() >= 0.95, np.bincount(st)
    assert np.max(line_distance(x[ok])) <= dist
    # independent check of |psi| at the converged points with the direct sum
    sub = np.where(ok)[0][:300]
    assert np.max(np.abs(oracle.forward(c, x[sub]))) <= (1e-9 if prec == "f64" else 1e-4)
    # merge points closer than one coarse cell / 4
    keep = dedupe(res.x, res.status, 0.25 / N).cpu().numpy()
    assert keep.sum() >= 1 and keep.sum() <= ok.sum()
    kept = x[keep]
    dd = kept[:, None, :] - kept[None, :, :]
    dd -= np.rint(dd)
    dist2 = (dd ** 2).sum(-1) + np.eye(len(kept))
    assert dist2.min() > (0.25 / N) ** 2


@pytest.mark.gpu
def test_cuda_newton_matches_oracle_iteration():
    from paper_1605_01244_gb300 import Plan
    from paper_1605_01244_gb300.newton import locate
    N = 32
    c = wl.gpe_coeffs((N, N, N), L, A)
    seeds = seeds_near_lines(24, 0.003, seed=72)
    plan = Plan((N, N, N), len(seeds), m=7, precision="f64")
    xo, so = oracle_newton(c, seeds, 1e-10, 30, 2.0 / N)
    for gradient in ("series", "window"):
        res = locate(plan, torch.from_numpy(c).cuda(), torch.from_numpy(seeds).cuda(), tol=1e-10,
                     max_step=2.0 / N, gradient=gradient)
        st = res.status.cpu().numpy()
        both = (st == 1) & (so == 1)
        assert both.mean() >= 0.9, gradient
        assert np.max(np.abs(res.x.cpu().numpy()[both] - xo[both])) <= 1e-9, gradient
