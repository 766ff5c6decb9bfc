"""Vortex-tube evaluation (the paper's sftubeeval3, Sec. 4.3).

CPU pins of the restatement (oracle/tube_ref.py) on a series whose density
is known in closed form: psi = 1 + exp(2 pi i x1) has rho = 2 - 2 cos(2 pi
(x1 + 1/2)), zero on the plane x1 = -1/2, so the kept points and their
children can be enumerated by hand.  GPU: the CUDA refinement
(nfft3_tube_refine) and the NFFT-driven tube_eval against the restatement
driven by the FP64 direct sum.
"""
import numpy as np
import pytest

import oracle
from oracle import tube_ref
from paper_1605_01244_gb300 import workloads as wl


def two_mode_coeffs(N=(4, 4, 4)):
    c = np.zeros(N, np.complex128)
    c[N[0] // 2, N[1] // 2, N[2] // 2] = 1.0        # k = 0
    c[N[0] // 2 + 1, N[1] // 2, N[2] // 2] = 1.0    # k = (1, 0, 0)
    return c


def test_density_of_the_two_mode_series_is_closed_form():
    c = two_mode_coeffs()
    x = wl.uniform_points(50, seed=3)
    rho = tube_ref.density(oracle.forward(c, x))
    assert np.max(np.abs(rho - (2 + 2 * np.cos(2 * np.pi * x[:, 0])))) <= 1e-13


def test_two_levels_by_hand():
    """R = (8, 4, 4) nodes on [-1/2, 1/2)^3 (h = 1/8, 1/4, 1/4).  rho at the
    nodes is 2 - 2 cos(pi i / 4): level 1 (rhobar 0.6) keeps i in {0, 1, 7}
    (rho 0, 2 - sqrt 2, 2 - sqrt 2): 3 x 16 parents, 27 children each.
    Level 2 (rhobar 0.1) keeps exactly the children of the i = 0 parents
    (their x1 offsets 0, +-1/24 give rho 0 and 2 - 2 cos(pi/12) = 0.068; the
    others are at least 2 - 2 cos(pi/6) = 0.27): 16 x 27 parents, 27 children."""
    c = two_mode_coeffs()
    R, lo = (8, 4, 4), (-0.5, -0.5, -0.5)
    hi = tuple(-0.5 + (r - 1) / r for r in R)
    x0, h = tube_ref.lattice(R, lo, hi)
    assert np.allclose(h, [1 / 8, 1 / 4, 1 / 4])
    psi0 = oracle.forward(c, x0)
    lvl1 = tube_ref.refine(x0, psi0, 0.6, h)
    assert lvl1.shape == (3 * 16 * 27, 3)
    # the first parent is the node (-1/2, -1/2, -1/2); its children in (a, b, c) order
    exp = np.array([[-0.5 + a / 24, -0.5 + b / 12, -0.5 + cc / 12]
                    for a in (-1, 0, 1) for b in (-1, 0, 1) for cc in (-1, 0, 1)])
    assert np.max(np.abs(lvl1[:27] - exp)) <= 1e-15
    x, rho = tube_ref.tube_eval(c, [0.6, 0.1], R, lo, hi, lambda p: oracle.forward(c, p))
    assert x.shape == (16 * 27 * 27, 3)
    d = x[:, 0] + 0.5
    d -= np.rint(d)
    assert np.max(np.abs(d)) <= 1 / 24 + 1 / 72 + 1e-15
    assert np.max(np.abs(rho - (2 - 2 * np.cos(2 * np.pi * d)))) <= 1e-13
    # a wrong child step (h instead of h / 3) or a strict inequality changes the counts
    assert tube_ref.refine(x0, psi0, 1e-20, h).shape[0] == 16 * 27   # rho = 0 (to rounding) at i = 0


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cuda_refinement_matches_restatement(prec):
    import torch
    from paper_1605_01244_gb300 import tube
    g = wl.rng(5)
    M = 3001
    x = g.uniform(-0.5, 0.5, (M, 3))
    psi = g.standard_normal(M) + 1j * g.standard_normal(M)
    cd = torch.complex128 if prec == "f64" else torch.complex64
    psi_t = torch.from_numpy(psi).to(cd).cuda()
    # the restatement on the same (rounded) values
    psi_r = psi_t.cpu().numpy().astype(np.complex128)
    h = (0.01, 0.02, 0.03)
    for rb in (0.0, 0.5, 2.0, 100.0):
        got = tube.refine(torch.from_numpy(x).cuda(), psi_t, rb, h, prec).cpu().numpy()
        ref = tube_ref.refine(x, psi_r, rb, h)
        assert got.shape == ref.shape, rb
        assert np.array_equal(got, ref), rb
    assert tube.refine(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                       psi_t[:0], 1.0, h, prec).shape == (0, 3)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_tube_eval_matches_direct_sum_restatement(prec, tol):
    """Two levels on a two-vortex snapshot (N = 16^3) in a box around the
    cores: the same points as the restatement (thresholds are away from any
    node's rho), rho within the family's accuracy."""
    import torch
    from paper_1605_01244_gb300 import tube
    N = 16
    c = wl.gpe_coeffs((N, N, N), 8.0, 0.5)
    cd = torch.complex128 if prec == "f64" else torch.complex64
    R, lo, hi = (9, 9, 9), (-0.1, -0.1, -0.1), (0.1, 0.1, 0.1)
    rhobar = [0.05, 0.02]
    x, rho = tube.tube_eval(torch.from_numpy(c).to(cd).cuda(), rhobar, R, lo, hi, prec,
                            m=6 if prec == "f64" else 4)
    xr, rr = tube_ref.tube_eval(c, rhobar, R, lo, hi, lambda p: oracle.forward(c, p))
    x = x.cpu().numpy()
    assert x.shape == xr.shape and x.shape[0] > 0
    assert np.max(np.abs(x - xr)) <= 1e-15
    assert np.max(np.abs(rho.cpu().numpy() - rr)) <= tol * max(1.0, np.max(rr))
