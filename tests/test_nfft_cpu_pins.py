"""Pins of the plain numpy NFFT restatement (oracle/nfft_cpu.py).

The paper treats the NFFT as a black box with cost O(N log N + M|log eps|^3)
(Sec. 1, Sec. 2.2.1); these tests fix the window mathematics independently:

* the Kaiser-Bessel pair: quadrature of the truncated window equals the
  closed-form I0 transform up to an O(1) absolute term (the transform of the
  oscillating tail cut off beyond |tau| = alpha), i.e. to ~1e-13 relative
  where I0 is large (the identity the deconvolution relies on);
* the approximation converges to the FP64 direct sum geometrically in m, at
  the rate exp(-2 pi sqrt(1 - 1/sigma)) per unit of m;
* the fast forward and fast adjoint are exact transposes (to rounding);
* grid nodes and half-integer u (edge taps) are handled;
* the gradient and adjoint approximate the direct gradient/adjoint.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import nfft_cpu
from paper_1605_01244_gb300 import workloads as wl


def _gauss_legendre(f, lo, hi, n=400):
    t, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
    return 0.5 * (hi - lo) * np.sum(w * f(x))


@pytest.mark.parametrize("m,sigma,N", [(6, 2.0, 16), (3, 2.0, 16), (4, 1.5, 32), (7, 2.0, 64), (3, 1.25, 64)])
def test_kaiser_bessel_pair_quadrature(m, sigma, N):
    n = int(sigma * N)
    b = nfft_cpu.kb_b(n, N)
    al = m + 0.5
    for k in range(-N // 2, N // 2 + 1):
        nu = k / n
        # the window is analytic in tau on [-alpha, alpha]: Gauss-Legendre converges fast
        q = _gauss_legendre(lambda t: nfft_cpu.kb_phi(np.minimum(t, al), m, b) * np.cos(2 * math.pi * nu * t),
                            -al, al)
        ref = nfft_cpu.kb_Phi(k, n, m, b)
        assert abs(q - ref) <= 0.1 + 1e-13 * ref, (k, q, ref)


def test_window_edges():
    m, b = 4, nfft_cpu.kb_b(32, 16)
    al = m + 0.5
    assert nfft_cpu.kb_phi(al, m, b) == pytest.approx(b / math.pi, rel=1e-15)
    assert nfft_cpu.kb_phi(-al, m, b) == 0.0
    assert nfft_cpu.kb_phi(al + 1e-9, m, b) == 0.0
    assert nfft_cpu.kb_phi(0.0, m, b) == pytest.approx(math.sinh(b * al) / (math.pi * al), rel=1e-14)


def test_converges_geometrically_in_m():
    N = (16, 12, 20)
    c = wl.gaussian_coeffs(N, 1e9, seed=0)      # flat spectrum: the worst case
    x = wl.uniform_points(300, seed=1)
    fd = oracle.forward(c, x)
    n = tuple(2 * v for v in N)
    errs = []
    for m in range(2, 7):
        f = nfft_cpu.forward(c, x, n, m)
        errs.append(np.linalg.norm(f - fd) / np.linalg.norm(fd))
    rate = math.exp(-2 * math.pi * math.sqrt(1 - 1 / 2.0))   # per unit of m at sigma = 2
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 / e0 == pytest.approx(rate, rel=0.35), errs
    assert errs[-1] < 5e-12


def test_small_random_m6_meets_fp64_gate():
    c, x = wl.small_random()
    fd = oracle.forward(c, x)
    f = nfft_cpu.forward(c, x, (32, 32, 32), 6)
    assert np.linalg.norm(f - fd) / np.linalg.norm(fd) <= 1e-12


def test_grid_nodes_and_half_integer_u():
    N = (8, 10, 6)
    n = (16, 20, 12)
    c = wl.gaussian_coeffs(N, 3.0, seed=2)
    grids = [np.arange(v) / v - 0.5 for v in n]
    X = np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1).reshape(-1, 3)
    for pts in (X, X + 0.5 / np.asarray(n)):       # t = 0 exactly, then u half-integer
        fd = oracle.forward(c, pts)
        f = nfft_cpu.forward(c, pts, n, 6)
        assert np.linalg.norm(f - fd) / np.linalg.norm(fd) <= 1e-11


def test_fast_forward_and_adjoint_are_transposes():
    N = (8, 6, 10)
    n = (16, 12, 20)
    c = wl.gaussian_coeffs(N, 1e9, seed=3)
    x = wl.uniform_points(70, seed=4)
    g = wl.rng(5)
    f = g.standard_normal(70) + 1j * g.standard_normal(70)
    for m in (2, 5):
        lhs = np.vdot(f, nfft_cpu.forward(c, x, n, m))
        rhs = np.vdot(nfft_cpu.adjoint(f, x, N, n, m), c)
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_adjoint_approximates_direct():
    N = (8, 12, 10)
    n = (16, 24, 20)
    x = wl.uniform_points(200, seed=6)
    g = wl.rng(7)
    f = g.standard_normal(200) + 1j * g.standard_normal(200)
    hd = oracle.adjoint(f, x, N)
    h = nfft_cpu.adjoint(f, x, N, n, 6)
    assert np.linalg.norm(h - hd) / np.linalg.norm(hd) <= 5e-12


def test_gradient_approximates_direct():
    N = (12, 8, 10)
    n = (24, 16, 20)
    c = wl.gaussian_coeffs(N, 3.0, seed=8)
    x = wl.uniform_points(150, seed=9)
    fd, gd = oracle.forward_grad(c, x)
    f, g = nfft_cpu.forward_grad(c, x, n, 6)
    assert np.linalg.norm(f - fd) / np.linalg.norm(fd) <= 3e-12
    for d in range(3):
        assert np.linalg.norm(g[:, d] - gd[:, d]) / np.linalg.norm(gd[:, d]) <= 1e-11


def test_window_derivative_matches_difference_quotients():
    """kb_dphi is the derivative of kb_phi: central differences (h = 1e-5,
    error ~ h^2 phi''' / 6) inside the support, including close to the ends
    where its small-argument series takes over."""
    for m, b in ((3, math.pi * 1.5), (6, math.pi * 1.5), (4, math.pi * (2 - 1 / 1.25))):
        al = m + 0.5
        tau = np.concatenate([np.linspace(-al + 1e-3, al - 1e-3, 101), [al - 1e-6, -al + 2e-6, 0.0]])
        h = 1e-7 if m == 6 else 1e-5
        fd = (nfft_cpu.kb_phi(tau + h, m, b) - nfft_cpu.kb_phi(tau - h, m, b)) / (2 * h)
        inside = (tau + h <= al) & (tau - h > -al)
        got = nfft_cpu.kb_dphi(tau, m, b)
        scale = np.max(np.abs(got))
        assert np.max(np.abs(got[inside] - fd[inside])) <= 1e-6 * scale, m
    # limit at the support end and zero at the centre
    b = math.pi * 1.5
    assert abs(nfft_cpu.kb_dphi(3.5, 3, b) - (-3.5 * b ** 3 / (3 * math.pi))) <= 1e-12 * b ** 3
    assert nfft_cpu.kb_dphi(0.0, 3, b) == 0.0


def test_window_derivative_gradient_converges_to_direct():
    """The window-derivative gradient approximates the direct gradient and
    converges geometrically in m (about one unit of m behind the i k-method);
    its value output is the plain NFFT's."""
    N = (12, 8, 10)
    n = (24, 16, 20)
    c = wl.gaussian_coeffs(N, 3.0, seed=8)
    x = wl.uniform_points(150, seed=9)
    fd, gd = oracle.forward_grad(c, x)
    errs = []
    for m in (3, 4, 5, 6, 7):
        f, g = nfft_cpu.forward_grad_window(c, x, n, m)
        assert np.array_equal(f, nfft_cpu.forward(c, x, n, m)) or \
            np.max(np.abs(f - nfft_cpu.forward(c, x, n, m))) <= 1e-13 * np.max(np.abs(f))
        errs.append(max(np.linalg.norm(g[:, d] - gd[:, d]) / np.linalg.norm(gd[:, d]) for d in range(3)))
    assert errs[-1] <= 1e-11
    rate = math.exp(-2 * math.pi * math.sqrt(1 - 1 / 2.0))
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert e1 <= 4 * rate * e0, errs
    # a sign or scale mistake in the derivative weights would not converge
    f6, g6 = nfft_cpu.forward_grad(c, x, n, 6)
    _, w7 = nfft_cpu.forward_grad_window(c, x, n, 7)
    assert np.linalg.norm(w7 - g6) / np.linalg.norm(g6) <= 1e-10
