"""Pins of the FP64 direct-sum oracle against facts fixed by the paper and by
mathematics (not against itself).

* single mode: c = delta_{k0} gives exp(2 pi i k0.x), checked against an
  arbitrary-precision value (the transform definition of Sec. 2.2.1);
* grid points x = -1/2 + l/N: the series equals N1N2N3 * ifftn of the
  shifted coefficients (Sec. 2.1, the ifftn evaluation; the (-1)^k factor is
  the shift of Sec. 2.2.1's coefficient mapping);
* Parseval (Sec. 2) and the gradient-energy identity (Sec. 2, after eq. (Lambda));
* linearity; the adjoint identity <A c, f> = <c, A^H f>;
* brute force in 40-digit arithmetic on tiny inputs;
* gradient: single-mode closed form and central finite differences.

Non-cubic N are used throughout so that a transposed axis or a swapped
index fails.
"""
import mpmath
import numpy as np
import pytest

import oracle
from oracle import mp_reference
from paper_1605_01244_gb300 import workloads as wl

SHAPES = [(4, 6, 8), (8, 4, 6), (6, 8, 4)]


def _mp_mode(k0, x):
    with mpmath.workdps(40):
        ph = sum(mpmath.mpf(int(k)) * mpmath.mpf(float(v)) for k, v in zip(k0, x))
        return complex(mpmath.exp(2j * mpmath.pi * ph))


@pytest.mark.parametrize("N", SHAPES + [(16, 16, 16)])
def test_single_mode_is_exact_exponential(N):
    x = wl.uniform_points(40, seed=3) * 3.0   # any real x: the series is 1-periodic
    rng = wl.rng(7)
    for _ in range(6):
        i = tuple(int(rng.integers(0, n)) for n in N)
        k0 = tuple(i[d] - N[d] // 2 for d in range(3))
        c = np.zeros(N, np.complex128)
        c[i] = 1.0
        f = oracle.forward(c, x)
        ref = np.array([_mp_mode(k0, xj) for xj in x])
        assert np.max(np.abs(f - ref)) <= 2e-15, (k0, np.max(np.abs(f - ref)))


@pytest.mark.parametrize("N", SHAPES + [(8, 8, 8)])
def test_grid_points_equal_inverse_dft(N):
    c = wl.gaussian_coeffs(N, 3.0, seed=1)
    grids = [np.arange(n) / n - 0.5 for n in N]
    X = np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1).reshape(-1, 3)
    f = oracle.forward(c, X).reshape(N)
    k1, k2, k3 = wl.freq_grid(N)
    sign = (-1.0) ** (np.abs(k1) + np.abs(k2) + np.abs(k3))
    ref = np.fft.ifftn(np.fft.ifftshift(c * sign)) * np.prod(N)
    assert np.max(np.abs(f - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", SHAPES)
def test_parseval_on_grid(N):
    c = wl.gaussian_coeffs(N, 5.0, seed=2)
    grids = [np.arange(n) / n - 0.5 for n in N]
    X = np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1).reshape(-1, 3)
    f = oracle.forward(c, X)
    lhs = np.sum(np.abs(c) ** 2)
    rhs = np.sum(np.abs(f) ** 2) / np.prod(N)
    assert abs(lhs - rhs) <= 1e-13 * lhs


def test_linearity():
    N = (6, 4, 8)
    c1 = wl.gaussian_coeffs(N, 3.0, seed=4)
    c2 = wl.gaussian_coeffs(N, 3.0, seed=5)
    x = wl.uniform_points(50, seed=6)
    al, be = 0.7 - 1.3j, -2.1 + 0.4j
    lhs = oracle.forward(al * c1 + be * c2, x)
    rhs = al * oracle.forward(c1, x) + be * oracle.forward(c2, x)
    assert np.linalg.norm(lhs - rhs) <= 1e-14 * np.linalg.norm(rhs)


@pytest.mark.parametrize("N", SHAPES)
def test_adjoint_identity(N):
    c = wl.gaussian_coeffs(N, 3.0, seed=8)
    x = wl.uniform_points(50, seed=9)
    g = wl.rng(10)
    f = g.standard_normal(50) + 1j * g.standard_normal(50)
    lhs = np.vdot(f, oracle.forward(c, x))          # <A c, f> = f^H A c
    rhs = np.vdot(oracle.adjoint(f, x, N), c)        # <c, A^H f> = (A^H f)^H c
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_adjoint_single_point_closed_form():
    N = (4, 6, 8)
    x = np.array([[0.1234, -0.377, 0.4101]])
    h = oracle.adjoint(np.array([1.0 + 0j]), x, N)
    k1, k2, k3 = wl.freq_grid(N)
    ref = np.exp(-2j * np.pi * (k1 * x[0, 0] + k2 * x[0, 1] + k3 * x[0, 2]))
    assert np.max(np.abs(h - ref)) <= 1e-14


def test_adjoint_at_selected_frequencies():
    """The sampled-frequency adjoint (one compensated sum over all points per
    k) against the separable full adjoint at every k of a small band, the
    closed form of one point at frequencies far outside any band, and a
    40-digit brute force of a few terms."""
    N = (4, 6, 8)
    x = wl.mixed_points(300, 0.05, seed=41)
    g = wl.rng(42)
    f = g.standard_normal(300) + 1j * g.standard_normal(300)
    k1, k2, k3 = wl.freq_grid(N)
    ks = np.stack(np.broadcast_arrays(k1, k2, k3), -1).reshape(-1, 3)
    h = oracle.adjoint_at(f, x, ks)
    hf = oracle.adjoint(f, x, N).reshape(-1)
    assert np.max(np.abs(h - hf)) <= 1e-13 * np.max(np.abs(hf))
    big = np.array([[1000, -37, 2 ** 20], [-(2 ** 24), 5, 0], [0, 0, 0]])
    xp = np.array([[0.1234, -0.377, 0.4101]])
    h1 = oracle.adjoint_at(np.array([1.0 + 0j]), xp, big)
    with mpmath.workdps(40):
        for q in range(3):
            ph = sum(int(big[q, d]) * mpmath.mpf(float(xp[0, d])) for d in range(3))
            ref = complex(mpmath.exp(-2j * mpmath.pi * ph))
            assert abs(h1[q] - ref) <= 1e-15
    # many equal terms: compensated summation keeps the exact multiple
    xs = np.tile(np.array([[0.25, 0.0, 0.0]]), (100000, 1))
    hs = oracle.adjoint_at(np.full(100000, 0.1 + 0j), xs, np.array([[1, 0, 0]]))
    assert abs(hs[0] - (-1j * 0.1 * 100000)) <= 1e-15 * 1e4


def test_brute_force_high_precision():
    N = (4, 4, 6)
    c = wl.gaussian_coeffs(N, 2.0, seed=11)
    x = wl.uniform_points(6, seed=12)
    f = oracle.forward(c, x)
    ref = mp_reference.forward(c, x)
    assert np.max(np.abs(f - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_gradient_single_mode():
    N = (6, 8, 4)
    k0 = (2, -4, 1)
    c = np.zeros(N, np.complex128)
    c[tuple(k + n // 2 for k, n in zip(k0, N))] = 1.0
    x = wl.uniform_points(30, seed=13)
    f, g = oracle.forward_grad(c, x)
    e = np.array([_mp_mode(k0, xj) for xj in x])
    ref = 2j * np.pi * np.asarray(k0)[None, :] * e[:, None]
    assert np.max(np.abs(g - ref)) <= 1e-13
    assert np.max(np.abs(f - e)) <= 2e-15


def test_gradient_finite_differences():
    N = (8, 6, 10)
    c = wl.gaussian_coeffs(N, 3.0, seed=14)
    x = wl.uniform_points(40, seed=15)
    _, g = oracle.forward_grad(c, x)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (oracle.forward(c, x + e) - oracle.forward(c, x - e)) / (2 * h)
        # truncation h^2 |f'''|/6 + rounding eps |f| / h
        assert np.linalg.norm(fd - g[:, d]) <= 1e-7 * np.linalg.norm(g[:, d])


@pytest.mark.parametrize("N", [(6, 8, 4), (8, 8, 8)])
def test_gradient_energy_identity(N):
    c = wl.gaussian_coeffs(N, 3.0, seed=16)
    grids = [np.arange(n) / n - 0.5 for n in N]
    X = np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1).reshape(-1, 3)
    _, g = oracle.forward_grad(c, X)
    k1, k2, k3 = wl.freq_grid(N)
    # the Nyquist mode -N/2 is differentiated as -N/2 (not symmetrised)
    lhs = np.sum(4 * np.pi ** 2 * (k1 * k1 + k2 * k2 + k3 * k3) * np.abs(c) ** 2)
    rhs = np.sum(np.abs(g) ** 2) / np.prod(N)
    assert abs(lhs - rhs) <= 1e-12 * lhs


def test_periodicity_and_empty():
    N = (4, 6, 8)
    c = wl.gaussian_coeffs(N, 3.0, seed=17)
    x = wl.uniform_points(20, seed=18)
    shift = np.array([3.0, -2.0, 1.0])
    assert np.max(np.abs(oracle.forward(c, x) - oracle.forward(c, x + shift))) <= 1e-12
    assert oracle.forward(c, np.zeros((0, 3))).shape == (0,)
    assert np.all(oracle.adjoint(np.zeros(0), np.zeros((0, 3)), N) == 0)


def test_nested_sums_accurate_at_the_benchmark_size():
    """At N = 256^3 (the precision-sweep coefficients) the oracle's nested
    per-dimension sums agree with an exactly rounded sum (math.fsum) of the
    1.7e7 individually formed terms c_k e^{2 pi i k.x} to 1e-14 of |f|: the
    plain sums are accurate enough at the largest size the tests use them."""
    import math
    N = (256, 256, 256)
    c = wl.gaussian_coeffs(N, 40.0, seed=0)
    x = np.array([[0.1234567, -0.3141592, 0.2718281], [-0.4999, 0.0021, 0.377]])
    f = oracle.forward(c, x)
    k = [np.arange(n) - n // 2 for n in N]
    for j in range(len(x)):
        e = [np.exp(2j * np.pi * ((kd * x[j, d]) - np.round(kd * x[j, d]))) for d, kd in enumerate(k)]
        terms = (c * e[0][:, None, None] * e[1][None, :, None] * e[2][None, None, :]).ravel()
        exact = complex(math.fsum(terms.real), math.fsum(terms.imag))
        assert abs(f[j] - exact) <= 1e-14 * abs(exact), (j, abs(f[j] - exact) / abs(exact))
