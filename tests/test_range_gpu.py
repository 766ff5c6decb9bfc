"""The FP64 family over the whole FP64 input range (through the C ABI).

The FP64 family computes in double-float (float pairs), whose exponent range
is FP32's; each call therefore scales its inputs by an exact power of two
chosen from the largest input magnitude and scales its results back.  The
series is linear in c (and the adjoint in f), paper eq. (fs) and Sec. 2 put
no normalisation on the coefficients, so the oracle's direct sum on the
same scaled inputs is the reference; the 1e-12 gate must hold at every
scale.  Scaling by a power of two is exact, so the results for c 2^k must
also be exactly 2^k times those for c.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import nfft_cpu
from paper_1605_01244_gb300 import build, workloads as wl
from tests._util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

SCALES = [-200, -110, 110, 200]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _plan(c, x, m=6, sigma=2.0):
    from paper_1605_01244_gb300 import Plan
    plan = Plan(c.shape, len(x), m=m, sigma=sigma, precision="f64")
    plan.set_points(to_dev(x))
    return plan


@pytest.mark.parametrize("k", SCALES)
def test_scaled_coefficients_eval_and_gradients(k):
    c0, x = wl.small_random()
    c = np.ldexp(c0.real, k) + 1j * np.ldexp(c0.imag, k)
    plan = _plan(c, x)
    fd, gd = oracle.forward_grad(c, x)
    assert np.all(np.isfinite(fd)) and np.max(np.abs(fd)) > 0
    f = to_np(plan.eval(to_dev(c)))
    assert rel_l2(f, fd) <= 1e-12, ("eval", k, rel_l2(f, fd))
    f2, g = plan.eval_grad(to_dev(c))
    assert rel_l2(to_np(f2), fd) <= 1e-12
    assert rel_l2(to_np(g), gd) <= 1e-11, ("eval_grad", k, rel_l2(to_np(g), gd))
    # window-derivative gradient: ten times the i k-method's error at the same m
    _, gw = plan.eval_grad_window(to_dev(c))
    assert rel_l2(to_np(gw), gd) <= 1e-10
    # exactness of the power-of-two scaling against the unscaled inputs
    f0 = to_np(plan.eval(to_dev(c0)))
    assert np.array_equal(f, np.ldexp(f0.real, k) + 1j * np.ldexp(f0.imag, k))


@pytest.mark.parametrize("k", SCALES)
def test_scaled_values_adjoint(k):
    c, x = wl.small_random()
    rng = wl.rng(31)
    f0 = rng.standard_normal(len(x)) + 1j * rng.standard_normal(len(x))
    f = np.ldexp(f0.real, k) + 1j * np.ldexp(f0.imag, k)
    plan = _plan(c, x)
    h = to_np(plan.adjoint(to_dev(f)))
    hd = oracle.adjoint(f, x, c.shape)
    assert rel_l2(h, hd) <= 5e-12, ("adjoint", k, rel_l2(h, hd))


@pytest.mark.parametrize("k", [-200, 200])
def test_scaled_coefficients_other_paths(k, monkeypatch):
    """The cuFFT path (grids that are not powers of two), the one-thread
    double-float gather and the stored-grid gathers scale the same way."""
    N = (10, 14, 18)                      # n = (20, 28, 36): the cuFFT path
    c0 = wl.gaussian_coeffs(N, 3.0, seed=33)
    c = np.ldexp(c0.real, k) + 1j * np.ldexp(c0.imag, k)
    x = wl.uniform_points(500, seed=34)
    fd = oracle.forward(c, x)
    plan = _plan(c, x, m=7)
    assert plan.n == (20, 28, 36)
    assert rel_l2(to_np(plan.eval(to_dev(c))), fd) <= 1e-12
    plan.precompute(to_dev(c))
    assert rel_l2(to_np(plan.eval_stored()), fd) <= 1e-12
    monkeypatch.setenv("GBNFFT_GATHER", "thread")
    pt = _plan(c, x, m=7)
    assert rel_l2(to_np(pt.eval(to_dev(c))), fd) <= 1e-12
    monkeypatch.setenv("GBNFFT_GATHER", "native")
    pn = _plan(c, x, m=7)
    assert rel_l2(to_np(pn.eval(to_dev(c))), fd) <= 1e-12


def test_coefficients_spanning_forty_decades():
    """|c_k| from 1e-40 to 1 (log-uniform magnitudes, random phases)."""
    N = (16, 16, 16)
    rng = wl.rng(35)
    mag = 10.0 ** (-40.0 * rng.random(N))
    c = mag * np.exp(2j * np.pi * rng.random(N))
    x = wl.uniform_points(1000, seed=36)
    # the spectrum is flat in the band, whose window error at m = 6 (2e-12,
    # the estimate of the plan's m rule) exceeds the gate: m = 7
    plan = _plan(c, x, m=7)
    fd, gd = oracle.forward_grad(c, x)
    assert rel_l2(to_np(plan.eval(to_dev(c))), fd) <= 1e-12
    _, g = plan.eval_grad(to_dev(c))
    assert rel_l2(to_np(g), gd) <= 1e-11
    # the same spread of magnitudes scaled deep below FP32's range
    cs = c * 2.0 ** -300
    fs = to_np(plan.eval(to_dev(cs)))
    assert rel_l2(fs, oracle.forward(cs, x)) <= 1e-12
    # element by element against the same approximation in numpy (FP64)
    p6 = _plan(c, x, m=6)
    f6 = to_np(p6.eval(to_dev(c)))
    ref = nfft_cpu.forward(c, x, p6.n, 6)
    assert np.max(np.abs(f6 - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_zero_and_subnormal_inputs():
    c, x = wl.small_random()
    plan = _plan(c, x)
    z = np.zeros_like(c)
    assert np.count_nonzero(to_np(plan.eval(to_dev(z)))) == 0
    # a single subnormal coefficient: the result is that mode, times 2^-1060
    zs = z.copy()
    k0 = (3, -2, 5)
    zs[tuple(k + n // 2 for k, n in zip(k0, c.shape))] = 2.0 ** -1060
    f = to_np(plan.eval(to_dev(zs)))
    expect = 2.0 ** -1060 * np.exp(2j * np.pi * (x @ np.asarray(k0, np.float64)))
    # the result is itself subnormal: compare with the absolute resolution there
    assert np.max(np.abs(f - expect)) <= 2.0 ** -1060 * 1e-9 + 2.0 ** -1074 * 4
    h = to_np(plan.adjoint(torch.zeros(len(x), dtype=torch.complex128, device="cuda")))
    assert np.count_nonzero(h) == 0
