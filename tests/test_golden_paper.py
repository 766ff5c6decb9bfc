"""Pins from the errors the paper prints (tests/golden/paper_grid_errors.txt).

The paper checks its direct evaluations at the 64^3 regular grid against the
inverse FFT (Sec. 2.1) and finds infinity-norm differences of about 1e-13 for
64^3 random complex coefficients: rounding-level agreement, a few units in the
last place of values of order 10^2..10^3.  Reading: coefficients with real and
imaginary parts of unit size (standard normal here), and the printed values
as the FP64 rounding level of the experiment, i.e. a relative bound
error_inf / max|f| <= max printed value / 100 (~1e-15) -- the size the
printed numbers take on values of order 100.

The oracle's direct sum at (a sample of) the same grid must agree with numpy's
inverse FFT to that level; any index, sign or ordering mistake gives O(1)
differences.  The fast CPU NFFT at m = 8 (the largest window compiled in) must
come within the window-error bound of the same grid values.
"""
import os

import numpy as np

import oracle
from oracle import nfft_cpu

HERE = os.path.dirname(os.path.abspath(__file__))


def printed_errors():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_grid_errors.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if len(line) == 3:
                out[(line[0], line[1])] = float(line[2])
    return out


def grid_experiment(seed=1605):
    N = (64, 64, 64)
    g = np.random.default_rng(seed)
    c = g.standard_normal(N) + 1j * g.standard_normal(N)
    k = [np.arange(n) - n // 2 for n in N]
    sign = (-1.0) ** (k[0][:, None, None] + k[1][None, :, None] + k[2][None, None, :])
    ref = np.fft.ifftn(np.fft.ifftshift(c * sign)) * np.prod(N)
    nodes = np.stack(np.meshgrid(*[np.arange(v) / v - 0.5 for v in N], indexing="ij"), -1).reshape(-1, 3)
    return c, nodes, ref.reshape(-1), g


def test_fixture_has_the_printed_values():
    e = printed_errors()
    assert len(e) == 8
    assert e[("grid64_ndcovlt_vs_ifft", "matlab")] == 1.0725e-13
    assert all(1e-14 < v < 1e-12 for v in e.values())


def test_oracle_direct_sum_at_the_64cubed_grid():
    bound_rel = max(printed_errors().values()) / 100.0
    c, nodes, ref, g = grid_experiment()
    idx = g.choice(len(nodes), 2048, replace=False)
    f = oracle.forward(c, nodes[idx])
    err = np.max(np.abs(f - ref[idx]))
    assert err <= bound_rel * np.max(np.abs(ref)), (err, bound_rel * np.max(np.abs(ref)))


def test_cpu_nfft_at_the_64cubed_grid():
    """NFFT at the whole 64^3 grid vs the inverse FFT: the approximation error
    of a window whose relative aliasing/truncation error is E is at most
    E sum_k |c_k| at every point; E = 8 exp(-2 pi sqrt(1 - 1/sigma)(m + 1/2))
    (about 3e-16 at m = 8, sigma = 2)."""
    c, nodes, ref, _ = grid_experiment()
    f = nfft_cpu.forward(c, nodes, (128, 128, 128), 8)
    est = 8 * np.exp(-2 * np.pi * np.sqrt(0.5) * 8.5)
    err = np.max(np.abs(f - ref))
    assert err <= est * np.sum(np.abs(c)), (err, est * np.sum(np.abs(c)))
