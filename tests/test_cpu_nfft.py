"""The plain CPU NFFT (oracle/nfft_omp.c + scipy's FFT), the timed CPU
baseline of the method (Sec. 2.2.1), against the numpy restatement of the
same approximation (element by element, to rounding) and the FP64 direct sum
(the 1e-12 gate at m = 6), on one and on all host cores."""
import numpy as np
import pytest

import oracle
from oracle import cpu_nfft, nfft_cpu
from paper_1605_01244_gb300 import workloads as wl


def _max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("threads", [1, None])
def test_forward_matches_restatement_and_direct_sum(threads):
    c, x = wl.small_random()
    f, t = cpu_nfft.forward(c, x, (32, 32, 32), 6, threads=threads)
    assert set(t) == {"tables", "deconv", "fft", "gather"}
    assert _max_rel(f, nfft_cpu.forward(c, x, (32, 32, 32), 6)) <= 1e-13
    fd = oracle.forward(c, x)
    assert np.linalg.norm(f - fd) / np.linalg.norm(fd) <= 1e-12


@pytest.mark.parametrize("N,n,m", [((8, 12, 10), (16, 24, 20), 3), ((10, 14, 18), (20, 28, 36), 5),
                                   ((16, 16, 16), (32, 32, 32), 8)])
def test_shapes_and_cutoffs(N, n, m):
    c = wl.gaussian_coeffs(N, 1e9, seed=sum(N))
    x = wl.mixed_points(3000, 0.05, seed=m)
    f, _ = cpu_nfft.forward(c, x, n, m)
    assert _max_rel(f, nfft_cpu.forward(c, x, n, m)) <= 1e-13
    g = wl.rng(m)
    fv = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    h, t = cpu_nfft.adjoint(fv, x, N, n, m)
    assert set(t) == {"tables", "spread", "fft", "deconv"}
    assert _max_rel(h, nfft_cpu.adjoint(fv, x, N, n, m)) <= 1e-13


def test_adjoint_against_direct_sum_one_and_all_cores():
    c, x = wl.small_random()
    g = wl.rng(9)
    fv = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    hd = oracle.adjoint(fv, x, c.shape)
    for threads in (1, None):
        h, _ = cpu_nfft.adjoint(fv, x, c.shape, (32, 32, 32), 6, threads=threads)
        assert np.linalg.norm(h - hd) / np.linalg.norm(hd) <= 5e-12
    # a grid large enough for several slabs of first nodes per parity
    N, n = (32, 32, 32), (64, 64, 64)
    xc = wl.mixed_points(20000, 0.02, seed=10)
    fc = g.standard_normal(len(xc)) + 1j * g.standard_normal(len(xc))
    h1, _ = cpu_nfft.adjoint(fc, xc, N, n, 4, threads=1)
    ha, _ = cpu_nfft.adjoint(fc, xc, N, n, 4)
    assert _max_rel(ha, h1) <= 1e-13
    assert _max_rel(ha, nfft_cpu.adjoint(fc, xc, N, n, 4)) <= 1e-13
