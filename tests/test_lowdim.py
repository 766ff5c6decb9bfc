"""One- and two-dimensional NFFT (the paper's infft / infft2).

CPU pins of the restatements in oracle/nfft_cpu.py: the direct sum against a
single mode's closed form and against numpy's inverse FFT on the grid; the
NFFT restatement converging geometrically in m to the direct sum.  GPU:
nfft_lowdim_eval element-wise against the restatement and against the direct
sum at the FP64 gate."""
import math

import numpy as np
import pytest

from oracle import nfft_cpu
from paper_1605_01244_gb300 import workloads as wl
from tests._util import rel_l2


def coeffs(shape, seed):
    g = wl.rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def test_direct_single_mode_and_grid():
    g = wl.rng(1)
    x = g.uniform(-3, 3, (40, 2))
    c = np.zeros((6, 8), np.complex128)
    c[1, 6] = 1.0                                   # k = (-2, 2)
    f = nfft_cpu.direct_lowdim(c, x)
    assert np.max(np.abs(f - np.exp(2j * np.pi * (-2 * x[:, 0] + 2 * x[:, 1])))) <= 1e-14
    for N in (8, (6, 10)):
        c = coeffs(N, 2)
        Ns = c.shape
        grids = [np.arange(n) / n - 0.5 for n in Ns]
        X = np.stack(np.meshgrid(*grids, indexing="ij"), -1).reshape(-1, len(Ns))
        k = np.meshgrid(*[np.arange(n) - n // 2 for n in Ns], indexing="ij")
        sign = (-1.0) ** sum(np.abs(kk) for kk in k)
        ref = np.fft.ifftn(np.fft.ifftshift(c * sign)) * np.prod(Ns)
        assert np.max(np.abs(nfft_cpu.direct_lowdim(c, X) - ref.reshape(-1))) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(64,), (24, 18)])
def test_restatement_converges_to_direct(shape):
    c = coeffs(shape, 3)
    dim = len(shape)
    x = wl.rng(4).uniform(-0.5, 0.5, (300, dim))
    fd = nfft_cpu.direct_lowdim(c, x)
    n = tuple(2 * v for v in shape)
    errs = [rel_l2(nfft_cpu.forward_lowdim(c, x, n, m), fd) for m in (2, 3, 4, 5, 6)]
    rate = math.exp(-2 * math.pi * math.sqrt(0.5))
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert e1 <= 4 * rate * e0, errs
    assert errs[-1] <= 3e-12       # flat random spectrum: about 1e-12 at m = 6


@pytest.mark.gpu
@pytest.mark.parametrize("shape,sigma", [((64,), 2.0), ((4096,), 2.0), ((30,), 1.5), ((24, 18), 2.0),
                                         ((64, 64), 2.0), ((10, 14), 1.5)])
def test_gpu_lowdim_matches_restatement_and_direct(shape, sigma):
    import torch
    from paper_1605_01244_gb300.lowdim import nfft_eval
    c = coeffs(shape, 5)
    dim = len(shape)
    x = np.concatenate([wl.rng(6).uniform(-0.5, 0.5, (700, dim)), wl.rng(7).uniform(-4, 4, (300, dim)),
                        np.full((1, dim), -0.5), np.full((1, dim), 0.5)])
    m = 6
    f = nfft_eval(torch.from_numpy(c).cuda(), torch.from_numpy(x).cuda(), m=m, sigma=sigma).cpu().numpy()
    n = tuple(int(v) for v in [nfft_cpu_n(v, sigma) for v in shape])
    fr = nfft_cpu.forward_lowdim(c, x, n, m)
    assert np.max(np.abs(f - fr)) <= 1e-13 * np.max(np.abs(fr))
    assert rel_l2(f, nfft_cpu.direct_lowdim(c, x)) <= (3e-12 if sigma == 2.0 else 1e-10)


def nfft_cpu_n(N, sigma):
    """The oversampled size the library chooses: the smallest even 7-smooth
    integer >= sigma N."""
    n = math.ceil(sigma * N - 1e-9)
    n += n % 2
    while True:
        v = n
        for p in (2, 3, 5, 7):
            while v % p == 0:
                v //= p
        if v == 1:
            return n
        n += 2


@pytest.mark.gpu
def test_gpu_lowdim_errors():
    import torch
    from paper_1605_01244_gb300 import _lib
    from paper_1605_01244_gb300.lowdim import nfft_eval
    c = torch.from_numpy(coeffs((16,), 8)).cuda()
    with pytest.raises(ValueError):
        nfft_eval(c, torch.zeros((4, 1), dtype=torch.float64, device="cuda"), m=0)
    bad = torch.tensor([[0.1], [float("nan")]], dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.NFFTError) as e:
        nfft_eval(c, bad)
    assert e.value.code == _lib.NFFT3_ERR_POINTS
    assert nfft_eval(c, torch.zeros((0, 1), dtype=torch.float64, device="cuda")).shape == (0,)
