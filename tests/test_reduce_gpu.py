"""set_points' coordinate reduction, bit for bit.

For every coordinate the library forms, with FP64 round-to-nearest steps,
    x_w = x - floor(x + 1/2),  u = n (x_w + 1/2),  v = u - (m + 1/2),
    l0 = ceil(v),  s = l0 - v,
and stores l0 mod n with s (FP64 family) or s with its significand cut to
FP32 (mixed family).  For n = 2^L >= 8 the library takes the steps after
x_w + 1/2 on the integer pipe (except next to x = -1/2); they must give the same bits as numpy's FP64
arithmetic here, on random, boundary and tie-producing inputs, and the
stencil origins must be the oracle's.
"""
import numpy as np
import pytest
import torch

from oracle import nfft_cpu
from paper_1605_01244_gb300 import build, workloads as wl
from paper_1605_01244_gb300._lib import NFFTError
from paper_1605_01244_gb300.nfft import reduce_coords

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def expected(x, n, m):
    xw = x - np.floor(x + 0.5)
    u = n * (xw + 0.5)
    v = u - (m + 0.5)
    l0 = np.ceil(v)
    s = l0 - v
    s = np.where(s >= 1.0, 0.0, s)
    b = s.view(np.uint64)
    e = (b >> np.uint64(52)).astype(np.int64) - 1023
    f32 = (((e + 127) << 23) | ((b >> np.uint64(29)) & np.uint64(0x7FFFFF)).astype(np.int64)).astype(np.uint32)
    s32 = np.where(e < -126, np.float32(0), f32.view(np.float32))
    return (l0.astype(np.int64) % n).astype(np.int32), s, s32


def inputs(n, m, seed):
    g = wl.rng(seed)
    parts = [g.uniform(-0.5, 0.5, 100000),
             -0.5 + g.uniform(0, 2.0 ** -8, 20000),              # x_w + 1/2 below and above 2^-10
             0.5 - g.uniform(0, 1e-6, 5000),
             g.uniform(-1e3, 1e3, 20000),
             np.array([-0.5, 0.5, 0.0, -0.0, 1e6 + 0.125, -3.25, 7.0, -1e-300, 1e-300, 5e-324, -5e-324,
                       np.nextafter(0.5, 0), np.nextafter(-0.5, 0), np.nextafter(-0.5, -1), 0.25, -0.25])]
    # every exponent from 2^-62 to 2^-1 with random significands and signs
    e = g.integers(-62, 0, 40000)
    parts.append(np.ldexp(1.0 + g.random(40000), e) * np.where(g.random(40000) < 0.5, -1.0, 1.0))
    # grid nodes, half nodes and u - alpha at integers, with their FP64 neighbours
    l = np.arange(-2, n + 3, dtype=np.float64) if n <= 4096 else g.integers(-2, n + 3, 5000).astype(np.float64)
    for off in (0.0, 0.5, m + 0.5):
        base = (l + off) / n - 0.5
        parts += [base, np.nextafter(base, 1), np.nextafter(base, -1),
                  np.nextafter(np.nextafter(base, 1), 1), np.nextafter(np.nextafter(base, -1), -1)]
    return np.concatenate(parts)


@pytest.mark.parametrize("n", [8, 16, 32, 512, 1 << 20, 1 << 30, 24, 22, 510])
@pytest.mark.parametrize("m", [1, 3, 6, 8])
def test_reduction_matches_fp64_steps(n, m):
    x = inputs(n, m, seed=n + 17 * m)
    l0, s, s32 = reduce_coords(torch.from_numpy(x).cuda(), n, m)
    el0, es, es32 = expected(x, n, m)
    assert np.array_equal(l0.cpu().numpy(), el0)
    assert np.array_equal(s.cpu().numpy().view(np.uint64), es.view(np.uint64))
    assert np.array_equal(s32.cpu().numpy().view(np.uint32), es32.view(np.uint32))


@pytest.mark.parametrize("n", [16, 512])
def test_stencil_origins_are_the_oracles(n):
    m = 6
    x = inputs(n, m, seed=3)[: 3 * 30000].reshape(-1, 3)
    l0, _, _ = reduce_coords(torch.from_numpy(x).cuda(), n, m)
    ol0, _ = nfft_cpu._window_rows(x, (n, n, n), m, [1.0, 1.0, 1.0])
    for d in range(3):
        assert np.array_equal(l0[:, d].cpu().numpy().astype(np.int64), ol0[d] % n)


def test_non_finite_flagged():
    x = torch.tensor([0.1, float("nan"), 0.2], dtype=torch.float64, device="cuda")
    with pytest.raises(NFFTError):
        reduce_coords(x, 64, 3)
