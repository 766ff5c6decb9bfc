"""Deterministic adjoint (nfft3_set_deterministic), through the C ABI.

The default adjoint's spread adds its tile boxes to the grid with FP64
atomics, and the point order within a tile follows the sort's atomics, so
results vary in the last bits from run to run.  In deterministic mode the
points of a tile keep their original order (a stable radix sort) and the
boxes are added as exact fixed-point sums, so two runs give the same bits.
Checked at the benchmark size (N = 256^3, M = 10^7, clustered), against the
direct adjoint on sampled frequencies and against the default mode, and at
a small size against the direct sum at every frequency.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_01244_gb300 import build, workloads as wl
from paper_1605_01244_gb300._lib import NFFTError, NFFT3_ERR_ARG, NFFT3_ERR_NO_POINTS
from tests._util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_bitwise_reproducible_at_benchmark_size():
    from paper_1605_01244_gb300 import Plan
    c, x = wl.precision_sweep()
    g = wl.rng(81)
    f = torch.from_numpy(g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))).cuda()
    xd = to_dev(x)
    plan = Plan(c.shape, len(x), m=6)
    plan.set_points(xd)
    h_default = plan.adjoint(f)
    plan.set_deterministic(True)
    with pytest.raises(NFFTError) as e:
        plan.adjoint(f)
    assert e.value.code == NFFT3_ERR_NO_POINTS
    plan.set_points(xd)
    h1 = plan.adjoint(f).clone()
    h2 = plan.adjoint(f).clone()
    plan.set_points(xd)
    h3 = plan.adjoint(f)
    assert torch.equal(h1, h2) and torch.equal(h1, h3)
    assert _max_rel(to_np(h1), to_np(h_default)) <= 1e-12
    N = c.shape
    ks = np.concatenate([np.array([[0, 0, 0], [-128, -128, -128], [127, 127, 127]]),
                         np.stack([g.integers(-n // 2, n // 2, 29) for n in N], axis=1)])
    hs = to_np(h1[tuple(torch.from_numpy(ks[:, d] + N[d] // 2).cuda() for d in range(3))])
    hd = oracle.adjoint_at(to_np(f), x, ks)
    assert rel_l2(hs, hd) <= 5e-12
    # eval computes every point on its own: the point order does not change its bits
    ct = to_dev(c)
    fd_det = plan.eval(ct)
    p0 = Plan(c.shape, len(x), m=6)
    p0.set_points(xd)
    assert torch.equal(fd_det, p0.eval(ct))


@pytest.mark.parametrize("m", [3, 7, 8])
def test_small_size_against_direct_sum(m):
    from paper_1605_01244_gb300 import Plan
    N = (16, 20, 12)
    x = np.concatenate([wl.uniform_points(700, seed=82), wl.cluster_points(1300, 0.003, seed=83)])
    g = wl.rng(84)
    f = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    plan = Plan(N, len(x), m=m)
    plan.set_deterministic(True)
    plan.set_points(to_dev(x))
    h = to_np(plan.adjoint(to_dev(f)))
    hd = oracle.adjoint(f, x, N)
    assert rel_l2(h, hd) <= (5e-12 if m >= 7 else 5e-6)
    assert torch.equal(plan.adjoint(to_dev(f)), plan.adjoint(to_dev(f)))


def test_refused_where_not_supported():
    from paper_1605_01244_gb300 import Plan
    plan = Plan((8, 8, 8), 10, m=3, precision="f32")
    with pytest.raises(NFFTError) as e:
        plan.set_deterministic(True)
    assert e.value.code == NFFT3_ERR_ARG
    plan = Plan((8, 8, 8), 10, m=4)
    plan.set_deterministic(True)
    plan.set_deterministic(False)
    plan.set_points(torch.zeros((10, 3), dtype=torch.float64, device="cuda"))
    plan.adjoint(torch.ones(10, dtype=torch.complex128, device="cuda"))
