"""Exact evaluation on a rectilinear grid (the paper's igridftn, Sec. 2.1),
through nfft3*_grid_eval: against the FP64 direct sum at every grid point,
against numpy's inverse FFT on the 64^3 regular grid of the paper's own
check (tests/golden/paper_grid_errors.txt: agreement at the rounding level),
and against the NFFT on a local box lattice (the dense judge's lattice)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_01244_gb300 import workloads as wl
from tests._util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_01244_gb300 import build
    build.build()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 5e-6)])
def test_nonuniform_grid_against_direct_sum(prec, tol):
    from paper_1605_01244_gb300.grid import grid_eval
    N = (8, 12, 10)
    c = wl.gaussian_coeffs(N, 1e9, seed=50)
    g = wl.rng(51)
    ys = [np.sort(g.uniform(-0.7, 0.9, M)) for M in (7, 9, 11)]    # some outside [-1/2, 1/2): periodic
    cd = torch.complex128 if prec == "f64" else torch.complex64
    f = grid_eval(torch.from_numpy(c).to(cd).cuda(), *[torch.from_numpy(y).cuda() for y in ys])
    assert f.shape == (7, 9, 11) and f.dtype == cd
    pts = np.stack(np.meshgrid(*ys, indexing="ij"), -1).reshape(-1, 3)
    ref = oracle.forward(c, pts)
    assert rel_l2(f.cpu().numpy().reshape(-1).astype(np.complex128), ref) <= tol


def test_paper_regular_grid_check_against_ifft():
    """64^3 coefficients at the 64^3 grid x = -1/2 + l/64: the paper compares
    its evaluations with the inverse FFT and prints ~1e-13 (absolute, values
    of order 10^2..10^3); here the relative bound of the golden pin."""
    from paper_1605_01244_gb300.grid import grid_eval
    from tests.test_golden_paper import grid_experiment, printed_errors
    c, nodes, ref, _ = grid_experiment()
    y = torch.arange(64, dtype=torch.float64, device="cuda") / 64 - 0.5
    f = grid_eval(torch.from_numpy(c).cuda(), y, y, y).cpu().numpy().reshape(-1)
    bound_rel = max(printed_errors().values()) / 100.0
    assert np.max(np.abs(f - ref)) <= bound_rel * np.max(np.abs(ref))


def test_empty_and_box_lattice_against_nfft():
    from paper_1605_01244_gb300 import judge
    from paper_1605_01244_gb300.grid import grid_eval
    N = 32
    c = torch.from_numpy(wl.gpe_coeffs((N, N, N), 8.0, 0.4)).cuda()
    e = grid_eval(c, torch.zeros(0, dtype=torch.float64, device="cuda"),
                  torch.zeros(3, dtype=torch.float64, device="cuda"), torch.zeros(2, dtype=torch.float64, device="cuda"))
    assert e.shape == (0, 3, 2)
    R, lo, hi = (21, 17, 19), (-0.05, -0.04, -0.06), (0.05, 0.04, 0.03)
    fg = grid_eval(c, *judge.lattice_axes(R, lo, hi)).reshape(-1)
    x = judge.lattice(R, lo, hi)
    plan = judge.make_plan(c, x.shape[0])
    plan.set_points(x)
    fn = plan.eval(c)
    assert rel_l2(fg.cpu().numpy(), fn.cpu().numpy()) <= 1e-12
    # the dense judge finds the same crossings by either evaluation
    a = judge.dense_crossings(c, R, lo, hi, method="grid")
    b = judge.dense_crossings(c, R, lo, hi, method="nfft")
    assert a.points.shape == b.points.shape
    if a.points.shape[0]:
        pa = a.points.cpu().numpy()
        pb = b.points.cpu().numpy()
        assert np.array_equal(np.sort(pa, axis=0), np.sort(pb, axis=0))


def test_two_dimensional_grid_as_unit_third_dimension():
    """The paper's igridft2 (a 2D series on a rectilinear grid): the same
    contractions with N3 = M3 = 1 (y3 = 0) against the 2D direct sum."""
    from oracle import nfft_cpu
    from paper_1605_01244_gb300.grid import grid_eval
    g = wl.rng(55)
    c2 = g.standard_normal((12, 10)) + 1j * g.standard_normal((12, 10))
    y1 = np.sort(g.uniform(-0.5, 0.5, 9))
    y2 = np.sort(g.uniform(-0.5, 0.5, 13))
    f = grid_eval(torch.from_numpy(c2[:, :, None]).cuda(), torch.from_numpy(y1).cuda(), torch.from_numpy(y2).cuda(),
                  torch.zeros(1, dtype=torch.float64, device="cuda")).cpu().numpy()[:, :, 0]
    pts = np.stack(np.meshgrid(y1, y2, indexing="ij"), -1).reshape(-1, 2)
    ref = nfft_cpu.direct_lowdim(c2, pts).reshape(9, 13)
    assert np.max(np.abs(f - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("scale", [0, -200, 200])
def test_double_float_products_against_direct_sum(scale, monkeypatch):
    """GBNFFT_GRID_DF=1: the FP64 family's contractions in double-float on the
    FP32 pipe (about 48 significant bits), with c scaled into range by its
    largest magnitude; against the FP64 direct sum, on shapes that leave
    ragged edges in every tile of the product kernels."""
    from paper_1605_01244_gb300.grid import grid_eval
    monkeypatch.setenv("GBNFFT_GRID_DF", "1")
    N = (20, 34, 18)
    c = wl.gaussian_coeffs(N, 1e9, seed=56)
    c = np.ldexp(c.real, scale) + 1j * np.ldexp(c.imag, scale)
    g = wl.rng(57)
    ys = [g.uniform(-0.5, 0.5, M) for M in (67, 5, 71)]
    f = grid_eval(torch.from_numpy(c).cuda(), *[torch.from_numpy(y).cuda() for y in ys])
    pts = np.stack(np.meshgrid(*ys, indexing="ij"), -1).reshape(-1, 3)
    ref = oracle.forward(c, pts)
    assert rel_l2(f.cpu().numpy().reshape(-1), ref) <= 1e-13


@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 5e-6)])
def test_products_over_several_tiles(prec, tol):
    """Shapes spanning several 64 x 64 output tiles and K-slices with ragged
    tails in every dimension, against the direct sum on sampled grid points."""
    from paper_1605_01244_gb300.grid import grid_eval
    N = (70, 66, 36)
    c = wl.gaussian_coeffs(N, 20.0, seed=58)
    g = wl.rng(59)
    ys = [g.uniform(-0.5, 0.5, M) for M in (130, 67, 9)]
    cd = torch.complex128 if prec == "f64" else torch.complex64
    f = grid_eval(torch.from_numpy(c).to(cd).cuda(), *[torch.from_numpy(y).cuda() for y in ys]).cpu().numpy()
    idx = [g.integers(0, len(y), 300) for y in ys]
    pts = np.stack([ys[d][idx[d]] for d in range(3)], axis=1)
    ref = oracle.forward(c, pts)
    assert rel_l2(f[idx[0], idx[1], idx[2]].astype(np.complex128), ref) <= tol
