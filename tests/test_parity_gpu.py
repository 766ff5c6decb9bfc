"""Parity of the CUDA NFFT (through the C ABI) against the CPU oracle.

Two references:
* ``oracle.forward / forward_grad / adjoint`` -- the FP64 direct sums (the
  definition, paper eq. (fs)/(Fs), eq. (Lambda)); the gate is relative l2
  <= 1e-12 (FP64 family) and <= 1e-6 (mixed family);
* ``oracle.nfft_cpu`` -- the same approximation restated in numpy; the
  FP64 family must agree with it to rounding (1e-13 of max |f|, element by
  element), which checks every step of the kernels, not only the end result.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import nfft_cpu
from paper_1605_01244_gb300 import build, workloads as wl
from paper_1605_01244_gb300._lib import NFFTError, NFFT3_ERR_NO_POINTS, NFFT3_ERR_POINTS
from tests._util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

CD = {"f64": torch.complex128, "f32": torch.complex64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def gpu_eval(c, x, m, prec="f64", sigma=2.0):
    from paper_1605_01244_gb300 import Plan
    plan = Plan(c.shape, len(x), m=m, sigma=sigma, precision=prec)
    plan.set_points(to_dev(np.asarray(x, np.float64).reshape(-1, 3)))
    f = plan.eval(to_dev(c, CD[prec]))
    return to_np(f).astype(np.complex128), plan


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_small_random_fp64_gate():
    c, x = wl.small_random()
    f, plan = gpu_eval(c, x, m=6)
    assert plan.n == (32, 32, 32)
    assert rel_l2(f, oracle.forward(c, x)) <= 1e-12
    assert max_rel(f, nfft_cpu.forward(c, x, plan.n, 6)) <= 1e-13


def test_small_random_mixed_gate():
    """m chosen by the plan for eps = 1e-6 (m = 4 at sigma = 2) meets the mixed gate."""
    from paper_1605_01244_gb300 import Plan, choose_m
    c, x = wl.small_random()
    fd = oracle.forward(c, x)
    m = choose_m(1e-6)
    assert m == 4
    f, _ = gpu_eval(c, x, m=m, prec="f32")
    assert rel_l2(f, fd) <= 1e-6
    # one m lower the window error alone (6e-7 here) leaves no room for FP32 rounding
    f3, _ = gpu_eval(c, x, m=3, prec="f32")
    assert rel_l2(f3, fd) <= 1.5e-6


@pytest.mark.parametrize("N,M,m", [((8, 12, 10), 1, 1), ((8, 12, 10), 37, 2), ((16, 6, 20), 515, 3),
                                   ((4, 4, 4), 100, 5), ((20, 16, 12), 777, 7), ((10, 8, 6), 300, 8)])
def test_same_algorithm_as_cpu_nfft(N, M, m):
    c = wl.gaussian_coeffs(N, 1e9, seed=M)
    x = wl.uniform_points(M, seed=M + 1)
    f, plan = gpu_eval(c, x, m=m)
    assert max_rel(f, nfft_cpu.forward(c, x, plan.n, m)) <= 1e-13
    f32, plan32 = gpu_eval(c, x, m=m, prec="f32")
    assert rel_l2(f32, nfft_cpu.forward(c, x, plan32.n, m)) <= 2e-6


@pytest.mark.parametrize("mode", ["df", "fp64", "full"])
@pytest.mark.parametrize("m", [4, 6, 8])
def test_value_gather_weight_tables(mode, m, monkeypatch):
    """The FP64 value gather's tap weights: half-interval tables (degree 11 in
    u = 4s - 3, tap 2m - a reflected for s < 1/2) in double-float (default)
    or FP64, and the whole-interval FP64 table, each against the CPU NFFT
    restatement; points at s = 0, 1/2 and just below 1 included."""
    monkeypatch.setenv("GBNFFT_SLOT_WEIGHTS", mode)
    N = (16, 24, 20)
    n = (32, 48, 40)
    c = wl.gaussian_coeffs(N, 1e9, seed=m)
    edge = np.array([[0.0, 0.0, 0.0], [1 / 64, 1 / 96, 1 / 80], [-0.5, 0.5 - 1e-16, 1 / 64 - 1e-13],
                     [0.5 / 32, 0.5 / 48, 0.5 / 40]])
    x = np.concatenate([wl.uniform_points(600, seed=m + 1), edge])
    f, plan = gpu_eval(c, x, m=m)
    assert plan.n == n
    assert max_rel(f, nfft_cpu.forward(c, x, n, m)) <= 1e-13


def test_non_power_of_two_oversampling():
    N = (10, 14, 18)
    c = wl.gaussian_coeffs(N, 1e9, seed=3)
    x = wl.uniform_points(400, seed=4)
    f, plan = gpu_eval(c, x, m=5, sigma=1.5)
    assert plan.n == (16, 22, 28) or all(v >= 1.5 * w for v, w in zip(plan.n, N))
    assert max_rel(f, nfft_cpu.forward(c, x, plan.n, 5)) <= 1e-13


def test_edge_points():
    N = (8, 10, 12)
    c = wl.gaussian_coeffs(N, 3.0, seed=5)
    n = (16, 20, 24)
    nodes = np.stack(np.meshgrid(*[np.arange(v) / v - 0.5 for v in n], indexing="ij"), -1).reshape(-1, 3)
    half = nodes + 0.5 / np.asarray(n)
    special = np.array([[-0.5, -0.5, -0.5], [0.5, 0.5, 0.5], [np.nextafter(0.5, 0), -0.5, 0.0],
                        [1e6 + 0.125, -3.25, 7.0], [-1e-300, 1e-300, 0.0], [0.49999999999, -0.49999999999, 0.3]])
    for pts in (nodes, half, special):
        f, plan = gpu_eval(c, pts, m=6)
        assert plan.n == n
        assert max_rel(f, nfft_cpu.forward(c, pts, n, 6)) <= 1e-13
        assert rel_l2(f, oracle.forward(c, pts)) <= 1e-11


def test_all_points_in_one_cell():
    c = wl.gaussian_coeffs((16, 16, 16), 4.0, seed=6)
    x = wl.cluster_points(5000, 1e-4, seed=7)
    f, plan = gpu_eval(c, x, m=6)
    assert max_rel(f, nfft_cpu.forward(c, x, plan.n, 6)) <= 1e-13


def test_empty_and_errors():
    from paper_1605_01244_gb300 import Plan
    c = to_dev(wl.gaussian_coeffs((8, 8, 8), 3.0), torch.complex128)
    plan = Plan((8, 8, 8), 0, m=4)
    plan.set_points(torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert plan.eval(c).shape == (0,)
    h = plan.adjoint(torch.zeros(0, dtype=torch.complex128, device="cuda"))
    assert torch.count_nonzero(h).item() == 0
    plan2 = Plan((8, 8, 8), 4, m=4)
    with pytest.raises(NFFTError) as e:
        plan2.eval(c)
    assert e.value.code == NFFT3_ERR_NO_POINTS
    bad = torch.tensor([[0.1, 0.2, 0.3], [float("nan"), 0, 0], [0, 0, 0], [0, float("inf"), 0]],
                       dtype=torch.float64, device="cuda")
    with pytest.raises(NFFTError) as e:
        plan2.set_points(bad)
    assert e.value.code == NFFT3_ERR_POINTS
    with pytest.raises(NFFTError):
        plan2.eval(c)          # the failed set_points left no points


def test_gradient_against_oracle():
    from paper_1605_01244_gb300 import Plan
    N = (12, 16, 10)
    c = wl.gaussian_coeffs(N, 3.0, seed=8)
    x = wl.uniform_points(600, seed=9)
    fd, gd = oracle.forward_grad(c, x)
    for prec, m, tol_f, tol_g in (("f64", 6, 1e-12, 1e-11), ("f32", 4, 1e-6, 5e-6)):
        plan = Plan(N, len(x), m=m, precision=prec)
        plan.set_points(to_dev(x))
        f, g = plan.eval_grad(to_dev(c, CD[prec]))
        f = to_np(f).astype(np.complex128)
        g = to_np(g).astype(np.complex128)
        assert rel_l2(f, fd) <= tol_f, prec
        for d in range(3):
            assert rel_l2(g[:, d], gd[:, d]) <= tol_g, (prec, d)
        # the value from eval_grad agrees with eval (the value gather and the
        # four-grid gather sum the taps in different orders)
        fe = to_np(plan.eval(to_dev(c, CD[prec]))).astype(np.complex128)
        assert max_rel(f, fe) <= (5e-14 if prec == "f64" else 1e-6)
    # f may be omitted
    plan = Plan(N, len(x), m=6)
    plan.set_points(to_dev(x))
    f, g = plan.eval_grad(to_dev(c, CD["f64"]), want_f=False)
    assert f is None and rel_l2(to_np(g)[:, 0], gd[:, 0]) <= 1e-11


def test_gradient_same_algorithm_as_cpu_nfft():
    from paper_1605_01244_gb300 import Plan
    N = (8, 10, 12)
    c = wl.gaussian_coeffs(N, 1e9, seed=10)
    x = wl.uniform_points(200, seed=11)
    plan = Plan(N, len(x), m=5)
    plan.set_points(to_dev(x))
    f, g = plan.eval_grad(to_dev(c))
    fc, gc = nfft_cpu.forward_grad(c, x, plan.n, 5)
    assert max_rel(to_np(g), gc) <= 1e-13
    assert max_rel(to_np(f), fc) <= 1e-13


@pytest.mark.parametrize("prec,m,tol", [("f64", 6, 5e-12), ("f32", 4, 1e-6)])
def test_adjoint_against_oracle(prec, m, tol):
    from paper_1605_01244_gb300 import Plan
    N = (10, 8, 12)
    x = np.concatenate([wl.uniform_points(700, seed=12), wl.cluster_points(300, 0.01, seed=13)])
    g = wl.rng(14)
    f = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    plan = Plan(N, len(x), m=m, precision=prec)
    plan.set_points(to_dev(x))
    h = to_np(plan.adjoint(to_dev(f, CD[prec]))).astype(np.complex128)
    assert rel_l2(h, oracle.adjoint(f, x, N)) <= tol
    if prec == "f64":
        assert max_rel(h, nfft_cpu.adjoint(f, x, N, plan.n, m)) <= 1e-12


def test_fast_adjoint_identity():
    from paper_1605_01244_gb300 import Plan
    N = (16, 12, 8)
    c = wl.gaussian_coeffs(N, 1e9, seed=15)
    x = wl.mixed_points(2000, 0.05, seed=16)
    g = wl.rng(17)
    f = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    plan = Plan(N, len(x), m=4)
    plan.set_points(to_dev(x))
    Ac = to_np(plan.eval(to_dev(c)))
    Ahf = to_np(plan.adjoint(to_dev(f)))
    lhs, rhs = np.vdot(f, Ac), np.vdot(Ahf, c)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_host_path_matches_device_path(prec):
    from paper_1605_01244_gb300 import Plan
    c, x = wl.small_random(M=3000)
    plan = Plan(c.shape, len(x), m=5, precision=prec)
    xh = torch.from_numpy(x).contiguous()
    ch = torch.from_numpy(c).to(CD[prec]).contiguous()
    fh = torch.empty(len(x), dtype=CD[prec])
    plan.eval_host(xh, ch, fh)
    plan.set_points(xh.cuda())
    fdev = plan.eval(ch.cuda()).cpu()
    assert torch.equal(fh, fdev)
    # staging is sized for the capacity: a smaller first call, then the full count
    plan2 = Plan(c.shape, len(x), m=5, precision=prec)
    plan2.set_num_points(100)
    f_small = torch.empty(100, dtype=CD[prec])
    plan2.eval_host(xh[:100].contiguous(), ch, f_small)
    assert torch.equal(f_small, fdev[:100]) or max_rel(f_small.numpy(), fdev[:100].numpy()) <= 1e-15
    plan2.set_num_points(len(x))
    f_full = torch.empty(len(x), dtype=CD[prec])
    plan2.eval_host(xh, ch, f_full)
    assert torch.equal(f_full, fdev)
    # back-to-back calls with new coefficients and points: the transform of
    # the next call (on the plan's second stream) must not overtake the
    # gather of the previous one
    for seed in (7, 8):
        c2, x2 = wl.small_random(M=3000, seed=seed)
        x2h, c2h = torch.from_numpy(x2).contiguous(), torch.from_numpy(c2).to(CD[prec]).contiguous()
        f2 = torch.empty(len(x2), dtype=CD[prec])
        plan2.eval_host(x2h, c2h, f2)
        plan.set_points(x2h.cuda())
        assert torch.equal(f2, plan.eval(c2h.cuda()).cpu())


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_eval_points_matches_set_points_then_eval(prec):
    """nfft3*_eval_points (the transform of c overlapping the sort of x)
    against set_points followed by eval: the same bits, on back-to-back
    calls with new points and coefficients, with a clustered population
    (dense batches) included; non-finite points fail like set_points; an
    empty plan returns at once."""
    from paper_1605_01244_gb300 import Plan, _lib
    N = (32, 32, 32)
    M = 20001
    plan = Plan(N, M, m=5, precision=prec)
    ref = Plan(N, M, m=5, precision=prec)
    for seed in (1, 2, 3):
        c = to_dev(wl.gaussian_coeffs(N, 6.0, seed=seed), CD[prec])
        x = to_dev(wl.mixed_points(M, 0.01, seed=seed + 10))
        f = plan.eval_points(x, c)
        ref.set_points(x)
        assert torch.equal(f, ref.eval(c))
    bad = x.clone()
    bad[7, 1] = float("nan")
    with pytest.raises(NFFTError) as e:
        plan.eval_points(bad, c)
    assert e.value.code == NFFT3_ERR_POINTS
    empty = Plan(N, 0, m=5, precision=prec)
    assert empty.eval_points(torch.empty((0, 3), dtype=torch.float64, device="cuda"), c).shape == (0,)


@pytest.mark.parametrize("prec,m,tol", [("f64", 6, 1e-12), ("f32", 3, 1e-6)])
def test_precision_sweep_full_size_sampled(prec, m, tol):
    """N = 256^3, M = 10^7 (half uniform, half clustered, std 0.02), the
    benchmark's launch configuration; 2000 sampled outputs (1000 from each
    population) against the FP64 direct sum."""
    from paper_1605_01244_gb300 import Plan
    c, x = wl.precision_sweep()
    M = len(x)
    plan = Plan(c.shape, M, m=m, precision=prec)
    plan.set_points(to_dev(x))
    f = plan.eval(to_dev(c, CD[prec]))
    idx = np.concatenate([wl.rng(99).choice(M // 2, 1000, replace=False),
                          M // 2 + wl.rng(98).choice(M - M // 2, 1000, replace=False)])
    fs = to_np(f[torch.from_numpy(idx).cuda()]).astype(np.complex128)
    fd = oracle.forward(c, x[idx])
    err = rel_l2(fs, fd)
    print("precision sweep %s m=%d: rel-l2 %.3e" % (prec, m, err))
    assert err <= tol
    assert np.all(np.isfinite(to_np(f)))


@pytest.mark.parametrize("prec,tol", [("f64", 2e-14), ("f32", 3e-7)])
def test_window_polynomials_accuracy(prec, tol):
    """Each tap's weight polynomial (fitted at plan creation, evaluated by
    Horner in the family's precision) against the exact long-double window."""
    import ctypes
    from paper_1605_01244_gb300 import Plan, _lib
    for sigma in (1.25, 2.0, 8.0):
        for m in range(1, 9):
            plan = Plan((16, 12, 10), 1, m=m, sigma=sigma, precision=prec)
            err = ctypes.c_double()
            _lib.call("nfft3_window_error", plan._h, ctypes.byref(err))
            assert err.value <= tol, (sigma, m, err.value)


@pytest.mark.parametrize("m", [2, 3, 6, 8])
def test_gather_variants_agree(m, monkeypatch):
    """Gather variants selected by GBNFFT_GATHER: default (lane groups over the
    padded grid; for the FP64 family double-float on the FP32 pipe, the value
    gather spreading each plane's taps over all lanes -- GBNFFT_DF_COLUMNS=1
    keeps one column per lane -- and tap weights by FP64 Horner, or by
    double-float Horner with GBNFFT_DF_WEIGHTS=df), tma (mixed-family values from TMA-staged shared-memory tiles),
    thread (one thread per point) and native (FP64 family on the FP64 pipe).  Every variant must match the CPU NFFT, for eval and
    eval_grad: to rounding in FP64, to FP32 accuracy in the mixed family."""
    from paper_1605_01244_gb300 import Plan
    N = (12, 16, 10)
    c = wl.gaussian_coeffs(N, 1e9, seed=30 + m)
    x = wl.mixed_points(900, 0.03, seed=31)
    ref = None
    for prec, modes in (("f64", ("default", "df-columns", "df-weights", "thread", "native")),
                        ("f32", ("default", "tma", "thread"))):
        for mode in modes:
            monkeypatch.delenv("GBNFFT_DF_WEIGHTS", raising=False)
            monkeypatch.delenv("GBNFFT_DF_COLUMNS", raising=False)
            if mode == "default":
                monkeypatch.delenv("GBNFFT_GATHER", raising=False)
            elif mode == "df-weights":
                monkeypatch.delenv("GBNFFT_GATHER", raising=False)
                monkeypatch.setenv("GBNFFT_DF_WEIGHTS", "df")
            elif mode == "df-columns":
                monkeypatch.delenv("GBNFFT_GATHER", raising=False)
                monkeypatch.setenv("GBNFFT_DF_COLUMNS", "1")
            else:
                monkeypatch.setenv("GBNFFT_GATHER", mode)
            plan = Plan(N, len(x), m=m, precision=prec)
            plan.set_points(to_dev(x))
            f = to_np(plan.eval(to_dev(c, CD[prec]))).astype(np.complex128)
            fg, g = plan.eval_grad(to_dev(c, CD[prec]))
            fg = to_np(fg).astype(np.complex128)
            g = to_np(g).astype(np.complex128)
            if ref is None:
                ref = nfft_cpu.forward_grad(c, x, plan.n, m)
            fc, gc = ref
            if prec == "f64":
                assert max_rel(f, fc) <= 1e-13, mode
                assert max_rel(fg, fc) <= 1e-13, mode
                assert max_rel(g, gc) <= 1e-13, mode
            else:
                assert rel_l2(f, fc) <= 2e-6, mode
                assert rel_l2(fg, fc) <= 2e-6, mode
                assert rel_l2(g, gc) <= 5e-6, mode


@pytest.mark.parametrize("m", [2, 3, 5])
def test_f32_shared_table_gather(m, monkeypatch):
    """Cubic grids share one window table across dimensions; the FP32 value
    gather then keeps the lane's tap polynomial in registers and walks points
    grid-stride (gather_col_f32_cube_kernel).  It must match the per-point
    table kernel (GBNFFT_F32_NO_CUBE=1) and the CPU NFFT, including a ragged
    tail of points (M not a multiple of the points per warp)."""
    from paper_1605_01244_gb300 import Plan
    N = (16, 16, 16)
    c = wl.gaussian_coeffs(N, 1e9, seed=90 + m)
    x = wl.mixed_points(2003, 0.05, seed=91)
    fc = nfft_cpu.forward(c, x, (32, 32, 32), m)
    out = {}
    for mode in ("cube", "table"):
        monkeypatch.delenv("GBNFFT_F32_NO_CUBE", raising=False)
        if mode == "table":
            monkeypatch.setenv("GBNFFT_F32_NO_CUBE", "1")
        plan = Plan(N, len(x), m=m, precision="f32")
        plan.set_points(to_dev(x))
        out[mode] = to_np(plan.eval(to_dev(c, torch.complex64))).astype(np.complex128)
        assert rel_l2(out[mode], fc) <= 2e-6, mode
    assert max_rel(out["cube"], out["table"]) <= 1e-6


@pytest.mark.parametrize("N,m", [((32, 32, 32), 3), ((32, 32, 32), 8), ((16, 24, 20), 2), ((16, 24, 20), 5)])
def test_split_value_gather(N, m, monkeypatch):
    """The mixed family's value gather splits the points: sort keys (one tile,
    one (x, y) cell of stencil centres) with at least GBNFFT_DENSE_MIN points
    (default 12) go to dense batches, one point per lane; the rest go to the
    column kernel through an index list.  Every threshold -- no split (0), all
    keys of >= 4 points dense, none dense -- must match the CPU NFFT and each
    other, on a tight cluster (hundreds of points per cell), a wider one and
    uniform points, with ragged batch sizes, on cubic and non-cubic grids."""
    from paper_1605_01244_gb300 import Plan
    c = wl.gaussian_coeffs(N, 1e9, seed=60 + m)
    x = np.concatenate([wl.cluster_points(20011, 0.004, seed=61), wl.cluster_points(5003, 0.05, seed=62),
                        wl.uniform_points(3001, seed=63)])
    fc = nfft_cpu.forward(c, x, tuple(2 * v for v in N), m)
    out = {}
    for dm in ("default", "0", "4", "1000000"):
        monkeypatch.delenv("GBNFFT_DENSE_MIN", raising=False)
        if dm != "default":
            monkeypatch.setenv("GBNFFT_DENSE_MIN", dm)
        plan = Plan(N, len(x), m=m, precision="f32")
        plan.set_points(to_dev(x))
        out[dm] = to_np(plan.eval(to_dev(c, torch.complex64))).astype(np.complex128)
        assert rel_l2(out[dm], fc) <= 2e-6, dm
        # the stored-grid gather takes the same split
        plan.precompute(to_dev(c, torch.complex64))
        assert np.array_equal(to_np(plan.eval_stored()).astype(np.complex128), out[dm]), dm
    for dm in ("0", "4", "1000000"):
        assert max_rel(out["default"], out[dm]) <= 1e-6, dm


@pytest.mark.parametrize("N", [(16, 32, 8), (8, 1024, 8), (64, 64, 64)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fused_transform_matches_cufft_and_cpu(N, prec, monkeypatch):
    """Power-of-two grids take the fused transform (deconvolution, radix-8
    Stockham line passes in shared memory -- double-float for the FP64 family --
    and the padded output) by default; GBNFFT_FFT=cufft takes cuFFT plus the
    separate deconvolution and padding kernels.  Both must match the CPU NFFT
    for eval, eval_grad and stored evaluations, and in the FP32 family also
    with the tile-staged gather (centre-shifted padded layout).  n covers line
    lengths 16 .. 2048 (radix-8 passes followed by a radix-2 or -4 pass)."""
    from paper_1605_01244_gb300 import Plan
    c = wl.gaussian_coeffs(N, 1e9, seed=70)
    x = wl.mixed_points(1500, 0.05, seed=71)
    m = 6 if prec == "f64" else 3
    fc, gc = nfft_cpu.forward_grad(c, x, tuple(2 * v for v in N), m)
    tol_f, tol_g = (2e-13, 3e-13) if prec == "f64" else (2e-6, 5e-6)
    err = max_rel if prec == "f64" else rel_l2
    modes = [("fused", None), ("cufft", "cufft")] + ([("fused-tma", "tma")] if prec == "f32" else [])
    for name, env in modes:
        monkeypatch.delenv("GBNFFT_FFT", raising=False)
        monkeypatch.delenv("GBNFFT_GATHER", raising=False)
        if name == "cufft":
            monkeypatch.setenv("GBNFFT_FFT", "cufft")
        if name == "fused-tma":
            monkeypatch.setenv("GBNFFT_GATHER", "tma")
        plan = Plan(N, len(x), m=m, sigma=2.0, precision=prec)
        assert plan.n == tuple(2 * v for v in N)
        plan.set_points(to_dev(x))
        cd = to_dev(c, CD[prec])
        f = to_np(plan.eval(cd)).astype(np.complex128)
        fg, g = plan.eval_grad(cd)
        assert err(f, fc) <= tol_f, name
        assert err(to_np(fg).astype(np.complex128), fc) <= tol_f, name
        assert err(to_np(g).astype(np.complex128), gc) <= tol_g, name
        plan.precompute(cd, with_grad=True)
        fs, gs = plan.eval_grad_stored()
        assert err(to_np(gs).astype(np.complex128), gc) <= tol_g, name
        plan.precompute(cd)
        assert err(to_np(plan.eval_stored()).astype(np.complex128), fc) <= tol_f, name


@pytest.mark.parametrize("N,sigma", [((16, 16, 16), 2.0), ((12, 16, 10), 2.0), ((10, 14, 18), 1.5)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_window_derivative_gradient(N, sigma, prec, monkeypatch):
    """eval_grad_window (one transform, derivative of the window) against the
    CPU restatement of the same method (element-wise) and against the direct
    sum's gradient (at m + 1 it meets the i k-method's tolerance at m);
    power-of-two grids take the fused transform, the others cuFFT; the
    stored variant and the value output agree with eval."""
    from paper_1605_01244_gb300 import Plan
    monkeypatch.delenv("GBNFFT_GATHER", raising=False)
    c = wl.gaussian_coeffs(N, 3.0, seed=60)
    x = wl.mixed_points(800, 0.05, seed=61)
    fd, gd = oracle.forward_grad(c, x)
    # the method's error falls by about exp(-2 pi sqrt(1 - 1/sigma)) per unit of m
    tols = {2.0: ((6, 2e-10), (7, 1e-11)), 1.5: ((6, 2e-9), (7, 1e-10))}[sigma]
    for m, tol_d in tols if prec == "f64" else ((4, 5e-6), (5, 5e-6)):
        plan = Plan(N, len(x), m=m, sigma=sigma, precision=prec)
        plan.set_points(to_dev(x))
        cd = to_dev(c, CD[prec])
        f, g = plan.eval_grad_window(cd)
        f = to_np(f).astype(np.complex128)
        g = to_np(g).astype(np.complex128)
        fw, gw = nfft_cpu.forward_grad_window(c, x, plan.n, m)
        if prec == "f64":
            assert max_rel(g, gw) <= 1e-12, m
            assert max_rel(f, fw) <= 1e-13, m
        else:
            assert rel_l2(g, gw) <= 2e-6, m
        for d in range(3):
            assert rel_l2(g[:, d], gd[:, d]) <= tol_d, (m, d)
        fe = to_np(plan.eval(cd)).astype(np.complex128)
        assert max_rel(f, fe) <= (5e-14 if prec == "f64" else 1e-6)   # different tap order
        plan.precompute(cd)
        fs, gs = plan.eval_grad_window_stored()
        assert max_rel(to_np(gs).astype(np.complex128), g) <= (1e-14 if prec == "f64" else 1e-6)
        _, g2 = plan.eval_grad_window(cd, want_f=False)
        assert max_rel(to_np(g2).astype(np.complex128), g) <= (1e-14 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_precompute_then_stored_evaluations(prec):
    """One transform of c, then value and gradient at several point sets
    (smaller than the plan's capacity) match eval / eval_grad."""
    from paper_1605_01244_gb300 import Plan
    from paper_1605_01244_gb300._lib import NFFT3_ERR_NO_COEFFS
    N = (16, 12, 20)
    c = to_dev(wl.gaussian_coeffs(N, 1e9, seed=24), CD[prec])
    plan = Plan(N, 1000, m=5, precision=prec)
    ref = Plan(N, 1000, m=5, precision=prec)
    tol = 1e-13 if prec == "f64" else 2e-6
    with pytest.raises(NFFTError) as e:
        plan.set_points(to_dev(wl.uniform_points(1000, seed=25)))
        plan.eval_stored()
    assert e.value.code == NFFT3_ERR_NO_COEFFS
    plan.precompute(c, with_grad=True)
    for M, seed in ((1000, 26), (333, 27), (1, 28)):
        x = to_dev(wl.mixed_points(M, 0.04, seed=seed))
        plan.set_num_points(M)
        plan.set_points(x)
        f = to_np(plan.eval_stored()).astype(np.complex128)
        fg, g = plan.eval_grad_stored()
        ref.set_num_points(M)
        ref.set_points(x)
        fr, gr = ref.eval_grad(c)
        fr = to_np(fr).astype(np.complex128)
        gr = to_np(gr).astype(np.complex128)
        assert max_rel(f, fr) <= tol and max_rel(to_np(fg).astype(np.complex128), fr) <= tol
        assert max_rel(to_np(g).astype(np.complex128), gr) <= tol
    # eval overwrites the stored grids
    plan.eval(c)
    with pytest.raises(NFFTError):
        plan.eval_stored()
    with pytest.raises(ValueError):
        plan.set_num_points(1001)


@pytest.mark.parametrize("sigma", [2.0, 1.5])
def test_pruned_and_full_fft_agree(sigma, monkeypatch):
    """The default transform skips the planes l1 outside the band (2D FFTs on
    the in-band planes, then 1D along l1); GBNFFT_FFT=full uses one 3D plan.
    eval, eval_grad and adjoint must agree with each other and the CPU NFFT."""
    from paper_1605_01244_gb300 import Plan
    N = (12, 10, 14)
    c = wl.gaussian_coeffs(N, 1e9, seed=40)
    x = wl.mixed_points(700, 0.05, seed=41)
    fr = wl.rng(42).standard_normal(700) + 0j
    out = {}
    for mode in ("pruned", "full"):
        if mode == "full":
            monkeypatch.setenv("GBNFFT_FFT", "full")
        else:
            monkeypatch.delenv("GBNFFT_FFT", raising=False)
        plan = Plan(N, len(x), m=5, sigma=sigma, precision="f64")
        plan.set_points(to_dev(x))
        f = to_np(plan.eval(to_dev(c)))
        _, g = plan.eval_grad(to_dev(c))
        h = to_np(plan.adjoint(to_dev(fr)))
        out[mode] = (f, to_np(g), h)
    fc, gc = nfft_cpu.forward_grad(c, x, plan.n, 5)
    hc = nfft_cpu.adjoint(fr, x, N, plan.n, 5)
    # 7-smooth, non-power-of-two sizes at sigma = 1.5 round a little more
    for mode in out:
        f, g, h = out[mode]
        assert max_rel(f, fc) <= 3e-13, mode
        assert max_rel(g, gc) <= 3e-13, mode
        assert max_rel(h, hc) <= 1e-12, mode


@pytest.mark.parametrize("prec,m,N", [("f64", 6, (24, 20, 32)), ("f64", 8, (8, 8, 8)), ("f64", 1, (16, 10, 12)),
                                      ("f64", 7, (20, 24, 16)), ("f64", 4, (32, 32, 32)), ("f64", 8, (24, 16, 20)),
                                      ("f64", 6, (8, 8, 8)), ("f32", 3, (24, 20, 32)), ("f32", 8, (10, 12, 8))])
def test_tiled_spread_matches_direct_and_cpu(prec, m, N, monkeypatch):
    """The adjoint's tile spread (default) against the one-thread-per-point
    spread (GBNFFT_SPREAD=direct) and the CPU NFFT restatement.  A dense
    cluster puts hundreds of points in one tile (several chunks of one tile).
    N = 8^3 gives n = 16, below the box of 20 nodes (m = 6, the line-owned
    kernel: a box row reaches the grid's row in two pieces, and box lines land
    on the same grid row twice) and of 24 nodes (m = 8, the half-box kernel,
    whose nodes wrap onto each other).  The FP64 half boxes hold an odd number
    of planes at m = 1 and m = 7 (one warp then owns a single plane)."""
    from paper_1605_01244_gb300 import Plan
    x = np.concatenate([wl.uniform_points(900, seed=60), wl.cluster_points(1100, 0.002, seed=61)])
    g = wl.rng(62)
    f = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    out = {}
    for mode in ("tiles", "direct"):
        if mode == "direct":
            monkeypatch.setenv("GBNFFT_SPREAD", "direct")
        else:
            monkeypatch.delenv("GBNFFT_SPREAD", raising=False)
        plan = Plan(N, len(x), m=m, precision=prec)
        plan.set_points(to_dev(x))
        out[mode] = to_np(plan.adjoint(to_dev(f, CD[prec]))).astype(np.complex128)
    hc = nfft_cpu.adjoint(f, x, N, plan.n, m)
    if prec == "f64":
        assert max_rel(out["tiles"], out["direct"]) <= 1e-12
        assert max_rel(out["tiles"], hc) <= 1e-12
    else:
        # FP32 sums of ~1000 contributions per node in the cluster: both spreads
        # round at the FP32 level, in different orders; the tiled one may not be
        # less accurate than the direct one
        e_tiles, e_direct = rel_l2(out["tiles"], hc), rel_l2(out["direct"], hc)
        assert e_tiles <= max(2 * e_direct, 1e-6), (e_tiles, e_direct)


@pytest.mark.parametrize("N", [(16, 32, 8), (8, 1024, 8), (64, 64, 64)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fused_adjoint_transform(N, prec, monkeypatch):
    """The adjoint's forward DFT of the band and deconvolution as three fused
    line passes (default for power-of-two grids; double-float in the FP64
    family) against the cuFFT transform plus deconvolution kernel
    (GBNFFT_ADJ_FFT=cufft) and the CPU NFFT restatement, for line lengths 16
    to 2048."""
    from paper_1605_01244_gb300 import Plan
    x = wl.mixed_points(1500, 0.05, seed=71)
    g = wl.rng(72)
    f = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    out = {}
    for mode in ("fused", "cufft"):
        if mode == "cufft":
            monkeypatch.setenv("GBNFFT_ADJ_FFT", "cufft")
        else:
            monkeypatch.delenv("GBNFFT_ADJ_FFT", raising=False)
        plan = Plan(N, len(x), m=5, precision=prec)
        plan.set_points(to_dev(x))
        out[mode] = to_np(plan.adjoint(to_dev(f, CD[prec]))).astype(np.complex128)
    hc = nfft_cpu.adjoint(f, x, N, plan.n, 5)
    if prec == "f64":
        assert max_rel(out["fused"], hc) <= 1e-12
        assert max_rel(out["fused"], out["cufft"]) <= 1e-12
    else:
        assert rel_l2(out["fused"], hc) <= 2e-6
        assert rel_l2(out["fused"], out["cufft"]) <= 2e-6
