"""Core-proposal CNN.

CPU: the numpy reference (oracle/cnn_ref.py) is pinned against torch's CPU
conv3d (a library routine) and against finite differences of its own loss.
GPU: every CUDA kernel (forward, input gradient, weight gradient, loss, Adam)
against that reference on BF16-representable inputs, the full backward of
the network against the reference chain, training lowers the loss, and the
learned proposals recover the dense judge's cores on held-out snapshots while
refining a small fraction of the cells the dense judge evaluates.
"""
import numpy as np
import pytest
import torch

from oracle import cnn_ref
from paper_1605_01244_gb300 import workloads as wl


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().double().numpy()


def test_reference_conv_matches_torch_cpu():
    g = wl.rng(80)
    for k, ci, co in ((3, 3, 5), (1, 4, 2), (3, 2, 2)):
        x = g.standard_normal((2, ci, 6, 6, 6))
        w = g.standard_normal((co, ci, k, k, k))
        b = g.standard_normal(co)
        ref = torch.nn.functional.conv3d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b),
                                         padding=k // 2).numpy()
        y = cnn_ref.conv3d(x, w, b)
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
        # adjointness of dgrad and wgrad against the forward map
        dy = g.standard_normal(y.shape)
        dx = cnn_ref.conv3d_dgrad(dy, w)
        assert abs(np.vdot(dy, cnn_ref.conv3d(x, w)) - np.vdot(dx, x)) <= 1e-10 * abs(np.vdot(dx, x))
        dw, db = cnn_ref.conv3d_wgrad(dy, x, k)
        assert abs(np.vdot(dy, cnn_ref.conv3d(x, w)) - np.vdot(dw, w)) <= 1e-10 * abs(np.vdot(dw, w))
        assert np.allclose(db, dy.sum(axis=(0, 2, 3, 4)))


def test_reference_loss_gradient_finite_differences():
    g = wl.rng(81)
    y = g.standard_normal((2, 4, 3, 3, 3))
    t = (g.random((2, 27)) < 0.3).astype(float)
    o = g.uniform(-0.5, 0.5, (2, 27, 3))
    loss, dy = cnn_ref.core_loss(y, t, o, 0.7, 4.0)
    h = 1e-6
    for idx in [(0, 0, 1, 2, 0), (1, 0, 0, 0, 2), (0, 2, 1, 1, 1), (1, 3, 2, 0, 1)]:
        yp = y.copy()
        yp[idx] += h
        ym = y.copy()
        ym[idx] -= h
        fd = (cnn_ref.core_loss(yp, t, o, 0.7, 4.0)[0] - cnn_ref.core_loss(ym, t, o, 0.7, 4.0)[0]) / (2 * h)
        assert abs(fd - dy[idx]) <= 1e-6 + 1e-5 * abs(fd)


@pytest.mark.gpu
@pytest.mark.parametrize("k,ci,co,relu", [(3, 3, 16, True), (3, 16, 16, True), (1, 16, 4, False)])
def test_conv_kernels_match_reference(k, ci, co, relu):
    import ctypes
    from paper_1605_01244_gb300 import _lib
    g = wl.rng(82 + k + ci)
    B, D = 2, 7
    x = bf16_round(np.abs(g.standard_normal((B, ci, D, D, D))) if relu else g.standard_normal((B, ci, D, D, D)))
    w = bf16_round(g.standard_normal((co, ci, k, k, k)) * 0.3)
    b = g.standard_normal(co).astype(np.float32).astype(float)
    xt = torch.from_numpy(x).to(torch.bfloat16).cuda()
    wt = torch.from_numpy(w).to(torch.bfloat16).cuda()
    bt = torch.from_numpy(b).float().cuda()
    P = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    yf = torch.empty((B, co, D, D, D), dtype=torch.float32, device="cuda")
    _lib.call("cnn_conv3d_fwd", P(xt), P(wt), P(bt), B, ci, co, D, k, int(relu), None, P(yf), None)
    ref = cnn_ref.conv3d(x, w, b)
    if relu:
        ref = np.maximum(ref, 0)
    assert np.max(np.abs(yf.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))
    dy = g.standard_normal((B, co, D, D, D))
    dyt = torch.from_numpy(dy).float().cuda()
    dy32 = dyt.double().cpu().numpy()
    dx = torch.empty((B, ci, D, D, D), dtype=torch.float32, device="cuda")
    mask = xt if relu else None
    _lib.call("cnn_conv3d_dgrad", P(dyt), P(wt), B, ci, co, D, k, P(mask), P(dx), None)
    dref = cnn_ref.conv3d_dgrad(dy32, w)
    if relu:
        dref = dref * (x > 0)
    assert np.max(np.abs(dx.cpu().numpy() - dref)) <= 1e-5 * np.max(np.abs(dref))
    dw = torch.empty((co, ci, k, k, k), dtype=torch.float32, device="cuda")
    db = torch.empty(co, dtype=torch.float32, device="cuda")
    _lib.call("cnn_conv3d_wgrad", P(dyt), P(xt), B, ci, co, D, k, P(dw), P(db), None)
    wref, bref = cnn_ref.conv3d_wgrad(dy32, x, k)
    assert np.max(np.abs(dw.cpu().numpy() - wref)) <= 1e-5 * np.max(np.abs(wref))
    assert np.max(np.abs(db.cpu().numpy() - bref)) <= 1e-5 * np.max(np.abs(bref))


@pytest.mark.gpu
@pytest.mark.parametrize("k,ci,co", [(3, 16, 16), (1, 16, 4), (3, 3, 16)])
def test_tiled_conv_kernels_several_tiles(k, ci, co, monkeypatch):
    """The shared-memory tiled kernels (8 x 8 x 4 voxel tiles) on a lattice of
    several ragged tiles, against the reference and the one-output-per-thread
    kernels (GBNFFT_CNN_NAIVE=1); with their times at the experiment's size
    (12 snapshots of 49^3 coarse nodes)."""
    import ctypes
    from paper_1605_01244_gb300 import _lib
    g = wl.rng(95 + k + ci)
    P = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    B, D = 3, 13
    x = bf16_round(np.abs(g.standard_normal((B, ci, D, D, D))))
    w = bf16_round(g.standard_normal((co, ci, k, k, k)) * 0.3)
    b = g.standard_normal(co).astype(np.float32).astype(float)
    dy = g.standard_normal((B, co, D, D, D)).astype(np.float32)
    xt = torch.from_numpy(x).to(torch.bfloat16).cuda()
    wt = torch.from_numpy(w).to(torch.bfloat16).cuda()
    bt = torch.from_numpy(b).float().cuda()
    dyt = torch.from_numpy(dy).cuda()

    def run():
        yf = torch.empty((B, co, D, D, D), dtype=torch.float32, device="cuda")
        _lib.call("cnn_conv3d_fwd", P(xt), P(wt), P(bt), B, ci, co, D, k, 1, None, P(yf), None)
        dx = torch.empty((B, ci, D, D, D), dtype=torch.float32, device="cuda")
        _lib.call("cnn_conv3d_dgrad", P(dyt), P(wt), B, ci, co, D, k, P(xt), P(dx), None)
        dw = torch.empty((co, ci, k, k, k), dtype=torch.float32, device="cuda")
        db = torch.empty(co, dtype=torch.float32, device="cuda")
        _lib.call("cnn_conv3d_wgrad", P(dyt), P(xt), B, ci, co, D, k, P(dw), P(db), None)
        return [t.double().cpu().numpy() for t in (yf, dx, dw, db)]

    yf, dx, dw, db = run()
    ref = np.maximum(cnn_ref.conv3d(x, w, b), 0)
    dref = cnn_ref.conv3d_dgrad(dy.astype(float), w) * (x > 0)
    wref, bref = cnn_ref.conv3d_wgrad(dy.astype(float), x, k)
    for got, want in ((yf, ref), (dx, dref), (dw, wref), (db, bref)):
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))
    monkeypatch.setenv("GBNFFT_CNN_NAIVE", "1")
    for got, want in zip((yf, dx, dw, db), run()):
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))
    # times at the experiment's size, tiled against one output per thread
    B, D = 12, 49
    xt = torch.zeros((B, ci, D, D, D), dtype=torch.bfloat16, device="cuda").uniform_()
    dyt = torch.zeros((B, co, D, D, D), dtype=torch.float32, device="cuda").normal_()
    ms = {}
    for mode in ("tiled", "naive"):
        if mode == "tiled":
            monkeypatch.delenv("GBNFFT_CNN_NAIVE", raising=False)
        else:
            monkeypatch.setenv("GBNFFT_CNN_NAIVE", "1")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        run()
        torch.cuda.synchronize()
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms[mode] = e0.elapsed_time(e1)
    print("conv k=%d %d->%d at 12 x 49^3, fwd + dgrad + wgrad: tiled %.2f ms, one output per thread %.2f ms"
          % (k, ci, co, ms["tiled"], ms["naive"]))


@pytest.mark.gpu
def test_network_gradients_match_reference_chain():
    from paper_1605_01244_gb300.cnn import CoreCNN, LAYERS
    g = wl.rng(90)
    B, D = 2, 6
    model = CoreCNN(seed=3)
    x = torch.from_numpy(g.standard_normal((B, 3, D, D, D))).to(torch.bfloat16).cuda()
    t = torch.from_numpy((g.random((B, D ** 3)) < 0.2).astype(np.float32)).cuda()
    o = torch.from_numpy(g.uniform(-0.5, 0.5, (B, D ** 3, 3)).astype(np.float32)).cuda()
    loss, grads = model.gradients(x, t, o, lam=0.5, pos_weight=3.0)
    # reference: the same chain in FP64 with BF16-rounded weights and BF16 activations
    a = x.double().cpu().numpy()
    acts = [a]
    for li, (ci, co, k, relu) in enumerate(LAYERS):
        w = model.wbf[li].double().cpu().numpy()
        z = cnn_ref.conv3d(acts[-1], w, model.b[li].double().cpu().numpy())
        if relu:
            acts.append(bf16_round(np.maximum(z, 0)))
        else:
            head = z
    rloss, dy = cnn_ref.core_loss(head, t.double().cpu().numpy(), o.double().cpu().numpy(), 0.5, 3.0)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss)
    rgrads = [None] * len(LAYERS)
    for li in range(len(LAYERS) - 1, -1, -1):
        ci, co, k, _ = LAYERS[li]
        dw, db = cnn_ref.conv3d_wgrad(dy, acts[li], k)
        rgrads[li] = (dw, db)
        if li > 0:
            dy = cnn_ref.conv3d_dgrad(dy, model.wbf[li].double().cpu().numpy()) * (acts[li] > 0)
    for li in range(len(LAYERS)):
        gw = grads[li].double().cpu().numpy()
        gb = grads[len(LAYERS) + li].double().cpu().numpy()
        assert np.max(np.abs(gw - rgrads[li][0])) <= 1e-4 * np.max(np.abs(rgrads[li][0])) + 1e-9, li
        assert np.max(np.abs(gb - rgrads[li][1])) <= 1e-4 * np.max(np.abs(rgrads[li][1])) + 1e-9, li


@pytest.mark.gpu
def test_adam_kernel_matches_formula():
    import ctypes
    from paper_1605_01244_gb300 import _lib
    g = wl.rng(91)
    n = 1000
    w = torch.from_numpy(g.standard_normal(n).astype(np.float32)).cuda()
    w0 = w.clone()
    grad = torch.from_numpy(g.standard_normal(n).astype(np.float32)).cuda()
    m1 = torch.zeros(n, device="cuda")
    m2 = torch.zeros(n, device="cuda")
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    for step in (1, 2):
        _lib.call("cnn_adam", P(w), P(wb), P(grad), P(m1), P(m2), n, ctypes.c_float(1e-2), ctypes.c_float(0.9),
                  ctypes.c_float(0.999), ctypes.c_float(1e-8), step, None)
    # two identical gradient steps: m1 = (1 - .9^2) g, m2 = (1 - .999^2) g^2 at step 2
    gg = grad.double().cpu().numpy()
    wr = w0.double().cpu().numpy()
    a = np.zeros(n)
    v = np.zeros(n)
    for step in (1, 2):
        a = 0.9 * a + 0.1 * gg
        v = 0.999 * v + 0.001 * gg * gg
        wr = wr - 1e-2 * (a / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    assert np.max(np.abs(w.double().cpu().numpy() - wr)) <= 1e-5
    assert torch.equal(wb, w.to(torch.bfloat16))


@pytest.mark.gpu
def test_learned_proposals_recover_the_dense_cores():
    """Train on 12 swept snapshots (N = 64^3), evaluate on 4 held-out offsets a.
    The method without the network is the dense judge (every fine cell of the
    box); the learned path must recover >= 99 % of its core points while
    refining at most 15 % of the cells.  The rho-threshold baseline is
    reported alongside."""
    from paper_1605_01244_gb300 import core_experiment
    out = core_experiment.run(N=64, r=6)
    print(out)
    assert out["loss_last"] < 0.5 * out["loss_first"]
    for res in out["heldout"]:
        assert res["learned"]["recall"] >= 0.99, res
        assert res["learned"]["cells"] <= 0.15 * res["total_cells"], res
    # what the network buys over the rho-threshold tube criterion (both set for
    # full recall on the training snapshots): fewer cells to refine
    learned = sum(r["learned"]["cells"] for r in out["heldout"])
    rho = sum(r["rho"]["cells"] for r in out["heldout"])
    print("held-out cells refined: learned %d, rho threshold %d" % (learned, rho))
    assert learned <= rho
