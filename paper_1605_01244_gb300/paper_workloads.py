"""The paper's own timing workloads (Sec. 2.1 and Sec. 2.2.1), on this library.

* 64^3 random complex coefficients evaluated at M = 1000 random points
  (the paper: NFFT 0.131 s MATLAB / 0.096 s Octave, one-loop sum 3.3 / 4.0 s);
* the same coefficients at the 64^3 regular grid (the paper: NFFT 2.27 s /
  2.74 s, ndcovlt 0.050 / 0.032 s, ifftn 0.010 / 0.011 s).

Each is timed with CUDA events around the whole call (plan creation outside,
FP64 family, m = 6 and 8, sigma = 2; the first call untimed), and the error is the
paper's: infinity norm against the direct sum (random points: separable
exponential tables contracted in FP64 torch) or the inverse FFT (regular grid).  ``python -m paper_1605_01244_gb300.paper_workloads``
prints one JSON line.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import workloads as wl
from .grid import grid_eval
from .nfft import Plan


def _time(fn, reps=20):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / reps * 1e-3


def direct_sum(c: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """f_j = sum_k c_k exp(2 pi i k.x_j) by the definition: per-dimension
    tables exp(2 pi i k_d x_jd) (phase reduced mod 1 first), contracted."""
    tabs = []
    for d in range(3):
        k = torch.arange(c.shape[d], dtype=torch.float64, device=c.device) - c.shape[d] // 2
        ph = x[:, d:d + 1] * k[None, :]
        tabs.append(torch.exp(2j * torch.pi * (ph - torch.round(ph))))
    return torch.einsum("abc,ja,jb,jc->j", c, tabs[0], tabs[1], tabs[2])


def run(seed: int = 1605):
    N = (64, 64, 64)
    g = np.random.default_rng(seed)
    c = g.standard_normal(N) + 1j * g.standard_normal(N)
    cd = torch.from_numpy(c).cuda()
    out = {}
    # 1000 random points (physical domain mapped to the torus: uniform in [-1/2, 1/2))
    x = g.uniform(-0.5, 0.5, (1000, 3))
    xd = torch.from_numpy(x).cuda()
    ref = direct_sum(cd, xd).cpu().numpy()
    nodes = np.stack(np.meshgrid(*[np.arange(v) / v - 0.5 for v in N], indexing="ij"), -1).reshape(-1, 3)
    k = [np.arange(n) - n // 2 for n in N]
    sign = (-1.0) ** (k[0][:, None, None] + k[1][None, :, None] + k[2][None, None, :])
    ref_grid = (np.fft.ifftn(np.fft.ifftshift(c * sign)) * np.prod(N)).reshape(-1)
    nd = torch.from_numpy(nodes).cuda()
    for m in (6, 8):
        plan = Plan(N, len(x), m=m, sigma=2.0, precision="f64")

        def random_points():
            plan.set_points(xd)
            return plan.eval(cd)

        f, t = _time(random_points)
        err = float(np.max(np.abs(f.cpu().numpy() - ref)))
        out["random1000_m%d" % m] = {"seconds": t, "points_per_s": 1000 / t, "error_inf": err,
                                     "error_inf_rel": err / float(np.max(np.abs(ref))),
                                     "paper_seconds": {"nfft_matlab": 0.130843, "nfft_octave": 0.0957451,
                                                       "one_loop_matlab": 3.295020, "one_loop_octave": 3.95735}}
        gplan = Plan(N, nodes.shape[0], m=m, sigma=2.0, precision="f64")

        def grid_points():
            gplan.set_points(nd)
            return gplan.eval(cd)

        f, t = _time(grid_points)
        err = float(np.max(np.abs(f.cpu().numpy() - ref_grid)))
        out["grid64_nfft_m%d" % m] = {"seconds": t, "error_inf": err,
                                      "error_inf_rel": err / float(np.max(np.abs(ref_grid))),
                                      "paper_seconds": {"nfft_matlab": 2.267151, "nfft_octave": 2.74056}}
    y = torch.arange(64, dtype=torch.float64, device="cuda") / 64 - 0.5
    f, t = _time(lambda: grid_eval(cd, y, y, y))
    err = float(np.max(np.abs(f.cpu().numpy().reshape(-1) - ref_grid)))
    out["grid64_rectilinear"] = {"seconds": t, "error_inf": err,
                                 "error_inf_rel": err / float(np.max(np.abs(ref_grid))),
                                 "paper_seconds": {"ndcovlt_matlab": 0.049872, "ndcovlt_octave": 0.0321529,
                                                   "two_loops_matlab": 0.201674, "ifftn_matlab": 0.010371}}
    return out


if __name__ == "__main__":
    print(json.dumps(run()))
