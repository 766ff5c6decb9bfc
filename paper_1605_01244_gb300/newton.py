"""Vortex-core locator: Newton iteration onto the zeros of psi.

Each iteration sets the current points on the plan, evaluates psi and its
gradient with ``eval_grad`` and applies the minimum-norm Gauss-Newton step
dx = -J^T (J J^T)^{-1} F (``nfft3_newton_step``, F = (Re psi, Im psi),
J = [Re grad psi; Im grad psi]) to every point still active.  Converged
points are then de-duplicated (``nfft3_dedupe``).  The paper thresholds
rho = |psi|^2 on refined grids instead (Sec. 4.3, sftubeeval3).

Coordinates are torus coordinates (see ``mapping``); lengths are in torus
units.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from .nfft import Plan

ACTIVE, CONVERGED, SINGULAR, DIVERGED = 0, 1, 2, 3


@dataclass
class NewtonResult:
    x: torch.Tensor          # (M, 3) float64, final points
    status: torch.Tensor     # (M,) int32: ACTIVE (not converged), CONVERGED, SINGULAR, DIVERGED
    resid: torch.Tensor      # (M,) float64, |psi| at the last evaluation
    iterations: int


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def locate(plan: Plan, c: torch.Tensor, seeds: torch.Tensor, tol: float | None = None,
           max_iter: int = 30, max_step: float | None = None, precomputed: bool = False,
           gradient: str = "window") -> NewtonResult:
    """Newton from ``seeds`` (M x 3 float64 CUDA tensor; the plan's capacity must be >= M).

    The series is deconvolved and transformed once (``precompute``; skipped
    when ``precomputed``), then every iteration is a set_points + stored
    gather of psi and grad psi + the step kernel.  gradient="window" takes the
    Jacobian from the derivative of the window (one stored grid); "series"
    from the i k-weighted series (four stored grids, ``precompute`` with
    with_grad).  The converged points are zeros of psi itself, so the
    Jacobian's approximation error only affects the iteration count.
    tol: |psi| below which a point is converged (default 1e-10 for FP64 plans,
    1e-5 for mixed).  max_step: largest accepted step (default two coarse
    cells, 2 / max N_d).
    """
    if tol is None:
        tol = 1e-10 if plan.precision == "f64" else 1e-5
    if max_step is None:
        max_step = 2.0 / max(plan.N)
    M = seeds.shape[0]
    if plan.M != M:
        plan.set_num_points(M)
    if gradient not in ("window", "series"):
        raise ValueError("gradient must be 'window' or 'series'")
    if not precomputed:
        plan.precompute(c, with_grad=gradient == "series")
    x = seeds.detach().to(torch.float64).clone().contiguous()
    status = torch.zeros(M, dtype=torch.int32, device=x.device)
    resid = torch.full((M,), float("inf"), dtype=torch.float64, device=x.device)
    prec = 64 if plan.precision == "f64" else 32
    it = 0
    for it in range(1, max_iter + 1):
        plan.set_points(x)
        f, g = plan.eval_grad_window_stored() if gradient == "window" else plan.eval_grad_stored()
        _lib.call("nfft3_newton_step", prec, M, _p(x), _p(f), _p(g), _p(status), _p(resid),
                  float(tol), float(max_step), ctypes.c_void_p(plan.stream.cuda_stream))
        if not bool((status == ACTIVE).any()):
            break
    return NewtonResult(x, status, resid, it)


def dedupe(x: torch.Tensor, status: torch.Tensor, radius: float,
           stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Boolean mask of converged points kept after merging those within ``radius``."""
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    keep = torch.zeros(x.shape[0], dtype=torch.int32, device=x.device)
    _lib.call("nfft3_dedupe", x.shape[0], _p(x.contiguous()), _p(status.contiguous()), float(radius),
              _p(keep), ctypes.c_void_p(s.cuda_stream))
    return keep.bool()
