"""Vortex-tube evaluation: the paper's refinement of the density inside vortex
tubes (Sec. 4.3, sftubeeval3), on the GPU.

Start from the points of the equispaced grid (here: the nodes of a box
lattice with R points per dimension, spacing h) and their values psi.  For
each level i: keep the points with rho = |psi|^2 <= rhobar[i], replace every
kept point by the 27 points of the step-h/3 grid centred on it
(``nfft3_tube_refine``), divide h by 3, and evaluate psi at the new points by
the NFFT.  The result is the last level's points with their rho; the
vortex cores are where rho is smallest (the paper then keeps rho <= 0.0012,
Sec. 5).  The series is transformed once; the plan's capacity bounds one
evaluation batch, and larger levels are evaluated in batches.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib, judge
from .nfft import Plan


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def evaluate_points(plan: Plan, x: torch.Tensor) -> torch.Tensor:
    """psi at the points x (K x 3 float64 CUDA) from the plan's stored grid,
    in batches of the plan's capacity."""
    K = x.shape[0]
    out = torch.empty(K, dtype=plan.cdtype, device=x.device)
    cap = plan.capacity
    for a in range(0, K, cap):
        b = min(K, a + cap)
        plan.set_num_points(b - a)
        plan.set_points(x[a:b])
        plan.eval_stored(out=out[a:b])
    return out


def refine(x: torch.Tensor, psi: torch.Tensor, rhobar: float, h, precision: str = "f64",
           stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """One refinement: the 27-point children (step h/3) of the points with
    |psi|^2 <= rhobar, in input order."""
    M = x.shape[0]
    prec = 64 if precision == "f64" else 32
    ws = torch.empty(max(1, _lib.lib().nfft3_tube_workspace_bytes(M)), dtype=torch.uint8, device=x.device)
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    kept = ctypes.c_int64()
    hd = (ctypes.c_double * 3)(*[float(v) for v in h])
    # first call with no output buffer: the number of kept points
    code = _lib.lib().nfft3_tube_refine(prec, _p(x), _p(psi), M, float(rhobar), hd, None, 0, ctypes.byref(kept),
                                        _p(ws), ws.numel(), st)
    if code not in (0, _lib.NFFT3_ERR_TOO_LARGE):
        _lib.check("nfft3_tube_refine", code)
    out = torch.empty((27 * kept.value, 3), dtype=torch.float64, device=x.device)
    if kept.value:
        _lib.check("nfft3_tube_refine",
                   _lib.lib().nfft3_tube_refine(prec, _p(x), _p(psi), M, float(rhobar), hd, _p(out), out.shape[0],
                                                ctypes.byref(kept), _p(ws), ws.numel(), st))
    return out


def tube_eval(c: torch.Tensor, rhobar, R, lo, hi, precision: str = "f64", plan: Plan | None = None,
              m: int | None = None):
    """Tube points and rho after len(rhobar) refinements, starting from the
    R1 x R2 x R3 lattice spanning [lo, hi] (torus coordinates).  Returns
    (points (K, 3) float64, rho (K,) float64)."""
    R = tuple(int(r) for r in R)
    if plan is None:
        cap = R[0] * R[1] * R[2]
        plan = (judge.make_plan(c, cap, precision) if m is None
                else Plan(c.shape, cap, m=m, precision=precision))
    plan.precompute(c)
    x = judge.lattice(R, lo, hi, device=c.device)
    h = [(float(b) - float(a)) / max(r - 1, 1) for a, b, r in zip(lo, hi, R)]
    psi = evaluate_points(plan, x)
    for rb in rhobar:
        x = refine(x, psi, rb, h, precision)
        h = [v / 3.0 for v in h]
        psi = evaluate_points(plan, x) if x.shape[0] else psi[:0]
    rho = psi.real.double() ** 2 + psi.imag.double() ** 2
    return x, rho
