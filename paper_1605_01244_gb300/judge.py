"""Dense local-grid judge of vortex cores.

psi is evaluated by the NFFT on a fine R1 x R2 x R3 lattice spanning a local
box, every lattice face around which the phase of psi winds by +-2 pi is
reported (``nfft3_plaquette_crossings``), and the face centres are refined
onto the zero set by the Newton locator and de-duplicated.  The result is the
ground truth and the fallback for the learned proposals, and the referee of
their miss rate.  (The paper renders isosurfaces of rho = |psi|^2 on fine
rectilinear grids for the same purpose, Sec. 5.)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib, newton
from .nfft import Plan


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _d3(v):
    return (ctypes.c_double * 3)(*[float(a) for a in v])


@dataclass
class Crossings:
    points: torch.Tensor   # (K, 3) float64 face centres (torus coordinates)
    direction: torch.Tensor  # (K,) int32: +-(face normal 1..3), sign = winding
    psi: torch.Tensor | None = None


def lattice(R, lo, hi, device="cuda") -> torch.Tensor:
    """R1 R2 R3 x 3 lattice points lo + i h, h = (hi - lo)/(R - 1)."""
    R = tuple(int(r) for r in R)
    h = [(float(b) - float(a)) / max(r - 1, 1) for a, b, r in zip(lo, hi, R)]
    x = torch.empty((R[0] * R[1] * R[2], 3), dtype=torch.float64, device=device)
    _lib.call("nfft3_lattice_points", _p(x), R[0], R[1], R[2], _d3(lo), _d3(h),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return x


def crossings_from_samples(psi: torch.Tensor, R, lo, hi, cap: int = 1 << 22) -> Crossings:
    """Plaquette test on psi sampled at ``lattice(R, lo, hi)`` (flat, complex CUDA tensor)."""
    R = tuple(int(r) for r in R)
    h = [(float(b) - float(a)) / max(r - 1, 1) for a, b, r in zip(lo, hi, R)]
    prec = 64 if psi.dtype == torch.complex128 else 32
    out = torch.empty((cap, 3), dtype=torch.float64, device=psi.device)
    odir = torch.empty(cap, dtype=torch.int32, device=psi.device)
    count = torch.zeros(1, dtype=torch.int64, device=psi.device)
    _lib.call("nfft3_plaquette_crossings", prec, _p(psi.contiguous()), R[0], R[1], R[2], _d3(lo), _d3(h),
              _p(out), _p(odir), cap, _p(count), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    k = int(count.item())
    if k > cap:
        raise RuntimeError("%d crossings exceed the capacity %d" % (k, cap))
    return Crossings(out[:k], odir[:k], psi)


def make_plan(c: torch.Tensor, capacity: int, precision: str = "f64", eps: float | None = None) -> Plan:
    """A plan for the series c that later calls resize (set_num_points) up to ``capacity``."""
    if eps is None:
        eps = 1e-12 if precision == "f64" else 1e-6
    return Plan(c.shape, capacity, m=0, eps=eps, precision=precision)


def lattice_axes(R, lo, hi, device="cuda"):
    """The three coordinate axes of ``lattice(R, lo, hi)`` (same values)."""
    R = tuple(int(r) for r in R)
    h = [(float(b) - float(a)) / max(r - 1, 1) for a, b, r in zip(lo, hi, R)]
    return [float(lo[d]) + torch.arange(R[d], dtype=torch.float64, device=device) * h[d] for d in range(3)]


def dense_crossings(c: torch.Tensor, R, lo, hi, precision: str = "f64", plan: Plan | None = None,
                    precomputed: bool = False, method: str = "nfft") -> Crossings:
    """Evaluate the series c on the lattice and run the plaquette test.
    method="nfft": the NFFT at the lattice points; "grid": the exact
    rectilinear-grid evaluation (three dense contractions, ``grid.grid_eval``)."""
    R = tuple(int(r) for r in R)
    M = R[0] * R[1] * R[2]
    if method == "grid":
        from .grid import grid_eval
        cc = c if precision == "f64" else c.to(torch.complex64)
        psi = grid_eval(cc, *lattice_axes(R, lo, hi, c.device)).reshape(-1)
        return crossings_from_samples(psi, R, lo, hi)
    if method != "nfft":
        raise ValueError("method must be 'nfft' or 'grid'")
    if plan is None:
        plan = make_plan(c, M, precision)
    plan.set_num_points(M)
    if not precomputed:
        plan.precompute(c, with_grad=False)
    x = lattice(R, lo, hi, c.device)
    plan.set_points(x)
    psi = plan.eval_stored()
    del x
    return crossings_from_samples(psi, R, lo, hi)


def dense_cores(c: torch.Tensor, R, lo, hi, precision: str = "f64", merge_radius: float | None = None,
                plan: Plan | None = None):
    """Core points: crossings refined by Newton, de-duplicated.  Returns (points, crossings).

    One plan serves the lattice evaluation and the Newton iterations; the
    series is transformed once (one grid: Newton differentiates the window)."""
    R = tuple(int(r) for r in R)
    if plan is None:
        plan = make_plan(c, R[0] * R[1] * R[2], precision)
    plan.precompute(c)
    cr = dense_crossings(c, R, lo, hi, precision, plan=plan, precomputed=True)
    if cr.points.shape[0] == 0:
        return cr.points, cr
    res = newton.locate(plan, c, cr.points, precomputed=True)
    if merge_radius:
        keep = newton.dedupe(res.x, res.status, merge_radius)
    else:
        keep = res.status == newton.CONVERGED
    return res.x[keep], cr


def recall(found: torch.Tensor, truth: torch.Tensor, radius: float) -> float:
    """Fraction of truth points with a found point within ``radius`` (periodic distance)."""
    if truth.shape[0] == 0:
        return 1.0
    if found.shape[0] == 0:
        return 0.0
    hit = torch.zeros(truth.shape[0], dtype=torch.bool, device=truth.device)
    for s in range(0, found.shape[0], 4096):
        d = truth[:, None, :] - found[None, s:s + 4096, :]
        d = d - torch.round(d)
        hit |= (d.pow(2).sum(-1) <= radius * radius).any(dim=1)
    return float(hit.float().mean().item())
