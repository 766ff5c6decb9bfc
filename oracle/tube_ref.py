"""Plain numpy restatement of the vortex-tube evaluation -- TEST INFRASTRUCTURE.

Only tests use this module.  The paper's sftubeeval3 (Sec. 4.3): starting
from the points of an equispaced grid with step h, keep the points whose
density rho = |psi|^2 is at most rhobar, replace each by the 27 points of the
grid of step h/3 centred on it, and evaluate rho there; for a vector of
rhobar values repeat with the new points and h/3.  psi comes from the FP64
direct sum (``oracle.forward``).  Child order: kept points in input order,
then (a, b, c) in {-1, 0, 1}^3 with c fastest.
"""
from __future__ import annotations

import numpy as np


def density(psi):
    psi = np.asarray(psi, dtype=np.complex128)
    return psi.real * psi.real + psi.imag * psi.imag


def children(points, h):
    """The 27 points p + (a h1/3, b h2/3, c h3/3) of every row p of points."""
    h3 = np.asarray(h, dtype=np.float64) / 3.0
    off = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.float64)
    return (np.asarray(points, dtype=np.float64)[:, None, :] + off[None, :, :] * h3[None, None, :]).reshape(-1, 3)


def refine(points, psi, rhobar, h):
    keep = density(psi) <= rhobar
    return children(np.asarray(points)[keep], h)


def lattice(R, lo, hi):
    h = [(b - a) / max(r - 1, 1) for a, b, r in zip(lo, hi, R)]
    axes = [lo[d] + np.arange(R[d]) * h[d] for d in range(3)]
    return np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3), h


def tube_eval(c, rhobar, R, lo, hi, evaluate):
    """evaluate(points) -> psi.  Returns (points, rho) of the last level."""
    x, h = lattice(R, lo, hi)
    psi = evaluate(x)
    for rb in rhobar:
        x = refine(x, psi, rb, h)
        h = [v / 3.0 for v in h]
        psi = evaluate(x) if len(x) else np.zeros(0, np.complex128)
    return x, density(psi)
