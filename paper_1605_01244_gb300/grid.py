"""Exact evaluation of the series on a rectilinear grid (the paper's
igridftn, Sec. 2.1): f[i1, i2, i3] = sum_k c_k exp(2 pi i k.(y1[i1], y2[i2],
y3[i3])) by three dense contractions (``nfft3*_grid_eval``).  Cost
O(N^3 M + N^2 M^2 + N M^3) for M points per dimension: for a full lattice
of a local box this is a few large GEMMs, against the NFFT's M^3 window sums."""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def grid_eval(c: torch.Tensor, y1: torch.Tensor, y2: torch.Tensor, y3: torch.Tensor,
              stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """c: (N1, N2, N3) complex128 or complex64 CUDA; y_d: 1-D float64 CUDA
    torus coordinates.  Returns f of shape (M1, M2, M3), dtype of c."""
    if c.dtype not in (torch.complex128, torch.complex64) or not c.is_cuda or c.dim() != 3:
        raise ValueError("c must be a 3-D complex128/complex64 CUDA tensor")
    c = c.contiguous()
    ys = [y.to(torch.float64).contiguous() for y in (y1, y2, y3)]
    prec = 64 if c.dtype == torch.complex128 else 32
    N = tuple(c.shape)
    M = tuple(int(y.numel()) for y in ys)
    ws_bytes = _lib.lib().nfft3_grid_eval_workspace_bytes(prec, *N, *M)
    ws = torch.empty(max(1, ws_bytes), dtype=torch.uint8, device=c.device)
    f = torch.empty(M, dtype=c.dtype, device=c.device)
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    name = "nfft3d_grid_eval" if prec == 64 else "nfft3f_grid_eval"
    _lib.call(name, _p(c), N[0], N[1], N[2], _p(ys[0]), M[0], _p(ys[1]), M[1], _p(ys[2]), M[2], _p(f),
              _p(ws), ws.numel(), st)
    return f
