"""One- and two-dimensional NFFT (the paper's infft and infft2): FP64
evaluation of a 1D or 2D truncated Fourier series at arbitrary points with the
same window as the 3D path (``nfft_lowdim_eval``)."""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def nfft_eval(c: torch.Tensor, x: torch.Tensor, m: int = 6, sigma: float = 2.0,
              stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """c: (N1,) or (N1, N2) complex128 CUDA, centred order; x: (M,) or (M, 1)
    for 1D, (M, 2) for 2D, float64 CUDA (torus coordinates).  Returns f (M,)."""
    if c.dtype != torch.complex128 or not c.is_cuda or c.dim() not in (1, 2):
        raise ValueError("c must be a 1-D or 2-D complex128 CUDA tensor")
    dim = c.dim()
    x = x.to(torch.float64).reshape(-1, dim).contiguous()
    c = c.contiguous()
    N = (ctypes.c_int * dim)(*c.shape)
    ws_bytes = _lib.lib().nfft_lowdim_workspace_bytes(dim, N, int(m), float(sigma))
    if ws_bytes == 0:
        raise ValueError("invalid sizes, m or sigma")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=c.device)
    M = x.shape[0]
    f = torch.empty(M, dtype=torch.complex128, device=c.device)
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _lib.call("nfft_lowdim_eval", dim, N, M, int(m), float(sigma), _p(x), _p(c), _p(f), _p(ws), ws_bytes, st)
    return f
