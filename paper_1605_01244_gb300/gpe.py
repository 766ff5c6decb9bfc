"""Gross-Pitaevskii solver (the paper's Sec. 3, TSSP with Strang splitting)
over torch CUDA tensors: argument marshalling for ``gpe_*`` of libgbnfft.

    solver = GPE((n1, n2, n3), (L1, L2, L3))
    solver.steps(psi, tau, nsteps)      # psi: (n1, n2, n3) complex128 CUDA, in place
    mass, energy = solver.mass_energy(psi)
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


class GPE:
    """TSSP integrator of psi_t = (i/2) Lap psi + (i/2)(1 - |psi|^2) psi on a periodic box."""

    def __init__(self, n, L, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("the GPE solver needs a CUDA device (no CPU fallback exists)")
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _lib.call("gpe_plan_create", ctypes.byref(h), *self.n, *self.L, ctypes.c_void_p(self.stream.cuda_stream))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().gpe_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, psi):
        if (not isinstance(psi, torch.Tensor) or psi.dtype != torch.complex128 or psi.device != self.device
                or tuple(psi.shape) != self.n or not psi.is_contiguous()):
            raise ValueError("psi must be a contiguous complex128 tensor of shape %s on %s" % (self.n, self.device))

    def steps(self, psi: torch.Tensor, tau: float, nsteps: int) -> torch.Tensor:
        """Advance psi in place by nsteps Strang steps of size tau."""
        self._check(psi)
        _lib.call("gpe_steps", self._h, ctypes.c_void_p(psi.data_ptr()), float(tau), int(nsteps))
        return psi

    def mass_energy(self, psi: torch.Tensor):
        """(sum |psi|^2 dV, the energy of eq. (energy))."""
        self._check(psi)
        m, e = ctypes.c_double(), ctypes.c_double()
        _lib.call("gpe_mass_energy", self._h, ctypes.c_void_p(psi.data_ptr()), ctypes.byref(m), ctypes.byref(e))
        return m.value, e.value
