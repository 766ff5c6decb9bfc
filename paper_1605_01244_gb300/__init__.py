"""gbnfft: 3D nonequispaced FFT (type-2 NFFT, its gradient and adjoint) on one GB300.

Evaluates f_j = sum_k c_k exp(2 pi i k.x_j) (Caliari & Zuccher, INFFTM,
eq. (fs) and Sec. 2.2.1) with hand-written sm_103a CUDA kernels behind the C
ABI of ``include/gbnfft.h``.  The CUDA library is loaded on first use of a
plan; there is no CPU fallback.
"""
from __future__ import annotations

__all__ = ["Plan", "choose_m", "NFFTError", "NFFTEval", "physical_to_torus"]


def __getattr__(name):
    if name in ("Plan", "choose_m"):
        from . import nfft
        return getattr(nfft, name)
    if name == "NFFTError":
        from ._lib import NFFTError
        return NFFTError
    if name == "NFFTEval":
        from .autograd import NFFTEval
        return NFFTEval
    if name == "physical_to_torus":
        from .mapping import physical_to_torus
        return physical_to_torus
    raise AttributeError(name)
