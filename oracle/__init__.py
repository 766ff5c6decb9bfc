"""FP64 CPU oracle for the 3D truncated Fourier series and its NFFT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The product
library (``paper_1605_01244_gb300``) never imports, links or executes it, and
this package imports nothing from the product.

Contents
--------
``direct.c`` (compiled to ``_build/liboracle.so``)
    Plain FP64 direct sums, the authority for parity:
    forward  f_j = sum_k c_k e^{+2 pi i k.x_j}     (paper eq. (fs)/(Fs), Sec. 2.2)
    gradient d_d f_j = sum_k 2 pi i k_d c_k e^{..} (paper eq. (Lambda))
    adjoint  h_k = sum_j f_j e^{-2 pi i k.x_j}     (transpose of the above; also at
                                                    selected k over many points)
``nfft_cpu.py``
    A plain, unblocked numpy restatement of the NFFT approximation of the
    same sums (deconvolve / oversampled FFT / window sum), used to pin the
    window mathematics and as a same-algorithm reference.
``nfft_omp.c`` + ``cpu_nfft.py``
    The plain CPU NFFT (OpenMP C steps, scipy's FFT), the timed CPU baseline
    of the method.
``mp_reference.py``
    Arbitrary-precision brute force for tiny cases (pins the C direct sum).

Conventions: coefficients are complex128 arrays of shape (N1, N2, N3) in
centred order, entry (i1, i2, i3) <-> k_d = i_d - N_d/2; points are float64
arrays of shape (M, 3) on the torus (any real value; the series is 1-periodic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def _compile(src: str, so: str, force: bool) -> str:
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    os.makedirs(_BUILD, exist_ok=True)
    tmp = so + ".tmp%d" % os.getpid()
    # No -ffast-math: the oracle keeps IEEE semantics and the libm cos/sin.
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    """Compile ``direct.c`` (``_build/liboracle.so``) and the plain CPU NFFT
    ``nfft_omp.c`` (``_build/libcpunfft.so``) with gcc/OpenMP; returns the
    direct-sum library's path."""
    _compile(os.path.join(_HERE, "nfft_omp.c"), os.path.join(_BUILD, "libcpunfft.so"), force)
    return _compile(os.path.join(_HERE, "direct.c"), _SO, force)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_forward_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                                ctypes.c_int64, dp, dp, dp]
            lib.oracle_forward_grad.restype = None
            lib.oracle_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int64, dp, dp, dp]
            lib.oracle_adjoint.restype = None
            lib.oracle_adjoint_at.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int64,
                                              dp, dp, dp]
            lib.oracle_adjoint_at.restype = None
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(c, x):
    c = np.ascontiguousarray(c, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    if c.ndim != 3:
        raise ValueError("c must have shape (N1, N2, N3)")
    if any(n % 2 for n in c.shape):
        raise ValueError("N_d must be even")
    return c, x


def forward(c, x) -> np.ndarray:
    """Direct FP64 sum f_j = sum_k c_k exp(2 pi i k.x_j); returns complex128 (M,)."""
    c, x = _prep(c, x)
    M = x.shape[0]
    f = np.zeros(M, dtype=np.complex128)
    if M:
        _load().oracle_forward_grad(*c.shape, _dptr(c), M, _dptr(x), _dptr(f), None)
    return f


def forward_grad(c, x):
    """Direct FP64 series and gradient; returns (f (M,), grad (M, 3)) complex128.

    grad[j, d] = sum_k 2 pi i k_d c_k exp(2 pi i k.x_j)  (eq. (Lambda), torus units).
    """
    c, x = _prep(c, x)
    M = x.shape[0]
    f = np.zeros(M, dtype=np.complex128)
    g = np.zeros((M, 3), dtype=np.complex128)
    if M:
        _load().oracle_forward_grad(*c.shape, _dptr(c), M, _dptr(x), _dptr(f), _dptr(g))
    return f, g


def adjoint(f, x, N) -> np.ndarray:
    """Direct FP64 adjoint h_k = sum_j f_j exp(-2 pi i k.x_j); returns (N1, N2, N3)."""
    N = tuple(int(v) for v in N)
    f = np.ascontiguousarray(f, dtype=np.complex128).reshape(-1)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    if f.shape[0] != x.shape[0]:
        raise ValueError("f and x disagree on M")
    h = np.zeros(N, dtype=np.complex128)
    _load().oracle_adjoint(*N, x.shape[0], _dptr(x), _dptr(f), _dptr(h))
    return h


def adjoint_at(f, x, k) -> np.ndarray:
    """Direct FP64 adjoint at selected frequencies: h_q = sum_j f_j exp(-2 pi i k_q.x_j)
    for the integer triples k (nk, 3), over all points, with compensated sums."""
    f = np.ascontiguousarray(f, dtype=np.complex128).reshape(-1)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    k = np.ascontiguousarray(k, dtype=np.int32).reshape(-1, 3)
    if f.shape[0] != x.shape[0]:
        raise ValueError("f and x disagree on M")
    h = np.zeros(k.shape[0], dtype=np.complex128)
    if k.shape[0]:
        _load().oracle_adjoint_at(k.shape[0], k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), x.shape[0],
                                  _dptr(x), _dptr(f), _dptr(h))
    return h


def num_threads() -> int:
    """OpenMP threads the direct sums use."""
    return int(_load().oracle_num_threads())


def freqs(Nd: int) -> np.ndarray:
    """Frequencies k_d = i_d - N_d/2 of the centred order."""
    return np.arange(Nd) - Nd // 2
