"""Plain CPU NFFT: OpenMP C steps (``nfft_omp.c``) around scipy's FFT -- TEST INFRASTRUCTURE.

Only tests and ``bench.py``'s CPU-baseline legs use this module; the product
never imports it.  It runs the NFFT of the paper's Sec. 2.2.1 (cost
O(N log N + M |log eps|^3)) on the host cores, FP64, with the Kaiser-Bessel
window of ``nfft_cpu.py``: deconvolve and zero-pad (C), unnormalised inverse
FFT of the n1 x n2 x n3 grid (scipy.fft, pocketfft, with ``workers`` threads),
window gather (C); the adjoint runs the transposes (C spread, scipy forward
FFT, C deconvolution).  Each call returns the result and the seconds spent
in each step.
"""
from __future__ import annotations

import ctypes
import os
import threading
import time

import numpy as np
import scipy.fft

from . import _BUILD, build

_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(os.path.join(_BUILD, "libcpunfft.so"))
            dp = ctypes.POINTER(ctypes.c_double)
            I, L = ctypes.c_int, ctypes.c_int64
            lib.cpu_nfft_set_threads.argtypes = [I]
            lib.cpu_nfft_set_threads.restype = None
            lib.cpu_nfft_threads.argtypes = []
            lib.cpu_nfft_threads.restype = I
            lib.cpu_nfft_tables.argtypes = [I, I, I, dp]
            lib.cpu_nfft_tables.restype = None
            lib.cpu_nfft_deconv.argtypes = [I, I, I, I, I, I, dp, dp, dp, dp, dp]
            lib.cpu_nfft_deconv.restype = None
            lib.cpu_nfft_deconv_adj.argtypes = [I, I, I, I, I, I, dp, dp, dp, dp, dp]
            lib.cpu_nfft_deconv_adj.restype = None
            lib.cpu_nfft_gather.argtypes = [I, I, I, I, I, I, dp, L, dp, I, dp]
            lib.cpu_nfft_gather.restype = None
            lib.cpu_nfft_spread.argtypes = [I, I, I, I, I, I, dp, L, dp, dp, I]
            lib.cpu_nfft_spread.restype = None
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def host_cores() -> int:
    """Cores this process may run on."""
    return len(os.sched_getaffinity(0))


def _tables(N, n, m):
    lib = _load()
    out = []
    for Nd, nd in zip(N, n):
        t = np.empty(Nd, dtype=np.float64)
        lib.cpu_nfft_tables(int(Nd), int(nd), int(m), _p(t))
        out.append(t)
    return out


class _Threads:
    """OpenMP thread count for the duration of one call (the count is a
    per-thread setting shared with the direct-sum library; it is restored)."""

    def __init__(self, threads):
        self.threads = int(threads)

    def __enter__(self):
        self.lib = _load()
        self.saved = self.lib.cpu_nfft_threads()
        self.lib.cpu_nfft_set_threads(self.threads)
        return self.lib

    def __exit__(self, *exc):
        self.lib.cpu_nfft_set_threads(self.saved)


def forward(c, x, n, m: int, threads: int | None = None):
    """f_j ~ sum_k c_k exp(2 pi i k.x_j) by the NFFT on `threads` host cores
    (default: all).  Returns (f, {"deconv": s, "fft": s, "gather": s, "tables": s})."""
    threads = threads or host_cores()
    with _Threads(threads) as lib:
        return _forward(lib, c, x, n, m, threads)


def _forward(lib, c, x, n, m, threads):
    c = np.ascontiguousarray(c, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    N = c.shape
    n = tuple(int(v) for v in n)
    t = {}
    t0 = time.perf_counter()
    d = _tables(N, n, m)
    t["tables"] = time.perf_counter() - t0
    G = np.empty(n, dtype=np.complex128)
    t0 = time.perf_counter()
    lib.cpu_nfft_deconv(*N, *n, _p(c), _p(d[0]), _p(d[1]), _p(d[2]), _p(G))
    t["deconv"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    g = scipy.fft.ifftn(G, norm="forward", overwrite_x=True, workers=threads)   # unnormalised e^{+}
    t["fft"] = time.perf_counter() - t0
    g = np.ascontiguousarray(g)
    f = np.empty(x.shape[0], dtype=np.complex128)
    t0 = time.perf_counter()
    lib.cpu_nfft_gather(*N, *n, _p(g), x.shape[0], _p(x), int(m), _p(f))
    t["gather"] = time.perf_counter() - t0
    return f, t


def adjoint(f, x, N, n, m: int, threads: int | None = None):
    """h_k ~ sum_j f_j exp(-2 pi i k.x_j) by the transposed NFFT steps.
    Returns (h (N1, N2, N3), {"spread": s, "fft": s, "deconv": s, "tables": s})."""
    threads = threads or host_cores()
    with _Threads(threads) as lib:
        return _adjoint(lib, f, x, N, n, m, threads)


def _adjoint(lib, f, x, N, n, m, threads):
    f = np.ascontiguousarray(f, dtype=np.complex128).reshape(-1)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    N = tuple(int(v) for v in N)
    n = tuple(int(v) for v in n)
    t = {}
    t0 = time.perf_counter()
    d = _tables(N, n, m)
    t["tables"] = time.perf_counter() - t0
    H = np.empty(n, dtype=np.complex128)
    t0 = time.perf_counter()
    lib.cpu_nfft_spread(*N, *n, _p(H), x.shape[0], _p(x), _p(f), int(m))
    t["spread"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Hk = np.ascontiguousarray(scipy.fft.fftn(H, overwrite_x=True, workers=threads))  # unnormalised e^{-}
    t["fft"] = time.perf_counter() - t0
    h = np.empty(N, dtype=np.complex128)
    t0 = time.perf_counter()
    lib.cpu_nfft_deconv_adj(*N, *n, _p(Hk), _p(d[0]), _p(d[1]), _p(d[2]), _p(h))
    t["deconv"] = time.perf_counter() - t0
    return h, t
