"""ctypes binding of libgbnfft.so (argument marshalling only).

Every entry point of ``include/gbnfft.h`` is declared here with the same name.
Loading fails loudly (ImportError/RuntimeError) when the library has not
been built; nothing in this package falls back to a CPU computation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libgbnfft.so")

NFFT3_OK = 0
NFFT3_WARN_EPS = 1
NFFT3_ERR_ARG = -1
NFFT3_ERR_ALLOC = -2
NFFT3_ERR_CUFFT = -3
NFFT3_ERR_CUDA = -4
NFFT3_ERR_NO_POINTS = -5
NFFT3_ERR_POINTS = -6
NFFT3_ERR_TOO_LARGE = -7
NFFT3_ERR_NO_COEFFS = -8

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
SIGNATURES = {
    "nfft3d_plan": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I64, _I, _D, _D, _P]),
    "nfft3f_plan": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I64, _I, _D, _D, _P]),
    "nfft3d_set_points": (_I, [_P, _P]),
    "nfft3f_set_points": (_I, [_P, _P]),
    "nfft3d_eval": (_I, [_P, _P, _P]),
    "nfft3f_eval": (_I, [_P, _P, _P]),
    "nfft3d_eval_grad": (_I, [_P, _P, _P, _P]),
    "nfft3f_eval_grad": (_I, [_P, _P, _P, _P]),
    "nfft3d_eval_grad_noalloc": (_I, [_P, _P, _P, _P]),
    "nfft3_set_deterministic": (_I, [_P, _I]),
    "gpe_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _D, _D, _D, _P]),
    "gpe_steps": (_I, [_P, _P, _D, _I]),
    "gpe_mass_energy": (_I, [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gpe_destroy": (_I, [_P]),
    "nfft3d_adjoint": (_I, [_P, _P, _P]),
    "nfft3f_adjoint": (_I, [_P, _P, _P]),
    "nfft3d_precompute": (_I, [_P, _P, _I]),
    "nfft3f_precompute": (_I, [_P, _P, _I]),
    "nfft3d_eval_stored": (_I, [_P, _P]),
    "nfft3f_eval_stored": (_I, [_P, _P]),
    "nfft3d_eval_grad_stored": (_I, [_P, _P, _P]),
    "nfft3f_eval_grad_stored": (_I, [_P, _P, _P]),
    "nfft3d_eval_points": (_I, [_P, _P, _P, _P]),
    "nfft3f_eval_points": (_I, [_P, _P, _P, _P]),
    "nfft3d_chain_x": (_I, [_P, _P, _P, _P]),
    "nfft3f_chain_x": (_I, [_P, _P, _P, _P]),
    "nfft3d_eval_grad_window": (_I, [_P, _P, _P, _P]),
    "nfft3f_eval_grad_window": (_I, [_P, _P, _P, _P]),
    "nfft3d_eval_grad_window_stored": (_I, [_P, _P, _P]),
    "nfft3f_eval_grad_window_stored": (_I, [_P, _P, _P]),
    "nfft3_set_num_points": (_I, [_P, _I64]),
    "nfft3d_eval_host": (_I, [_P, _P, _P, _P]),
    "nfft3f_eval_host": (_I, [_P, _P, _P, _P]),
    "nfft3d_destroy": (_I, [_P]),
    "nfft3f_destroy": (_I, [_P]),
    "nfft3_plan_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I64),
                             ctypes.POINTER(_I)]),
    "nfft3_set_stream": (_I, [_P, _P]),
    "nfft3_window_error": (_I, [_P, ctypes.POINTER(_D)]),
    "nfft3_sync": (_I, [_P]),
    "nfft3_error_string": (ctypes.c_char_p, [_I]),
    "nfft3_choose_m": (_I, [_D, _D]),
    "nfft3_timing_enable": (_I, [_P, _I]),
    "nfft3_timing_read": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64), ctypes.POINTER(_I64), _I]),
    "nfft3_reduce_coords": (_I, [_I, _I, _P, _I64, _P, _P, _P, _P, _P]),
    "nfft3_fma_peak": (_I, [_I, _I, _P, ctypes.POINTER(_D)]),
    "nfft3_newton_step": (_I, [_I, _I64, _P, _P, _P, _P, _P, _D, _D, _P]),
    "nfft3_dedupe": (_I, [_I64, _P, _P, _D, _P, _P]),
    "cnn_conv3d_fwd": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _I, _P, _P, _P]),
    "cnn_conv3d_dgrad": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
    "cnn_conv3d_wgrad": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
    "cnn_core_loss": (_I, [_P, _P, _P, _I, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P, _P]),
    "cnn_adam": (_I, [_P, _P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, _I, _P]),
    "nfft3_lattice_points": (_I, [_P, _I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "nfft3_tube_workspace_bytes": (ctypes.c_size_t, [_I64]),
    "nfft3_grid_eval_workspace_bytes": (ctypes.c_size_t, [_I, _I, _I, _I, _I, _I, _I]),
    "nfft_lowdim_workspace_bytes": (ctypes.c_size_t, [_I, _P, _I, _D]),
    "nfft_lowdim_eval": (_I, [_I, _P, _I64, _I, _D, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "nfft3d_grid_eval": (_I, [_P, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _P, ctypes.c_size_t, _P]),
    "nfft3f_grid_eval": (_I, [_P, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _P, ctypes.c_size_t, _P]),
    "nfft3_tube_refine": (_I, [_I, _P, _P, _I64, _D, ctypes.POINTER(_D), _P, _I64, ctypes.POINTER(_I64), _P,
                               ctypes.c_size_t, _P]),
    "nfft3_plaquette_crossings": (_I, [_I, _P, _I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), _P,
                                       _P, _I64, _P, _P]),
}

STAGES = ("set_points", "deconv", "fft", "gather", "spread", "fft_fwd", "deconv_adj", "split")

_lock = threading.Lock()
_lib = None


class NFFTError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (fn, error_string(code), code))


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO_PATH):
                raise RuntimeError(
                    "libgbnfft.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                    "g.build()\"` first" % SO_PATH)
            handle = ctypes.CDLL(SO_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def error_string(code: int) -> str:
    return lib().nfft3_error_string(int(code)).decode()


def check(fn: str, code: int) -> int:
    """Raise NFFTError for negative status codes; return warnings unchanged."""
    if code < 0:
        raise NFFTError(fn, code)
    return code


def call(name: str, *args) -> int:
    return check(name, getattr(lib(), name)(*args))
