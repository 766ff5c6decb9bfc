"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every symbol include/gbnfft.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1605_01244_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "gbnfft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nfft3\w*)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for fam in ("nfft3d", "nfft3f"):
        for op in ("plan", "set_points", "eval", "eval_grad", "adjoint", "destroy", "eval_host"):
            assert "%s_%s" % (fam, op) in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


def test_error_strings(lib):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert _lib.error_string(code)
    assert _lib.error_string(-99) == "unknown status"


def test_choose_m_rule(lib):
    # estimate 8 exp(-2 pi sqrt(1 - 1/sigma) (m + 1/2)) <= eps
    import math
    for eps in (1e-3, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-13):
        m = lib.nfft3_choose_m(eps, 2.0)
        est = lambda mm: 8 * math.exp(-2 * math.pi * math.sqrt(0.5) * (mm + 0.5))
        assert est(m) <= eps or m == 8
        assert m == 1 or est(m - 1) > eps
    assert lib.nfft3_choose_m(1e-6, 2.0) == 4
    assert lib.nfft3_choose_m(1e-12, 2.0) == 7
    assert lib.nfft3_choose_m(1e-30, 2.0) == 8


@pytest.mark.parametrize("args", [
    (15, 16, 16, 10, 6, 2.0, 0.0),    # odd N
    (16, 0, 16, 10, 6, 2.0, 0.0),     # N < 2
    (16, 16, 16, -1, 6, 2.0, 0.0),    # M < 0
    (16, 16, 16, 10, 9, 2.0, 0.0),    # m beyond the compiled range
    (16, 16, 16, 10, 6, 1.1, 0.0),    # sigma < 1.25
    (16, 16, 16, 10, 0, 2.0, -1.0),   # m from eps, but no eps
])
def test_plan_rejects_bad_arguments(lib, args):
    h = ctypes.c_void_p()
    for fam in ("nfft3d_plan", "nfft3f_plan"):
        code = getattr(lib, fam)(ctypes.byref(h), *args, None)
        assert code == _lib.NFFT3_ERR_ARG
        assert not h.value


def test_plan_rejects_too_large(lib):
    h = ctypes.c_void_p()
    assert lib.nfft3d_plan(ctypes.byref(h), 8192, 16, 16, 10, 6, 2.0, 0.0, None) == _lib.NFFT3_ERR_TOO_LARGE
    assert lib.nfft3d_plan(ctypes.byref(h), 16, 16, 16, 1 << 31, 6, 2.0, 0.0, None) == _lib.NFFT3_ERR_TOO_LARGE


def test_null_handles(lib):
    assert lib.nfft3d_destroy(None) == 0
    assert lib.nfft3f_destroy(None) == 0
    assert lib.nfft3_plan_info(None, None, None, None, None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3d_eval(None, None, None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3f_adjoint(None, None, None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3d_set_points(None, None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3_sync(None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3d_chain_x(None, None, None, None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3d_eval_points(None, None, None, None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3f_eval_points(None, None, None, None) == _lib.NFFT3_ERR_ARG
    assert lib.nfft3f_chain_x(None, None, None, None) == _lib.NFFT3_ERR_ARG


def test_reduce_coords_rejects_bad_arguments(lib):
    """Argument checks of nfft3_reduce_coords come before any CUDA call."""
    dummy = ctypes.c_void_p(16)
    st = ctypes.c_void_p(32)
    E = _lib.NFFT3_ERR_ARG
    assert lib.nfft3_reduce_coords(1, 3, dummy, 10, None, None, None, st, None) == E      # n < 2
    assert lib.nfft3_reduce_coords(64, 0, dummy, 10, None, None, None, st, None) == E     # m < 1
    assert lib.nfft3_reduce_coords(64, 9, dummy, 10, None, None, None, st, None) == E     # m > 8
    assert lib.nfft3_reduce_coords(64, 3, dummy, -1, None, None, None, st, None) == E     # M < 0
    assert lib.nfft3_reduce_coords(64, 3, dummy, 10, None, None, None, None, None) == E   # no status word
    assert lib.nfft3_reduce_coords(64, 3, None, 10, None, None, None, st, None) == E      # no x
