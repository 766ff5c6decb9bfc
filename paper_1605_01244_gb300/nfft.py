"""Python front end of libgbnfft: a plan object over torch CUDA tensors.

All arithmetic runs in the CUDA library; this module checks shapes, dtypes
and devices and passes raw pointers plus the plan's stream.

    plan = Plan((N1, N2, N3), M, m=6, sigma=2.0, precision="f64")
    plan.set_points(x)            # (M, 3) float64 CUDA tensor
    f = plan.eval(c)              # (N1, N2, N3) complex128 -> (M,) complex128
    f, g = plan.eval_grad(c)      # g: (M, 3), eq. (Lambda) in torus units
    h = plan.adjoint(f)           # (N1, N2, N3)

``precision="f32"`` selects the mixed family (complex64 data; coordinates
stay float64 and are reduced in FP64).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

_FAMILY = {"f64": ("nfft3d", torch.complex128), "f32": ("nfft3f", torch.complex64)}


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """A type-2 NFFT plan on the current CUDA device and stream."""

    def __init__(self, N, M: int, m: int = 0, sigma: float = 2.0, eps: float = 1e-12,
                 precision: str = "f64", stream: torch.cuda.Stream | None = None):
        if precision not in _FAMILY:
            raise ValueError("precision must be 'f64' or 'f32'")
        if not torch.cuda.is_available():
            raise RuntimeError("gbnfft needs a CUDA device (no CPU fallback exists)")
        self.prefix, self.cdtype = _FAMILY[precision]
        self.precision = precision
        self.N = tuple(int(v) for v in N)
        self.M = int(M)
        self.capacity = int(M)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        code = getattr(_lib.lib(), self.prefix + "_plan")(
            ctypes.byref(h), self.N[0], self.N[1], self.N[2], self.M, int(m), float(sigma),
            float(eps), ctypes.c_void_p(self.stream.cuda_stream))
        _lib.check(self.prefix + "_plan", code)
        self.warning = code
        self._h = h
        n = (ctypes.c_int * 3)()
        mm = ctypes.c_int()
        _lib.call("nfft3_plan_info", h, n, ctypes.byref(mm), None, None)
        self.n = tuple(int(v) for v in n)
        self.m = int(mm.value)
        self._x = None  # keeps the last point tensor alive while work is queued

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            getattr(_lib.lib(), self.prefix + "_destroy")(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- checks -------------------------------------------------------------
    def _cuda(self, t: torch.Tensor, dtype, shape, name):
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch tensor" % name)
        if t.device != self.device:
            raise ValueError("%s must live on %s" % (name, self.device))
        if t.dtype != dtype:
            raise TypeError("%s must have dtype %s (got %s)" % (name, dtype, t.dtype))
        if tuple(t.shape) != tuple(shape):
            raise ValueError("%s must have shape %s (got %s)" % (name, tuple(shape), tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        return t

    def _fn(self, suffix):
        return getattr(_lib.lib(), self.prefix + suffix)

    # -- operations ---------------------------------------------------------
    def set_points(self, x: torch.Tensor):
        """x: (M, 3) float64 CUDA tensor of torus coordinates (any reals)."""
        self._cuda(x, torch.float64, (self.M, 3), "x")
        _lib.check(self.prefix + "_set_points", self._fn("_set_points")(self._h, _ptr(x)))
        self._x = x

    def eval(self, c: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """f_j = sum_k c_k exp(2 pi i k.x_j); c: (N1, N2, N3) complex CUDA tensor."""
        self._cuda(c, self.cdtype, self.N, "c")
        if out is None:
            out = torch.empty(self.M, dtype=self.cdtype, device=self.device)
        self._cuda(out, self.cdtype, (self.M,), "out")
        _lib.check(self.prefix + "_eval", self._fn("_eval")(self._h, _ptr(c), _ptr(out)))
        return out

    def eval_grad(self, c: torch.Tensor, want_f: bool = True):
        """(f, grad) with grad[j, d] = sum_k 2 pi i k_d c_k exp(2 pi i k.x_j)."""
        self._cuda(c, self.cdtype, self.N, "c")
        f = torch.empty(self.M, dtype=self.cdtype, device=self.device) if want_f else None
        g = torch.empty((self.M, 3), dtype=self.cdtype, device=self.device)
        _lib.check(self.prefix + "_eval_grad",
                   self._fn("_eval_grad")(self._h, _ptr(c), _ptr(f), _ptr(g)))
        return f, g

    def eval_points(self, x: torch.Tensor, c: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """set_points(x) then eval(c) in one call (the transform of c overlaps
        the sort of x on a second stream where the plan allows)."""
        self._cuda(x, torch.float64, (self.M, 3), "x")
        self._cuda(c, self.cdtype, self.N, "c")
        if out is None:
            out = torch.empty(self.M, dtype=self.cdtype, device=self.device)
        self._cuda(out, self.cdtype, (self.M,), "out")
        _lib.check(self.prefix + "_eval_points", self._fn("_eval_points")(self._h, _ptr(x), _ptr(c), _ptr(out)))
        self._x = x
        return out

    def chain_x(self, G: torch.Tensor, grad: torch.Tensor) -> torch.Tensor:
        """(M, 3) float64 dL/dx with dL/dx_{j,d} = Re(conj(G_j) grad[j, d]):
        G the upstream gradient of f, grad from :meth:`eval_grad`."""
        self._cuda(G, self.cdtype, (self.M,), "G")
        self._cuda(grad, self.cdtype, (self.M, 3), "grad")
        gx = torch.empty((self.M, 3), dtype=torch.float64, device=self.device)
        _lib.check(self.prefix + "_chain_x", self._fn("_chain_x")(self._h, _ptr(G), _ptr(grad), _ptr(gx)))
        return gx

    def adjoint(self, f: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """h_k = sum_j f_j exp(-2 pi i k.x_j); f: (M,) complex CUDA tensor."""
        self._cuda(f, self.cdtype, (self.M,), "f")
        if out is None:
            out = torch.empty(self.N, dtype=self.cdtype, device=self.device)
        self._cuda(out, self.cdtype, self.N, "out")
        _lib.check(self.prefix + "_adjoint", self._fn("_adjoint")(self._h, _ptr(f), _ptr(out)))
        return out

    # -- one series at many point sets -----------------------------------------
    def precompute(self, c: torch.Tensor, with_grad: bool = False):
        """Deconvolve, FFT and pad c once; eval_stored / eval_grad_stored reuse it."""
        self._cuda(c, self.cdtype, self.N, "c")
        _lib.check(self.prefix + "_precompute", self._fn("_precompute")(self._h, _ptr(c), int(with_grad)))

    def eval_stored(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.M, dtype=self.cdtype, device=self.device)
        self._cuda(out, self.cdtype, (self.M,), "out")
        _lib.check(self.prefix + "_eval_stored", self._fn("_eval_stored")(self._h, _ptr(out)))
        return out

    def eval_grad_stored(self, want_f: bool = True):
        f = torch.empty(self.M, dtype=self.cdtype, device=self.device) if want_f else None
        g = torch.empty((self.M, 3), dtype=self.cdtype, device=self.device)
        _lib.check(self.prefix + "_eval_grad_stored", self._fn("_eval_grad_stored")(self._h, _ptr(f), _ptr(g)))
        return f, g

    def eval_grad_window(self, c: torch.Tensor, want_f: bool = True):
        """f and grad (M x 3) by differentiating the window: one transform
        instead of four; about ten times the i k-method's gradient error at
        the same m."""
        self._cuda(c, self.cdtype, self.N, "c")
        f = torch.empty(self.M, dtype=self.cdtype, device=self.device) if want_f else None
        g = torch.empty((self.M, 3), dtype=self.cdtype, device=self.device)
        _lib.check(self.prefix + "_eval_grad_window",
                   self._fn("_eval_grad_window")(self._h, _ptr(c), _ptr(f), _ptr(g)))
        return f, g

    def eval_grad_window_stored(self, want_f: bool = True):
        """eval_grad_window from the grid of a preceding precompute."""
        f = torch.empty(self.M, dtype=self.cdtype, device=self.device) if want_f else None
        g = torch.empty((self.M, 3), dtype=self.cdtype, device=self.device)
        _lib.check(self.prefix + "_eval_grad_window_stored",
                   self._fn("_eval_grad_window_stored")(self._h, _ptr(f), _ptr(g)))
        return f, g

    def set_num_points(self, M: int):
        """Use M points (at most the capacity given at creation); set_points must follow."""
        if M > self.capacity:
            raise ValueError("M exceeds the plan's capacity %d" % self.capacity)
        _lib.call("nfft3_set_num_points", self._h, int(M))
        self.M = int(M)

    def eval_host(self, x_host: torch.Tensor, c_host: torch.Tensor, f_host: torch.Tensor):
        """Host-buffer path: copy x and c in, set points, evaluate, copy f out, synchronise."""
        for t, dt, shp, nm in ((x_host, torch.float64, (self.M, 3), "x_host"),
                               (c_host, self.cdtype, self.N, "c_host"),
                               (f_host, self.cdtype, (self.M,), "f_host")):
            if t.device.type != "cpu" or t.dtype != dt or tuple(t.shape) != tuple(shp) or not t.is_contiguous():
                raise ValueError("%s must be a contiguous CPU tensor %s of shape %s" % (nm, dt, shp))
        _lib.check(self.prefix + "_eval_host",
                   self._fn("_eval_host")(self._h, _ptr(x_host), _ptr(c_host), _ptr(f_host)))
        return f_host

    def set_deterministic(self, on: bool = True):
        """Bitwise reproducible adjoints (FP64 plans): stable point
        order and exact fixed-point spread flushes.  set_points must follow."""
        _lib.call("nfft3_set_deterministic", self._h, int(bool(on)))

    def sync(self):
        _lib.call("nfft3_sync", self._h)


def choose_m(eps: float, sigma: float = 2.0) -> int:
    """Cutoff m the library picks for a target relative error eps."""
    return int(_lib.lib().nfft3_choose_m(float(eps), float(sigma)))


def reduce_coords(x: torch.Tensor, n: int, m: int):
    """set_points' reduction of each coordinate in ``x`` (float64 CUDA
    tensor, any shape) for an oversampled size n and cutoff m: the first
    stencil node l0 (int32, in [0, n)), the offset s in [0, 1) as the FP64
    family stores it (float64) and as the mixed family stores it (float32)."""
    if x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError("x must be a float64 CUDA tensor")
    xf = x.contiguous().reshape(-1)
    l0 = torch.empty(xf.shape, dtype=torch.int32, device=x.device)
    s = torch.empty(xf.shape, dtype=torch.float64, device=x.device)
    s32 = torch.empty(xf.shape, dtype=torch.float32, device=x.device)
    status = torch.empty(1, dtype=torch.int32, device=x.device)
    _lib.call("nfft3_reduce_coords", int(n), int(m), _ptr(xf), xf.numel(), _ptr(l0), _ptr(s), _ptr(s32),
              _ptr(status), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if int(status.item()) & 1:
        raise _lib.NFFTError("nfft3_reduce_coords", _lib.NFFT3_ERR_POINTS)
    return l0.reshape(x.shape), s.reshape(x.shape), s32.reshape(x.shape)
