"""Plain numpy NFFT (type 2 forward, type 1 adjoint, gradient) -- TEST INFRASTRUCTURE.

Only tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline legs
use this module; the product never imports it.

The paper (Sec. 2.2.1) uses the NFFT only as a black box with cost
O(N log N + M |log eps|^3) and states no window, oversampling or cutoff.  This
module restates the standard NFFT approximation of the series (the paper's
citation [KKP09]) from its derivation, step by step, with no blocking or
fusion:

  grid nodes   x_l = -1/2 + l/n_d  (l = 0..n_d-1, periodic),  u = n (x + 1/2)
  window       half-width alpha = m + 1/2 cells (the 2m+1 taps span it),
               phi(tau) = sinh(b sqrt(alpha^2 - tau^2)) / (pi sqrt(alpha^2 - tau^2))
               for -alpha < tau <= alpha (value b/pi at tau = alpha), 0 outside;
               b = pi (2 - 1/sigma), sigma = n/N
  its transform Phi(nu) = int phi(tau) e^{-2 pi i nu tau} dtau
                        = I0(alpha sqrt(b^2 - (2 pi nu)^2))     (|2 pi nu| <= b)
               (one excluded end point does not change the integral)
  step 1 (deconvolve + zero-pad)  G[k mod n] = c_k (-1)^{k1+k2+k3} / prod_d Phi(k_d/n_d)
  step 2 (oversampled FFT)        g_l = sum_k G_k e^{+2 pi i k.l/n}      (unnormalised)
  step 3 (window sum)             f_j = sum_l g_{l mod n} prod_d phi(u_{j,d} - l_d),
                                  l_d = ceil(u_{j,d} - alpha) + {0, ..., 2m}
                                  (exactly the nodes with -alpha < u - l <= alpha)

The (-1)^k factor moves the grid origin from 0 to -1/2.  The adjoint applies
the transposes in reverse order (spread, forward FFT, the same deconvolution),
and the gradient deconvolves 2 pi i k_d c_k in step 1.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import i0 as _i0


def kb_b(n: int, N: int) -> float:
    """Shape parameter b = pi (2 - 1/sigma), sigma = n/N."""
    return math.pi * (2.0 - N / n)


def kb_phi(tau, m: int, b: float):
    """Kaiser-Bessel window in grid units, half-width alpha = m + 1/2,
    support -alpha < tau <= alpha (value b/pi at tau = alpha)."""
    al = m + 0.5
    tau = np.asarray(tau, dtype=np.float64)
    s = np.sqrt(np.maximum((al - tau) * (al + tau), 0.0))
    safe = np.where(s > 0, s, 1.0)
    val = np.where(s > 0, np.sinh(b * s) / (math.pi * safe), b / math.pi)
    return np.where((tau > -al) & (tau <= al), val, 0.0)


def kb_dphi(tau, m: int, b: float):
    """Derivative of ``kb_phi`` in tau inside the support:
    phi'(tau) = -tau (b s cosh(b s) - sinh(b s)) / (pi s^3),  s = sqrt(alpha^2 - tau^2),
    with the series (b s)^3/3 + (b s)^5/30 + (b s)^7/840 of the bracket for
    small b s (its limit at the support ends is -tau b^3 / (3 pi))."""
    al = m + 0.5
    tau = np.asarray(tau, dtype=np.float64)
    s = np.sqrt(np.maximum((al - tau) * (al + tau), 0.0))
    z = b * s
    small = z < 1e-2
    zs = np.where(small, 1.0, z)
    ss = np.where(small, 1.0, s)
    exact = -tau * (zs * np.cosh(zs) - np.sinh(zs)) / (math.pi * ss ** 3)
    series = -tau * b ** 3 * (1.0 / 3.0 + z ** 2 / 30.0 + z ** 4 / 840.0) / math.pi
    val = np.where(small, series, exact)
    return np.where((tau > -al) & (tau <= al), val, 0.0)


def kb_Phi(k, n: int, m: int, b: float):
    """Fourier transform of ``kb_phi`` at nu = k/n: I0(alpha sqrt(b^2 - (2 pi k/n)^2))."""
    k = np.asarray(k, dtype=np.float64)
    return _i0((m + 0.5) * np.sqrt(b * b - (2.0 * math.pi * k / n) ** 2))


def _setup(N, n, m):
    N = tuple(int(v) for v in N)
    n = tuple(int(v) for v in n)
    if any(nd < Nd for nd, Nd in zip(n, N)):
        raise ValueError("n_d must be >= N_d")
    if m < 0:
        raise ValueError("m must be >= 0")
    ks = [np.arange(Nd) - Nd // 2 for Nd in N]
    bs = [kb_b(nd, Nd) for nd, Nd in zip(n, N)]
    # per-dimension deconvolution factors (-1)^k / Phi(k/n)
    dec = [((-1.0) ** np.abs(k)) / kb_Phi(k, nd, m, b) for k, nd, b in zip(ks, n, bs)]
    return N, n, ks, bs, dec


def _window_rows(x, n, m, bs):
    """Per point and dimension: first stencil node l0 = ceil(u - alpha) and the
    2m+1 window values phi(u - l0 - a), a = 0..2m."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    xw = x - np.floor(x + 0.5)          # wrap onto [-1/2, 1/2)
    al = m + 0.5
    l0s, ws = [], []
    a = np.arange(2 * m + 1)
    for d in range(3):
        u = n[d] * (xw[:, d] + 0.5)
        l0 = np.ceil(u - al)
        tau = u[:, None] - (l0[:, None] + a[None, :])
        l0s.append(l0.astype(np.int64))
        ws.append(kb_phi(tau, m, bs[d]))
    return l0s, ws


def forward(c, x, n, m: int):
    """NFFT approximation of f_j = sum_k c_k e^{2 pi i k.x_j} (steps 1-3)."""
    c = np.asarray(c, dtype=np.complex128)
    N, n, ks, bs, dec = _setup(c.shape, n, m)
    return _gather(_oversampled_grid(c, N, n, ks, dec), x, n, m, bs)


def _oversampled_grid(c, N, n, ks, dec):
    G = np.zeros(n, dtype=np.complex128)
    D = dec[0][:, None, None] * dec[1][None, :, None] * dec[2][None, None, :]
    G[np.ix_(ks[0] % n[0], ks[1] % n[1], ks[2] % n[2])] = c * D
    return np.fft.ifftn(G) * (n[0] * n[1] * n[2])  # unnormalised e^{+} transform


def _gather(g, x, n, m, bs):
    l0s, ws = _window_rows(x, n, m, bs)
    M = l0s[0].shape[0]
    f = np.zeros(M, dtype=np.complex128)
    a = np.arange(2 * m + 1)
    i3 = (l0s[2][:, None] + a[None, :]) % n[2]
    for p in range(2 * m + 1):
        i1 = (l0s[0] + p) % n[0]
        for q in range(2 * m + 1):
            i2 = (l0s[1] + q) % n[1]
            inner = np.sum(g[i1[:, None], i2[:, None], i3] * ws[2], axis=1)
            f += ws[0][:, p] * ws[1][:, q] * inner
    return f


def forward_grad(c, x, n, m: int):
    """NFFT approximation of the series and its gradient (i k-weighted series)."""
    c = np.asarray(c, dtype=np.complex128)
    N, n, ks, bs, dec = _setup(c.shape, n, m)
    f = _gather(_oversampled_grid(c, N, n, ks, dec), x, n, m, bs)
    grads = []
    for d in range(3):
        shape = [1, 1, 1]
        shape[d] = N[d]
        kd = ks[d].reshape(shape)
        cd = 2j * math.pi * kd * c
        grads.append(_gather(_oversampled_grid(cd, N, n, ks, dec), x, n, m, bs))
    return f, np.stack(grads, axis=1)


def forward_grad_window(c, x, n, m: int):
    """Gradient by differentiating the window instead of the series: one grid
    (steps 1-2 of ``forward``), then for each dimension d the window sum of
    step 3 with phi replaced by n_d phi' in dimension d, since
    d/dx_d phi(u_d - l_d) = n_d phi'(u_d - l_d) with u_d = n_d (x_d + 1/2).
    Returns (f, grad)."""
    c = np.asarray(c, dtype=np.complex128)
    N, n, ks, bs, dec = _setup(c.shape, n, m)
    g = _oversampled_grid(c, N, n, ks, dec)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    l0s, ws = _window_rows(x, n, m, bs)
    xw = x - np.floor(x + 0.5)
    a = np.arange(2 * m + 1)
    dws = []
    for d in range(3):
        u = n[d] * (xw[:, d] + 0.5)
        tau = u[:, None] - (l0s[d][:, None] + a[None, :])
        dws.append(n[d] * kb_dphi(tau, m, bs[d]))
    M = x.shape[0]
    f = np.zeros(M, dtype=np.complex128)
    grad = np.zeros((M, 3), dtype=np.complex128)
    i3 = (l0s[2][:, None] + a[None, :]) % n[2]
    for p in range(2 * m + 1):
        i1 = (l0s[0] + p) % n[0]
        for q in range(2 * m + 1):
            i2 = (l0s[1] + q) % n[1]
            rows = g[i1[:, None], i2[:, None], i3]
            inner = np.sum(rows * ws[2], axis=1)
            inner_d = np.sum(rows * dws[2], axis=1)
            f += ws[0][:, p] * ws[1][:, q] * inner
            grad[:, 0] += dws[0][:, p] * ws[1][:, q] * inner
            grad[:, 1] += ws[0][:, p] * dws[1][:, q] * inner
            grad[:, 2] += ws[0][:, p] * ws[1][:, q] * inner_d
    return f, grad


def adjoint(f, x, N, n, m: int):
    """NFFT approximation of h_k = sum_j f_j e^{-2 pi i k.x_j} (transposed steps)."""
    N, n, ks, bs, dec = _setup(N, n, m)
    f = np.asarray(f, dtype=np.complex128).reshape(-1)
    l0s, ws = _window_rows(x, n, m, bs)
    H = np.zeros(n, dtype=np.complex128)
    a = np.arange(2 * m + 1)
    i3 = (l0s[2][:, None] + a[None, :]) % n[2]
    for p in range(2 * m + 1):
        i1 = (l0s[0] + p) % n[0]
        for q in range(2 * m + 1):
            i2 = (l0s[1] + q) % n[1]
            vals = (f * ws[0][:, p] * ws[1][:, q])[:, None] * ws[2]
            np.add.at(H, (np.broadcast_to(i1[:, None], i3.shape),
                          np.broadcast_to(i2[:, None], i3.shape), i3), vals)
    Hk = np.fft.fftn(H)  # unnormalised e^{-} transform
    D = dec[0][:, None, None] * dec[1][None, :, None] * dec[2][None, None, :]
    return Hk[np.ix_(ks[0] % n[0], ks[1] % n[1], ks[2] % n[2])] * D


# ---- one- and two-dimensional series (the paper's infft / infft2) ----------

def direct_lowdim(c, x):
    """Direct sum f_j = sum_k c_k exp(2 pi i k.x_j) for a 1D or 2D c, with
    the phase k.x reduced in extended precision (np.longdouble) before the
    exponential."""
    c = np.asarray(c, dtype=np.complex128)
    dim = c.ndim
    x = np.asarray(x, dtype=np.float64).reshape(-1, dim)
    tabs = []
    for d in range(dim):
        k = (np.arange(c.shape[d]) - c.shape[d] // 2).astype(np.longdouble)
        ph = x[:, d].astype(np.longdouble)[:, None] * k[None, :]
        r = (ph - np.rint(ph)).astype(np.float64)
        tabs.append(np.exp(2j * np.pi * r))
    if dim == 1:
        return tabs[0] @ c
    return np.einsum("ja,ab,jb->j", tabs[0], c, tabs[1])


def forward_lowdim(c, x, n, m: int):
    """The NFFT approximation (steps 1-3 of ``forward``) in 1 or 2 dimensions."""
    c = np.asarray(c, dtype=np.complex128)
    dim = c.ndim
    N = c.shape
    n = tuple(int(v) for v in n)[:dim]
    x = np.asarray(x, dtype=np.float64).reshape(-1, dim)
    ks = [np.arange(Nd) - Nd // 2 for Nd in N]
    bs = [kb_b(nd, Nd) for nd, Nd in zip(n, N)]
    dec = [((-1.0) ** np.abs(k)) / kb_Phi(k, nd, m, b) for k, nd, b in zip(ks, n, bs)]
    G = np.zeros(n, dtype=np.complex128)
    D = dec[0] if dim == 1 else dec[0][:, None] * dec[1][None, :]
    G[np.ix_(*[k % nd for k, nd in zip(ks, n)])] = c * D
    g = np.fft.ifftn(G) * np.prod(n)
    xw = x - np.floor(x + 0.5)
    al = m + 0.5
    a = np.arange(2 * m + 1)
    idx, ws = [], []
    for d in range(dim):
        u = n[d] * (xw[:, d] + 0.5)
        l0 = np.ceil(u - al)
        idx.append(((l0[:, None] + a[None, :]).astype(np.int64)) % n[d])
        ws.append(kb_phi(u[:, None] - (l0[:, None] + a[None, :]), m, bs[d]))
    if dim == 1:
        return np.sum(g[idx[0]] * ws[0], axis=1)
    f = np.zeros(x.shape[0], dtype=np.complex128)
    for p in range(2 * m + 1):
        f += ws[0][:, p] * np.sum(g[idx[0][:, p:p + 1], idx[1]] * ws[1], axis=1)
    return f

