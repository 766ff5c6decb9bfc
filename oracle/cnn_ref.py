"""FP64 numpy reference of the core-proposal CNN's operations -- TEST INFRASTRUCTURE.

Only tests use this module.  Direct definitions, no blocking:

  conv3d:  y[b,o,p] = bias[o] + sum_{i,t} w[o,i,t] x[b,i,p+t-h]   (zero padding h = k//2)
  dgrad:   dx[b,i,q] = sum_{o,t} w[o,i,t] dy[b,o,q-t+h]
  wgrad:   dw[o,i,t] = sum_{b,p} dy[b,o,p] x[b,i,p+t-h],  db[o] = sum_{b,p} dy[b,o,p]
  loss:    mean_v (1 + (pw-1) t_v) BCE(l_v, t_v) + lam * sum_v t_v |o_v - o*_v|_1 / max(1, sum_v t_v)
"""
from __future__ import annotations

import numpy as np


def _shift(x, dz, dy, dx):
    """x shifted so that out[..., z, y, x] = x[..., z+dz, y+dy, x+dx] (zero outside)."""
    D = x.shape[-1]
    out = np.zeros_like(x)
    zs, ys, xs = [slice(max(0, -d), min(D, D - d)) for d in (dz, dy, dx)]
    zt, yt, xt = [slice(max(0, d), min(D, D + d)) for d in (dz, dy, dx)]
    out[..., zs, ys, xs] = x[..., zt, yt, xt]
    return out


def conv3d(x, w, bias=None):
    B, Ci, D = x.shape[0], x.shape[1], x.shape[2]
    Co, k = w.shape[0], w.shape[2]
    h = k // 2
    y = np.zeros((B, Co, D, D, D))
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                xs = _shift(x, dz - h, dy - h, dx - h)
                y += np.einsum("oi,bizyx->bozyx", w[:, :, dz, dy, dx], xs)
    if bias is not None:
        y += bias[None, :, None, None, None]
    return y


def conv3d_dgrad(dy, w):
    Co, Ci, k = w.shape[0], w.shape[1], w.shape[2]
    h = k // 2
    dx = np.zeros((dy.shape[0], Ci) + dy.shape[2:])
    for dz in range(k):
        for dyy in range(k):
            for dxx in range(k):
                ds = _shift(dy, -(dz - h), -(dyy - h), -(dxx - h))
                dx += np.einsum("oi,bozyx->bizyx", w[:, :, dz, dyy, dxx], ds)
    return dx


def conv3d_wgrad(dy, x, k):
    h = k // 2
    Co, Ci = dy.shape[1], x.shape[1]
    dw = np.zeros((Co, Ci, k, k, k))
    for dz in range(k):
        for dyy in range(k):
            for dxx in range(k):
                xs = _shift(x, dz - h, dyy - h, dxx - h)
                dw[:, :, dz, dyy, dxx] = np.einsum("bozyx,bizyx->oi", dy, xs)
    return dw, dy.sum(axis=(0, 2, 3, 4))


def core_loss(y, target, off_target, lam, pw=1.0):
    """y: (B,4,D,D,D); target: (B,D^3); off_target: (B,D^3,3).  Returns (loss, dy)."""
    B, D = y.shape[0], y.shape[2]
    n = B * D ** 3
    l = y[:, 0].reshape(B, -1)
    t = target.reshape(B, -1)
    npos = max(float(t.sum()), 1.0)
    wt = 1 + (pw - 1) * t
    bce = wt * (np.maximum(l, 0) - l * t + np.log1p(np.exp(-np.abs(l))))
    dy = np.zeros_like(y)
    dy[:, 0] = (wt * (1 / (1 + np.exp(-l)) - t) / n).reshape(B, D, D, D)
    loss = bce.sum() / n
    for c in range(3):
        o = y[:, 1 + c].reshape(B, -1)
        d = o - off_target.reshape(B, -1, 3)[:, :, c]
        loss += lam * (t * np.abs(d)).sum() / npos
        dy[:, 1 + c] = (lam * t * np.sign(d) / npos).reshape(B, D, D, D)
    return loss, dy
