"""Gross-Pitaevskii TSSP in numpy -- TEST INFRASTRUCTURE (like all of oracle/).

The paper's Sec. 3.1 restated step by step for a periodic box of sides L,
with numpy's FFT, FP64, no merging of half steps:

    eq. (GPE)       psi_t = (i/2) Lap psi + (i/2) (1 - |psi|^2) psi
    potential part  v(t) = exp(i t (1 - |v(0)|^2) / 2) v(0)        (exact, |v| constant)
    kinetic part    u_hat_k(t) = exp(-i t |kappa_k|^2 / 2) u_hat_k(0),  kappa_d = 2 pi k_d / L_d
    Strang step     psi_{n+1/2} = e^{tau A} e^{tau/2 B(psi_n)} psi_n,
                    psi_{n+1}   = e^{tau/2 B(psi_{n+1/2})} psi_{n+1/2}
    energy          E = (1/2) int |grad psi|^2 + (1/4) int (1 - |psi|^2)^2   (eq. (energy))
"""
from __future__ import annotations

import numpy as np


def wavenumbers(n, L):
    """kappa_d on the FFT grid: 2 pi k_d / L_d, k_d the signed FFT frequencies."""
    return [2.0 * np.pi * np.fft.fftfreq(nd, d=1.0 / nd) / Ld for nd, Ld in zip(n, L)]


def potential(v, t):
    return np.exp(0.5j * t * (1.0 - np.abs(v) ** 2)) * v


def kinetic(u, t, L):
    k1, k2, k3 = wavenumbers(u.shape, L)
    kap2 = k1[:, None, None] ** 2 + k2[None, :, None] ** 2 + k3[None, None, :] ** 2
    return np.fft.ifftn(np.exp(-0.5j * t * kap2) * np.fft.fftn(u))


def strang_step(psi, tau, L):
    half = kinetic(potential(psi, 0.5 * tau), tau, L)
    return potential(half, 0.5 * tau)


def run(psi, tau, nsteps, L):
    psi = np.asarray(psi, dtype=np.complex128)
    for _ in range(nsteps):
        psi = strang_step(psi, tau, L)
    return psi


def mass(psi, L):
    return float(np.sum(np.abs(psi) ** 2) * np.prod(L) / psi.size)


def energy(psi, L):
    k1, k2, k3 = wavenumbers(psi.shape, L)
    h = np.fft.fftn(psi)
    kap2 = k1[:, None, None] ** 2 + k2[None, :, None] ** 2 + k3[None, None, :] ** 2
    grad2 = np.sum(kap2 * np.abs(h) ** 2) / psi.size      # sum_x |grad psi|^2 (Parseval)
    pot = np.sum((1.0 - np.abs(psi) ** 2) ** 2)
    return float((0.5 * grad2 + 0.25 * pot) * np.prod(L) / psi.size)
