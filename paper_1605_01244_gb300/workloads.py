"""Seeded synthetic inputs (coefficients and points) for tests and benchmarks.

This module holds only input generation: random coefficients with a Gaussian
spectral envelope, point sets (uniform, Gaussian clusters, local lattices) and
the analytic two-vortex wavefunction sampled on a grid.  None of the NFFT's
arithmetic lives here; both the CUDA path and the CPU oracle consume these
arrays.  All draws use numpy's PCG64 generator so that the same seed gives the
same arrays on x86 and Arm hosts.

Workloads (torus points live in [-1/2, 1/2)^3):

* ``gaussian_coeffs(N, width)`` -- c_k = CN(0,1) exp(-|k|^2 / (2 width^2)),
  CN(0,1) having independent N(0, 1/2) real and imaginary parts.
* ``uniform_points(M)`` -- uniform in [-1/2, 1/2)^3.
* ``cluster_points(M, std)`` -- N(0, std^2) per coordinate, wrapped mod 1.
* ``two_vortex_initial`` -- two perpendicular straight vortices with the
  q = 2 Pade density profile, periodic on [-L, L)^3 (initial data of the
  Gross-Pitaevskii solver).
* ``two_vortex_psi`` / ``gpe_coeffs`` -- the wavefunction
  psi(x) = exp(-|x|^2/18) ((x1 - a) + i x2) ((x1 + a) - i x3) / (1 + |x|^2)
  sampled on the regular grid of [-L, L)^3 and turned into series
  coefficients by the paper's trapezoid rule (Sec. 2: psihat from fftn),
  mapped onto the torus (Sec. 2.2.1 mapping with the + sign).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def freq_grid(N):
    """k_d = i_d - N_d/2 along each axis, broadcastable to (N1, N2, N3)."""
    N1, N2, N3 = N
    k1 = (np.arange(N1) - N1 // 2)[:, None, None]
    k2 = (np.arange(N2) - N2 // 2)[None, :, None]
    k3 = (np.arange(N3) - N3 // 2)[None, None, :]
    return k1, k2, k3


def gaussian_coeffs(N, width: float, seed: int = 0) -> np.ndarray:
    """complex128 (N1, N2, N3): CN(0,1) * exp(-|k|^2/(2 width^2))."""
    g = rng(seed)
    N = tuple(int(v) for v in N)
    z = (g.standard_normal(N) + 1j * g.standard_normal(N)) * np.sqrt(0.5)
    k1, k2, k3 = freq_grid(N)
    env = np.exp(-(k1 * k1 + k2 * k2 + k3 * k3) / (2.0 * width * width))
    return (z * env).astype(np.complex128)


def uniform_points(M: int, seed: int = 0) -> np.ndarray:
    """float64 (M, 3) uniform in [-1/2, 1/2)^3."""
    return rng(seed).random((int(M), 3)) - 0.5


def cluster_points(M: int, std: float, seed: int = 0, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """float64 (M, 3): Gaussian cluster N(center, std^2) per coordinate, wrapped to [-1/2, 1/2)."""
    p = rng(seed).standard_normal((int(M), 3)) * std + np.asarray(center, dtype=np.float64)
    return p - np.floor(p + 0.5)


def mixed_points(M: int, std: float = 0.02, seed: int = 0) -> np.ndarray:
    """Half uniform, half Gaussian-clustered (std) points, interleaved order
    (uniform first half, cluster second half)."""
    M = int(M)
    mu = M // 2
    return np.concatenate([uniform_points(mu, seed), cluster_points(M - mu, std, seed + 1)], axis=0)


def lattice_points(P: int, side: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """P^3 points on a regular lattice filling the cube of the given side (torus units)."""
    t = (np.arange(P) + 0.5) / P * side - side / 2
    a, b, c = np.meshgrid(t, t, t, indexing="ij")
    pts = np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1) + np.asarray(center)
    return pts - np.floor(pts + 0.5)


def two_vortex_psi(N, L: float, a: float = 0.5) -> np.ndarray:
    """psi sampled on xi = -L + (2L/N) n, n = 0..N-1 per axis; complex128 (N1, N2, N3)."""
    axes = [-L + (2.0 * L / Nd) * np.arange(Nd) for Nd in N]
    x1, x2, x3 = np.meshgrid(*axes, indexing="ij")
    r2 = x1 * x1 + x2 * x2 + x3 * x3
    psi = np.exp(-r2 / 18.0) * ((x1 - a) + 1j * x2) * ((x1 + a) - 1j * x3) / (1.0 + r2)
    return psi.astype(np.complex128)


def torus_coeffs_from_samples(psi: np.ndarray) -> np.ndarray:
    """Coefficients c_k (centred order) of the torus series that interpolates psi.

    psi holds samples at x_n = -1/2 + n/N (torus units, i.e. the physical grid
    xi = a + n h mapped by (xi - a)/(b - a) - 1/2).  The trapezoid rule of the
    paper's Sec. 2 gives c_k = (1/N1N2N3) sum_n psi_n e^{-2 pi i k.x_n}
    = (-1)^{k1+k2+k3} fftshift(fftn(psi))_k / (N1 N2 N3).
    """
    N = psi.shape
    k1, k2, k3 = freq_grid(N)
    sign = (-1.0) ** (np.abs(k1) + np.abs(k2) + np.abs(k3))
    return (sign * np.fft.fftshift(np.fft.fftn(psi)) / float(np.prod(N))).astype(np.complex128)


def gpe_coeffs(N, L: float = 8.0, a: float = 0.5) -> np.ndarray:
    """Two-vortex ansatz coefficients on the torus for the box [-L, L)^3."""
    return torus_coeffs_from_samples(two_vortex_psi(N, L, a))


# --- straight-vortex initial data of the Gross-Pitaevskii equation ---------

# Diagonal Pade approximation rho_q(r) = (a1 r^2 + .. + aq r^2q) / (1 + b1 r^2
# + .. + bq r^2q) of the density of a two-dimensional vortex (Sec. 3: the
# density rho = f^2 solves eq. (GPErho), rho(0) = 0, rho(inf) = 1), obtained
# by the paper's recipe: substitute rho_q into eq. (GPErho), set the first
# 2q - 1 coefficients of the resulting series in r^2 to zero, and take
# aq = bq (rho -> 1).  The paper uses q = 4 and does not print its
# coefficients; q = 2 gives the exact rationals below (tests/test_gpe.py
# re-derives them).
PADE2_A = (11.0 / 32.0, 11.0 / 384.0)
PADE2_B = (1.0 / 3.0, 11.0 / 384.0)


def vortex_density(r):
    """rho_2(r): the q = 2 Pade density of a two-dimensional vortex."""
    r2 = np.asarray(r, dtype=np.float64) ** 2
    return (PADE2_A[0] * r2 + PADE2_A[1] * r2 * r2) / (1.0 + PADE2_B[0] * r2 + PADE2_B[1] * r2 * r2)


def periodic_vortex(u, v, L: float):
    """A straight vortex crossing the (u, v) plane at the origin, made
    periodic with period 2L in u and v: its wave function f(R) e^{i Theta},
    with R = (L/pi) sqrt(sin^2(pi u / L) + sin^2(pi v / L)) and Theta =
    atan2(sin(pi v / L), sin(pi u / L)).  Near the origin this is the vortex
    f(r) e^{i theta}; the sines add its three mirror images at distance L
    (circulations -1, -1, +1), so the winding around the periodic box is
    zero -- the periodic counterpart of the mirroring of Sec. 3."""
    su, sv = np.sin(np.pi * u / L), np.sin(np.pi * v / L)
    R = (L / np.pi) * np.sqrt(su * su + sv * sv)
    return np.sqrt(vortex_density(R)) * np.exp(1j * np.arctan2(sv, su))


def two_vortex_initial(n: int = 64, L: float = 8.0, d: float = 1.0) -> np.ndarray:
    """Two perpendicular straight vortices on the periodic box [-L, L)^3
    (n^3 points x = -L + 2 L i / n): one parallel to x3 through (x1, x2) =
    (-d, 0), one parallel to x2 through (x1, x3) = (d, 0); the initial
    condition is the product of their wave functions (Sec. 3).  complex128
    (n, n, n)."""
    x = -L + (2.0 * L / n) * np.arange(n)
    x1, x2, x3 = np.meshgrid(x, x, x, indexing="ij")
    return (periodic_vortex(x1 + d, x2, L) * periodic_vortex(x1 - d, x3, L)).astype(np.complex128)


# --- named workloads -------------------------------------------------------

def small_random(N=(16, 16, 16), M: int = 1000, seed: int = 0):
    """N=16^3 Gaussian-envelope (width 4) coefficients, M uniform points."""
    return gaussian_coeffs(N, 4.0, seed), uniform_points(M, seed + 100)


def precision_sweep(N: int = 256, M: int = 10_000_000, seed: int = 0):
    """N^3 Gaussian-envelope (width 40) coefficients; M points, half uniform,
    half clustered with std 0.02."""
    return gaussian_coeffs((N, N, N), 40.0, seed), mixed_points(M, 0.02, seed + 100)


def gpe_snapshot(N: int = 128, L: float = 8.0, P: int = 100, M_uniform: int = 1_000_000, seed: int = 0):
    """Two-vortex coefficients at N^3; P^3 lattice points in the physical box
    [-0.025, 0.025]^3 (torus side 0.05/(2L)) plus M_uniform uniform points."""
    c = gpe_coeffs((N, N, N), L)
    lat = lattice_points(P, 0.05 / (2.0 * L))
    return c, np.concatenate([lat, uniform_points(M_uniform, seed + 100)], axis=0)
