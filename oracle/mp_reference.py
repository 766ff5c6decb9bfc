"""Arbitrary-precision brute force for tiny cases -- TEST INFRASTRUCTURE.

Evaluates f_j = sum_k c_k exp(2 pi i k.x_j) term by term in mpmath at 40
significant digits, from the decimal expansion of the given doubles, for
checking the FP64 direct sum in ``direct.c`` (pure-Python loops: keep N and M
tiny).  Paper eq. (fs)/(Fs), torus form.
"""
from __future__ import annotations

import mpmath
import numpy as np


def forward(c, x, dps: int = 40) -> np.ndarray:
    c = np.asarray(c, dtype=np.complex128)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    N1, N2, N3 = c.shape
    out = np.zeros(x.shape[0], dtype=np.complex128)
    with mpmath.workdps(dps):
        two_pi_i = 2 * mpmath.pi * 1j
        for j in range(x.shape[0]):
            xs = [mpmath.mpf(float(v)) for v in x[j]]
            acc = mpmath.mpc(0)
            for i1 in range(N1):
                for i2 in range(N2):
                    for i3 in range(N3):
                        k = (i1 - N1 // 2, i2 - N2 // 2, i3 - N3 // 2)
                        ph = k[0] * xs[0] + k[1] * xs[1] + k[2] * xs[2]
                        cv = c[i1, i2, i3]
                        acc += mpmath.mpc(float(cv.real), float(cv.imag)) * mpmath.exp(two_pi_i * ph)
            out[j] = complex(acc)
    return out
