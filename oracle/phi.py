"""Scalar phi-functions (Sect. 2, Eqs. 5-6).

phi_0(z) = e^z and phi_k(z) = int_0^1 e^{(1-theta) z} theta^{k-1}/(k-1)! dtheta.
Two evaluations are given:
  * ``phi`` -- the power series phi_k(z) = sum_i z^i/(i+k)! for |z| < 2, and the
    recursion phi_{k+1}(z) = (phi_k(z) - 1/k!)/z (which follows from Eq. 6 by
    integrating by parts) elsewhere;
  * ``phi_quadrature`` -- Eq. 6 itself by adaptive quadrature (test pin only).
"""
from __future__ import annotations

import math

import numpy as np


def phi(k: int, z):
    """phi_k(z) elementwise for real or complex z (array or scalar)."""
    z = np.asarray(z)
    out = np.empty(z.shape, dtype=np.result_type(z.dtype, np.float64))
    small = np.abs(z) < 2.0
    if np.any(small):
        zs = z[small]
        acc = np.zeros(zs.shape, dtype=out.dtype)
        # terms z^i/(i+k)! for i = 0..45; |z| < 2 makes the tail < 2^46/46! ~ 1e-45
        for i in reversed(range(46)):
            acc = acc * zs + 1.0 / math.factorial(i + k)
        out[small] = acc
    big = ~small
    if np.any(big):
        zb = z[big]
        val = np.exp(zb)
        for j in range(k):  # phi_{j+1} = (phi_j - 1/j!) / z
            val = (val - 1.0 / math.factorial(j)) / zb
        out[big] = val
    return out if out.shape else out[()]


def phi_quadrature(k: int, z: complex) -> complex:
    """Eq. 6 evaluated by adaptive Gauss-Kronrod quadrature (scipy.integrate)."""
    from scipy.integrate import quad

    if k == 0:
        return complex(np.exp(z))
    f = lambda t, part: (part(np.exp((1 - t) * z) * t ** (k - 1))) / math.factorial(k - 1)
    re = quad(f, 0.0, 1.0, args=(np.real,), epsabs=1e-300, epsrel=1e-13, limit=200)[0]
    if np.imag(z) == 0:
        return complex(re, 0.0)
    im = quad(f, 0.0, 1.0, args=(np.imag,), epsabs=1e-300, epsrel=1e-13, limit=200)[0]
    return complex(re, im)
