"""O-exact: phi_k(hA) v without Krylov projection.

* ``phi_combination_dense`` -- Sect. 2.1, Eq. 7 with the augmented matrix of
  Eqs. 8-9, written out densely (tiny N only).
* ``phi_products_dense`` -- phi_0..phi_p(hA) v, one Eq. 7 evaluation per k.
* ``phi_products_fft_*`` -- periodic constant-coefficient operators are
  diagonalised by the DFT; phi_k is applied to each Fourier eigenvalue.
* ``phi_products_diagonal`` -- A = diag(lam): y_k = phi_k(h lam) .* v.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import operators
from .expm import expm_taylor
from .phi import phi


def phi_combination_dense(J: np.ndarray, vs, tau: float = 1.0, expm=None) -> np.ndarray:
    """sum_{j=0}^p tau^j phi_j(tau J) v_j  =  [I_N 0] exp(tau A) [v_0; e_p]   (Eq. 7)

    with A = [[J, B], [0, K]] (Eqs. 8-9), B = [b_p, ..., b_1] = [v_p, ..., v_1],
    K the p x p upper shift [[0, I_{p-1}], [0, 0]], e_p the p-th unit vector.
    (The printed Eq. 8 also multiplies J by tau inside A; with tau = 1, the
    case the paper uses, the two readings coincide.)"""
    expm = expm or expm_taylor
    J = np.asarray(J, dtype=np.float64)
    N = J.shape[0]
    p = len(vs) - 1
    A = np.zeros((N + p, N + p))
    A[:N, :N] = J
    for j in range(1, p + 1):
        A[:N, p - j + N] = vs[j]  # column of b_j within B = [b_p, ..., b_1]
    for i in range(p - 1):
        A[N + i, N + i + 1] = 1.0
    rhs = np.zeros(N + p)
    rhs[:N] = vs[0]
    if p > 0:
        rhs[N + p - 1] = 1.0
    return (expm(tau * A) @ rhs)[:N]


def phi_products_dense(A: np.ndarray, v: np.ndarray, h: float, p: int, expm=None) -> np.ndarray:
    """[phi_k(hA) v for k = 0..p] as a (p+1, N) array, each from Eq. 7 with a
    single nonzero v_k = v and J = hA."""
    A = np.asarray(A.todense() if hasattr(A, "todense") else A, dtype=np.float64)
    N = A.shape[0]
    out = np.zeros((p + 1, N))
    zero = np.zeros(N)
    for k in range(p + 1):
        vs = [zero] * (k + 1)
        vs = list(vs)
        vs[k] = v
        out[k] = phi_combination_dense(h * A, vs, 1.0, expm)
    return out


def phi_products_diagonal(lam: np.ndarray, v: np.ndarray, h: float, p: int) -> np.ndarray:
    return np.stack([phi(k, h * lam) * v for k in range(p + 1)])


def phi_products_fft_advdiff2d(cfg: dict, v: np.ndarray, h: float, p: int) -> np.ndarray:
    nx, ny = cfg["nx"], cfg["ny"]
    lam = operators.fourier_symbol_advdiff2d(nx, ny, cfg["dx"], cfg["diff"], cfg["vel"])
    vh = np.fft.fft2(v.reshape(ny, nx))
    return np.stack([np.real(np.fft.ifft2(phi(k, h * lam) * vh)).reshape(-1)
                     for k in range(p + 1)])


def phi_products_fft_adr3d(cfg: dict, v: np.ndarray, h: float, p: int, r_const: float) -> np.ndarray:
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    lam = operators.fourier_symbol_adr3d(nx, ny, nz, cfg["dx"], cfg["diff"], cfg["vel"], r_const)
    vh = np.fft.fftn(v.reshape(nz, ny, nx))
    return np.stack([np.real(np.fft.ifftn(phi(k, h * lam) * vh)).reshape(-1)
                     for k in range(p + 1)])


def scipy_expm(A):
    """Library cross-check for the oracle's own Taylor exponential."""
    return scipy.linalg.expm(A)
