"""Small dense matrix exponential for the oracle.

The paper does not say how e^{H_m} is evaluated (Sect. 2.2, Eq. 13 only uses
it).  The oracle uses the plainest correct method: scale A by 2^-s so that
||A 2^-s||_1 <= 1, sum the Taylor series until the next term is below the
unit roundoff relative to the partial sum, and square s times.
"""
from __future__ import annotations

import math

import numpy as np


def expm_taylor(A: np.ndarray) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    nrm = np.abs(A).sum(axis=0).max() if n else 0.0
    s = max(0, int(math.ceil(math.log2(nrm)))) if nrm > 1.0 else 0
    X = A / (2.0 ** s)
    E = np.eye(n)
    term = np.eye(n)
    for k in range(1, 60):
        term = term @ X / k
        E = E + term
        if np.abs(term).max() <= 1e-18 * max(1.0, np.abs(E).max()):
            break
    for _ in range(s):
        E = E @ E
    return E
