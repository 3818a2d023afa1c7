"""O-Krylov: phi_k(hA) v, k = 0..p, by Arnoldi projection (oracle).

Sect. 2.2, Eq. 13: e^{hA} v ~ beta V_m e^{h H_m} e_1.  The phi_k are read off
one exponential of the small augmented matrix -- the (m+p+1)-sized analogue of
Eqs. 8-9 with J -> h H_m and B -> [e_1, 0, ..., 0]:

    Hhat = [[h H_m, e_1, 0], [0, 0, I_p], [0, 0, 0]]
    exp(Hhat)[:m, 0]       = e^{h H_m} e_1
    exp(Hhat)[:m, m+k-1]   = phi_k(h H_m) e_1,   k = 1..p+1.

y_k = beta V_m exp(Hhat)[:m, col_k].  The extra column phi_{p+1} feeds the
a-posteriori error estimate err = beta h H_{m+1,m} |e_m^T phi_{p+1}(h H_m) e_1|
(a standard Saad-type estimate; the paper leaves the estimate to KIOPS).
"""
from __future__ import annotations

import numpy as np

from .arnoldi import arnoldi
from .expm import expm_taylor


def augmented_hessenberg(H: np.ndarray, h: float, p: int) -> np.ndarray:
    m = H.shape[1]
    n = m + p + 1
    Hh = np.zeros((n, n))
    Hh[:m, :m] = h * H[:m, :m]
    Hh[0, m] = 1.0
    for i in range(p):
        Hh[m + i, m + i + 1] = 1.0
    return Hh


def small_phi_coeffs(H: np.ndarray, h: float, p: int, expm=None):
    """Columns c_k = phi_k(h H_m) e_1 (k = 0..p+1) from one exponential."""
    expm = expm or expm_taylor
    m = H.shape[1]
    E = expm(augmented_hessenberg(H, h, p))
    cols = [E[:m, 0]] + [E[:m, m + k - 1] for k in range(1, p + 2)]
    return np.stack(cols)           # (p+2, m)


def phiv(matvec, v, h, p, m, variant="mgs", expm=None):
    """Returns (y, info): y is (p+1, N) with y_k ~ phi_k(hA) v."""
    v = np.asarray(v, dtype=np.float64)
    m = int(min(m, v.size))
    res = arnoldi(matvec, v, m, variant)
    me = res["m_eff"]
    H, V, beta = res["H"], res["V"], res["beta"]
    c = small_phi_coeffs(H[:me, :me] if me < m else H, h, p, expm)   # (p+2, me)
    y = beta * (c[:p + 1] @ V[:, :me].T)
    if res["breakdown"]:
        err = 0.0
    else:
        err = beta * h * H[me, me - 1] * abs(c[p + 1][me - 1])
    info = dict(res, err_est=err, coeffs=c)
    return y, info
