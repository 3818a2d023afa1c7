"""Exponential integrators of Sect. 4 built on phi-function linear combinations
(oracle; test infrastructure only, see the package docstring).

The problem is u' = F(u) (Sect. 2).  At u_n: J_n = dF/du(u_n), f_n = F(u_n),
and the nonlinear remainder R_n(z) = F(z) - f_n - J_n (z - u_n) (Sect. 2).

* EPI4 and EPI5, the exponential multistep methods of Sect. 4:
      u_{n+1} = u_n + phi_1(h J_n) h f_n + sum_{k=1}^{M} phi_k(h J_n) v_k,
      v_k = sum_{i=1}^{P} alpha_{k,i} h R_n(u_{n-i}),
  with the coefficient matrices A_4 (3 x 2) and A_5 (4 x 3) of Sect. 4 (row
  k, column i; their first rows are zero).  The printed A_6 (4 x 4) is not
  used: read the same way it gives order 2, not 6 (a row for phi_5 appears to
  be missing).  The paper gives no starting procedure for u_{-1}, ...,
  u_{-P}; ``integrate`` takes the first P steps with SRERK3.
* SRERK3, the stiffly resilient exponential Runge-Kutta method of Sect. 4:
      z_1     = u_n + phi_1(3/4 h J_n) 3/4 h f_n,
      u_{n+1} = u_n + phi_1(h J_n) h f_n + phi_3(h J_n) 32/9 h R_n(z_1).

Every combination sum_k phi_k(tau J) c_k is handed to ``lincomb(J, bs, tau)``
as sum_k tau^k phi_k(tau J) b_k with b_k = c_k / tau^k (Sect. 2.1, Eqs. 7-9),
so one call per stage and one per step, as in the paper.  ``lincomb`` is the
dense augmented exponential for tiny problems or the Krylov projection of
``lincomb.lincomb_krylov``.
"""
from __future__ import annotations

import numpy as np

from . import operators as OP
from .exact import phi_combination_dense
from .lincomb import lincomb_krylov

EPI_ALPHA = {
    4: np.array([[0.0, 0.0],
                 [-3.0 / 10.0, 3.0 / 40.0],
                 [32.0 / 5.0, -11.0 / 10.0]]),
    5: np.array([[0.0, 0.0, 0.0],
                 [-4.0 / 5.0, 2.0 / 5.0, -4.0 / 45.0],
                 [12.0, -9.0 / 2.0, 8.0 / 9.0],
                 [3.0, 0.0, -1.0 / 3.0]]),
}


def grayscott_problem(cfg: dict):
    """F and J of the Gray-Scott system whose Jacobian is ``operators.grayscott2d``:
    F(u, v) = [Du Lap u - u v^2 + F (1 - u);  Dv Lap v + u v^2 - (F + k) v]."""
    nx, ny, dx = cfg["nx"], cfg["ny"], cfg["dx"]
    Du, Dv, Fr, k = cfg["diff"], cfg["diff2"], cfg["F"], cfg["k"]
    n = nx * ny
    lap = OP._axis_ops((nx, ny), [OP.second_difference(nx, dx), OP.second_difference(ny, dx)])

    def F(w):
        u, v = w[:n], w[n:]
        return np.concatenate([Du * (lap @ u) - u * v * v + Fr * (1.0 - u),
                               Dv * (lap @ v) + u * v * v - (Fr + k) * v])

    def J(w):
        return OP.grayscott2d(nx, ny, dx, Du, Dv, Fr, k, w[:n], w[n:])

    return F, J


def linear_problem(A):
    """u' = A u (R is then identically zero)."""
    return (lambda w: A @ w), (lambda w: A)


def dense_lincomb(J, bs, tau):
    J = J.toarray() if hasattr(J, "toarray") else np.asarray(J)
    return phi_combination_dense(J, bs, tau)


def krylov_lincomb(m, nsub=1, variant="mgs"):
    def lc(J, bs, tau):
        return lincomb_krylov(lambda x: J @ x, bs, tau, m, nsub, variant)[0]
    return lc


def _combo(lincomb, J, cs, h):
    """sum_k phi_k(h J) c_k (c_0 .. c_p; None = zero) as one linear combination."""
    p = len(cs) - 1
    N = next(c for c in cs if c is not None).size
    bs = [np.zeros(N) if c is None else c / h ** k for k, c in enumerate(cs)]
    while p > 0 and cs[p] is None:
        p -= 1
    return lincomb(J, bs[:p + 1], h)


def srerk3_step(F, Jf, u, h, lincomb):
    f = F(u)
    J = Jf(u)
    z1 = u + _combo(lincomb, J, [None, 0.75 * h * f], 0.75 * h)
    R1 = F(z1) - f - J @ (z1 - u)
    return u + _combo(lincomb, J, [None, h * f, None, (32.0 / 9.0) * h * R1], h)


def epi_step(order, F, Jf, hist, h, lincomb):
    """One EPI step from hist = [u_n, u_{n-1}, ..., u_{n-P}]."""
    alpha = EPI_ALPHA[order]
    M, P = alpha.shape
    u = hist[0]
    f = F(u)
    J = Jf(u)
    R = [F(hist[i]) - f - J @ (hist[i] - u) for i in range(1, P + 1)]
    cs = [None] * (M + 1)
    cs[1] = h * f
    for k in range(1, M + 1):
        vk = sum(alpha[k - 1, i - 1] * h * R[i - 1] for i in range(1, P + 1))
        cs[k] = vk if cs[k] is None else cs[k] + vk
    return u + _combo(lincomb, J, cs, h)


def integrate(method: str, F, Jf, u0, h, nsteps, lincomb, history=None):
    """nsteps steps of 'srerk3', 'epi4' or 'epi5' from u0.  ``history``
    (u_{-1}, u_{-2}, ...) replaces the SRERK3 start of the multistep methods."""
    u = np.asarray(u0, dtype=np.float64).copy()
    if method == "srerk3":
        for _ in range(nsteps):
            u = srerk3_step(F, Jf, u, h, lincomb)
        return u
    order = int(method[3:])
    P = EPI_ALPHA[order].shape[1]
    hist = [u] + (list(history) if history is not None else [])
    done = 0
    while len(hist) < P + 1 and done < nsteps:          # SRERK3 start
        hist.insert(0, srerk3_step(F, Jf, hist[0], h, lincomb))
        done += 1
    for _ in range(done, nsteps):
        hist.insert(0, epi_step(order, F, Jf, hist[:P + 1], h, lincomb))
        hist = hist[:P + 1]
    return hist[0]
