"""Gradients of a phi_1 loss on the Gray-Scott Jacobian (oracle; test
infrastructure only, see the package docstring).

The adjoint workload differentiates

    L(v, h, theta) = 1/2 || phi_1(h A(theta)) v - y_t ||^2,   theta = (Du, Dv, F, k),

with A(theta) the Gray-Scott Jacobian of ``operators.grayscott2d``.  With the
residual r = phi_1(hA)v - y_t:

  dL/dv      = phi_1(hA)^T r = phi_1(h A^T) r.  phi_1 is a power series in its
               argument (Sect. 2, Eq. 6), so transposition commutes with it.
  dL/dh      = r . (phi_0(hA)v - phi_1(hA)v) / h.  From Eq. 6, h phi_1(hA) =
               integral_0^h e^{sA} ds, whose h-derivative is e^{hA} = phi_0(hA).
  dL/dtheta  = r . a,  a = d/dtheta [phi_1(hA)v], the Frechet derivative of the
               phi-product in the direction h dA/dtheta.  Sect. 2.1 (Eq. 7)
               writes phi_1(hA)v as the first block of exp([[hA, v], [0, 0]])
               e_{N+1}; the Frechet derivative of exp at X in direction E is the
               upper-right block of exp([[X, E], [0, X]]) (block-triangular
               augmentation).  Applied to the (N+1)-sized matrix of Eq. 7 the
               scalar rows stay constant and the remaining 2N-sized system is
               z' = h K z + [0; v], z(0) = 0, K = [[A, dA/dtheta], [0, A]],
               whose value at 1 is phi_1(hK)[0; v] (Eq. 6 as the solution of the
               forced linear ODE).  So a = top half of phi_1(hK)[0; v]: one more
               phi-product, on a 2N-sized block operator.

  dL/dF      (closed form) dA/dF = -I commutes with A, so d/dF phi_1(hA)v =
               -h phi_1'(hA) v, and term by term in the series of Eq. 6
               phi_1'(z) = sum_j (j+1) z^j / (j+2)! = phi_1(z) - phi_2(z):
               dL/dF = -h r . (phi_1(hA)v - phi_2(hA)v), read off one phi
               product with p = 2 (``dF_closed_form``).

``grads_krylov`` evaluates these with O-Krylov (``krylov.phiv``);
``grads_dense`` evaluates the same derivatives for tiny N with no Krylov step
and no closed form: dense exponentials of the Eq. 7 matrix and
``scipy.linalg.expm_frechet`` along dv, dh and each dA/dtheta.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import operators as OP
from .krylov import phiv

THETA = ("Du", "Dv", "F", "k")


def grayscott_parts(cfg: dict, inp: dict, theta=None):
    """A(theta) and its partial derivatives dA/dtheta_k (sparse), theta =
    (Du, Dv, F, k); the default theta is the workload's."""
    nx, ny, dx = cfg["nx"], cfg["ny"], cfg["dx"]
    Du, Dv, F, k = theta if theta is not None else (cfg["diff"], cfg["diff2"], cfg["F"], cfg["k"])
    A = OP.grayscott2d(nx, ny, dx, Du, Dv, F, k, inp["u0"], inp["v0"])
    n = nx * ny
    lap = OP._axis_ops((nx, ny), [OP.second_difference(nx, dx), OP.second_difference(ny, dx)])
    I = sp.identity(n, format="csr")
    Z = sp.csr_matrix((n, n))
    dA = [sp.bmat([[lap, Z], [Z, Z]], format="csr"),        # d/dDu
          sp.bmat([[Z, Z], [Z, lap]], format="csr"),        # d/dDv
          sp.bmat([[-I, Z], [Z, -I]], format="csr"),        # d/dF
          sp.bmat([[Z, Z], [Z, -I]], format="csr")]         # d/dk
    return A, dA


def loss(A, v, y_t, h, m, variant="mgs"):
    y, _ = phiv(lambda x: A @ x, v, h, 1, m, variant)
    r = y[1] - y_t
    return 0.5 * float(r @ r), y


def dF_closed_form(A, v, r, h, m, variant="mgs"):
    """dL/dF = -h r . (phi_1(hA)v - phi_2(hA)v) by O-Krylov with m steps (the
    closed form above; pinned against the Frechet form and dense expm_frechet)."""
    y, _ = phiv(lambda x: A @ x, v, h, 2, m, variant)
    return -h * float(r @ (y[1] - y[2]))


def grads_krylov(A, dA, v, y_t, h, m, variant="mgs", f_closed=False):
    """L, y = (phi_0, phi_1)(hA)v and the gradients, each by O-Krylov with m
    steps.  dL/dtheta uses the block-operator (Frechet) product for every
    component, or, with f_closed, the closed form for the F component."""
    L, y = loss(A, v, y_t, h, m, variant)
    r = y[1] - y_t
    At = A.T.tocsr()
    yt, _ = phiv(lambda x: At @ x, r, h, 1, m, variant)
    g_v = yt[1]
    g_h = float(r @ (y[0] - y[1])) / h
    N = v.size
    z0 = np.concatenate([np.zeros(N), v])
    g_t = []
    for k, E in enumerate(dA):
        if f_closed and THETA[k] == "F":
            g_t.append(dF_closed_form(A, v, r, h, m, variant))
            continue
        K = sp.bmat([[A, E], [None, A]], format="csr")
        yk, _ = phiv(lambda x: K @ x, z0, h, 1, m, variant)
        g_t.append(float(r @ yk[1][:N]))
    return dict(L=L, y=y, r=r, dv=g_v, dh=g_h, dtheta=np.array(g_t))


def _aug(X, w):
    """(N+1) x (N+1) matrix [[X, w], [0, 0]] (Eq. 7 with one vector)."""
    N = X.shape[0]
    M = np.zeros((N + 1, N + 1))
    M[:N, :N] = X
    M[:N, N] = w
    return M


def grads_dense(A, dA, v, y_t, h):
    """The same quantities for tiny N from dense exponentials of Eq. 7's matrix
    and Frechet derivatives of exp (scipy.linalg.expm_frechet)."""
    A = A.toarray()
    N = A.shape[0]
    Xa = _aug(h * A, v)
    y1 = sla.expm(Xa)[:N, N]
    r = y1 - y_t
    L = 0.5 * float(r @ r)
    # dv: the map v -> phi_1(hA) v is linear; its matrix has column i = phi_1(hA) e_i
    P1 = np.stack([sla.expm(_aug(h * A, e))[:N, N] for e in np.eye(N)], axis=1)
    g_v = P1.T @ r
    # dh: direction of d(Xa)/dh = [[A, 0], [0, 0]]
    _, Lh = sla.expm_frechet(Xa, _aug(A, np.zeros(N)))
    g_h = float(r @ Lh[:N, N])
    g_t = []
    for E in dA:
        _, Lt = sla.expm_frechet(Xa, _aug(h * E.toarray(), np.zeros(N)))
        g_t.append(float(r @ Lt[:N, N]))
    return dict(L=L, y1=y1, r=r, dv=g_v, dh=g_h, dtheta=np.array(g_t))
