"""Arnoldi processes of the paper, written plainly in the paper's order (oracle).

All functions take ``matvec`` (a callable v -> A v), the start vector b and the
subspace size m, and return a dict with
  V        N x (m_eff+1) basis (orthonormal in exact arithmetic)
  H        (m_eff+1) x m_eff upper Hessenberg matrix
  beta     ||b||
  m_eff    number of completed steps (< m after a lucky breakdown)
  syncs    list: global reductions charged to each step (final norm included
           in the last entry for the hybrid method)
  fallbacks number of explicit-norm fallbacks (hybrid only)

Breakdown threshold (the paper only says "nrm ~ 0", Alg. 1 and Alg. 4): a step
breaks down when the new vector's norm is <= BREAKDOWN_TOL * ||A v_j||.
"""
from __future__ import annotations

import numpy as np

BREAKDOWN_TOL = 1e-13


def mgs(matvec, b, m):
    """Alg. 1: Arnoldi with modified Gram-Schmidt; j+1 global syncs at step j."""
    b = np.asarray(b, dtype=np.float64)
    N = b.size
    V = np.zeros((N, m + 1))
    H = np.zeros((m + 1, m))
    beta = np.linalg.norm(b)
    V[:, 0] = b / beta
    syncs = []
    m_eff = m
    for j in range(1, m + 1):               # paper's j
        w = matvec(V[:, j - 1])              # v_{j+1} = A v_j
        nrm_aw = np.linalg.norm(w)
        for i in range(1, j + 1):            # orthogonalise against v_1..v_j
            H[i - 1, j - 1] = V[:, i - 1] @ w        # global sync
            w = w - H[i - 1, j - 1] * V[:, i - 1]
        nrm = np.linalg.norm(w)              # global sync
        syncs.append(j + 1)
        H[j, j - 1] = nrm
        if nrm <= BREAKDOWN_TOL * nrm_aw:    # lucky breakdown
            m_eff = j
            break
        V[:, j] = w / nrm
    return dict(V=V[:, :m_eff + 1], H=H[:m_eff + 1, :m_eff], beta=beta, m_eff=m_eff,
                syncs=syncs, fallbacks=0, breakdown=m_eff < m)


def cgs2(matvec, b, m):
    """Classical Gram-Schmidt applied twice (textbook; Sect. 2.3 names classical
    GS and its sync count).  3 global syncs per step: V^T w, V^T w again, ||w||."""
    b = np.asarray(b, dtype=np.float64)
    N = b.size
    V = np.zeros((N, m + 1))
    H = np.zeros((m + 1, m))
    beta = np.linalg.norm(b)
    V[:, 0] = b / beta
    syncs = []
    m_eff = m
    for j in range(1, m + 1):
        w = matvec(V[:, j - 1])
        nrm_aw = np.linalg.norm(w)
        Vj = V[:, :j]
        h1 = Vj.T @ w                         # global sync
        w = w - Vj @ h1
        h2 = Vj.T @ w                         # global sync
        w = w - Vj @ h2
        H[:j, j - 1] = h1 + h2
        nrm = np.linalg.norm(w)               # global sync
        syncs.append(3)
        H[j, j - 1] = nrm
        if nrm <= BREAKDOWN_TOL * nrm_aw:
            m_eff = j
            break
        V[:, j] = w / nrm
    return dict(V=V[:, :m_eff + 1], H=H[:m_eff + 1, :m_eff], beta=beta, m_eff=m_eff,
                syncs=syncs, fallbacks=0, breakdown=m_eff < m)


def iocgs(matvec, b, m, nprev=2):
    """Incomplete orthogonalisation (Sect. 2.3.1, IOP; the paper's reference
    baseline ioCGS): A v_j is orthogonalised against the previous ``nprev``
    basis vectors only, classically -- their inner products in one global
    sync, then the norm in a second (2 syncs per step).  The basis is not
    orthonormal and H is banded (entries j-nprev+1..j+1 of column j); the phi
    products use H and V as they are."""
    b = np.asarray(b, dtype=np.float64)
    N = b.size
    V = np.zeros((N, m + 1))
    H = np.zeros((m + 1, m))
    beta = np.linalg.norm(b)
    V[:, 0] = b / beta
    syncs = []
    m_eff = m
    for j in range(1, m + 1):
        w = matvec(V[:, j - 1])
        nrm_aw = np.linalg.norm(w)
        lo = max(1, j - nprev + 1)              # v_lo .. v_j
        Vp = V[:, lo - 1:j]
        h = Vp.T @ w                            # global sync
        w = w - Vp @ h
        H[lo - 1:j, j - 1] = h
        nrm = np.linalg.norm(w)                 # global sync
        syncs.append(2)
        H[j, j - 1] = nrm
        if nrm <= BREAKDOWN_TOL * nrm_aw:
            m_eff = j
            break
        V[:, j] = w / nrm
    return dict(V=V[:, :m_eff + 1], H=H[:m_eff + 1, :m_eff], beta=beta, m_eff=m_eff,
                syncs=syncs, fallbacks=0, breakdown=m_eff < m)


# ---------------------------------------------------------------------------
# Correction matrices of the hybrid method.  ``temp`` is the (j+1) x 2 array of
# Alg. 4 after its scalings; j is the paper's step index (1-based).

class CWY:
    """Alg. 5 (Sect. 3.2.1): T_{j,1:j-1} = -temp_{1:j-1,1}^T T_{1:j-1,1:j-1};
    H_{1:j,j} = T_j temp_{1:j,2}.  T is initialised to I_m (Alg. 4)."""

    def __init__(self, m):
        self.T = np.eye(m)

    def form(self, temp, j):
        T = self.T
        T[j - 1, :j - 1] = -(temp[:j - 1, 0] @ T[:j - 1, :j - 1])
        return T[:j, :j] @ temp[:j, 1]


class NCWY:
    """Alg. 6 (Sect. 3.2.2): two-term Neumann truncation T = I - L,
    T_{j,1:j-1} = -temp_{1:j-1,1}^T; H_{1:j,j} = T_j temp_{1:j,2}."""

    def __init__(self, m):
        self.T = np.eye(m)

    def form(self, temp, j):
        T = self.T
        T[j - 1, :j - 1] = -temp[:j - 1, 0]
        return T[:j, :j] @ temp[:j, 1]


class GSMGS:
    """Alg. 7 (Sect. 3.2.3): two Gauss-Seidel sweeps on the normal equations
    with the splitting V^T V = M - N, M = I + L, N = -L^T; M^{-1} follows the
    CWY recursion.  p = (I + N M^{-1}) temp_{1:j,2};  H_{1:j,j} solves M x = p."""

    def __init__(self, m):
        self.M = np.eye(m)
        self.Minv = np.eye(m)
        self.N = np.zeros((m, m))

    def form(self, temp, j):
        M, Minv, N = self.M, self.Minv, self.N
        M[j - 1, :j - 1] = temp[:j - 1, 0]
        N[:j - 1, j - 1] = -temp[:j - 1, 0]
        Minv[j - 1, :j - 1] = -(temp[:j - 1, 0] @ Minv[:j - 1, :j - 1])
        pvec = temp[:j, 1] + N[:j, :j] @ (Minv[:j, :j] @ temp[:j, 1])
        x = np.zeros(j)
        for r in range(j):                   # lower-triangular solve M x = p
            x[r] = (pvec[r] - M[r, :r] @ x[:r]) / M[r, r]
        return x


CORRECTIONS = {"hcwy": CWY, "hncwy": NCWY, "hgsmgs": GSMGS}


def hybrid(matvec, b, m, variant="hcwy"):
    """Alg. 4 (Sect. 3.3): hybrid low-synchronisation Arnoldi, one global
    reduction per step (plus the final norm and any norm-estimate fallbacks).

    Readings of the printed algorithm (the paper is ambiguous there):
      * the rescale of v_j, v_{j+1} by the previous norm estimate happens
        before the grouped reduction, so that temp_{j,1} is the true squared
        norm, as the text of Sect. 3.2.1 describes;
      * at j = 1 the correction step is skipped and H_{1,1} = temp_{1,2};
      * the written "H_{i:j,j}" is H_{1:j,j}, and "H_{j-1,j} = true_nrm" is the
        subdiagonal entry H_{j,j-1};
      * the fallback when temp_{j+1,2} < ss sets nrm_est = ||v_{j+1}|| by an
        explicit extra reduction;
      * Eq. 18's sum over i = 0..j is over i = 1..j;
      * "nrm_est ~ 0" is tested against BREAKDOWN_TOL * ||A v_j||; since the
        Pythagorean estimate cannot resolve norms below ~sqrt(eps) ||A v_j||,
        the lagged true norm of the next step (H_{j+1,j}) is tested the same
        way, and a breakdown found there ends the process at step j;
      * after the loop H_{m+1,m} = nrm_est * ||v_{m+1}||, the true norm of the
        projected vector (v_{m+1} was already divided by nrm_est).
    """
    corr = CORRECTIONS[variant](m)
    b = np.asarray(b, dtype=np.float64)
    N = b.size
    V = np.zeros((N, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = b                                         # v_1 = b, unnormalised
    nrm_est = 1.0
    beta = None
    syncs = []
    fallbacks = 0
    m_eff = m
    for j in range(1, m + 1):
        V[:, j] = matvec(V[:, j - 1])                   # v_{j+1} = A v_j
        if j > 1:
            V[:, j - 1:j + 1] *= nrm_est                # rescale by previous estimate
        temp = V[:, :j + 1].T @ V[:, j - 1:j + 1]       # one global reduction
        nsync = 1
        true_nrm = np.sqrt(temp[j - 1, 0])              # true norm of previous vector
        if j == 1:
            beta = true_nrm
        elif true_nrm <= BREAKDOWN_TOL * nrm_aw:        # lagged breakdown test
            H[j - 1, j - 2] = true_nrm
            syncs.append(nsync)
            m_eff = j - 1
            break
        V[:, j - 1:j + 1] /= true_nrm
        temp[:, 1] /= true_nrm
        temp[j - 1:j + 1, 1] /= true_nrm
        if j > 1:
            temp[:j - 1, 0] /= true_nrm
            H[:j, j - 1] = corr.form(temp, j)
            H[j - 1, j - 2] = true_nrm
        else:
            H[0, 0] = temp[0, 1]
        V[:, j] -= V[:, :j] @ H[:j, j - 1]              # project
        ss = np.sum(temp[:j, 1] ** 2)
        nrm_aw = np.sqrt(temp[j, 1])                    # ||A v_j|| (normalised v_j)
        if temp[j, 1] < ss:
            nrm_est = np.linalg.norm(V[:, j])           # explicit norm: extra reduction
            nsync += 1
            fallbacks += 1
        else:
            nrm_est = np.sqrt(temp[j, 1] - ss)          # Eq. 18
        syncs.append(nsync)
        if nrm_est <= BREAKDOWN_TOL * nrm_aw:
            H[j, j - 1] = nrm_est
            m_eff = j
            break
        V[:, j] /= nrm_est                              # "normalise" by the estimate
    if m_eff == m:
        nrm = np.linalg.norm(V[:, m])                   # final reduction
        syncs[-1] += 1
        V[:, m] /= nrm
        H[m, m - 1] = nrm_est * nrm
        Vout = V
        if H[m, m - 1] <= BREAKDOWN_TOL * nrm_aw:      # the last step exhausted the space
            return dict(V=Vout, H=H, beta=beta, m_eff=m, syncs=syncs, fallbacks=fallbacks,
                        breakdown=True)
    else:
        Vout = V[:, :m_eff + 1]
    return dict(V=Vout, H=H[:m_eff + 1, :m_eff], beta=beta, m_eff=m_eff, syncs=syncs,
                fallbacks=fallbacks, breakdown=m_eff < m)


VARIANTS = {"mgs": mgs, "cgs2": cgs2, "iocgs": iocgs,
            "hcwy": lambda f, b, m: hybrid(f, b, m, "hcwy"),
            "hncwy": lambda f, b, m: hybrid(f, b, m, "hncwy"),
            "hgsmgs": lambda f, b, m: hybrid(f, b, m, "hgsmgs")}


def arnoldi(matvec, b, m, variant="mgs"):
    return VARIANTS[variant](matvec, b, m)
