"""Linear combinations of phi-functions by Krylov projection of the augmented
operator, with fixed sub-stepping (oracle; test infrastructure only, see the
package docstring).

Sect. 2.1, Eqs. 7-9: for vectors b_0..b_p,

    u(tau) = sum_{j=0}^p tau^j phi_j(tau A) b_j = [I_N 0] exp(tau Aaug) [b_0; e_p],
    Aaug = [[A, B], [0, K]],  B = [b_p, ..., b_1],  K = [[0, I_{p-1}], [0, 0]].

(The printed Eq. 8 puts tau inside Aaug as well as in front of it; the reading
used here applies tau once, which is the form that reduces to the left-hand
side.  It is pinned below against the ODE u' = A u + sum_j t^{j-1}/(j-1)! b_j,
u(0) = b_0, whose solution the left-hand side is.)

The Krylov process runs on (N+p)-vectors: the product with Aaug is
A x_top + B x_bot on the first N entries and K x_bot on the last p, so only
products with A are needed (Sect. 2.1).  u is then the first N entries of
beta V_m exp(tau H_m) e_1 (Sect. 2.2, Eq. 13, with no phi augmentation of
H_m).

Sub-stepping (Sect. 2.2, the sub-step product of exponentials): tau is split
into nsub equal steps dt and w_{s+1} = exp(dt Aaug) w_s, w_0 = [b_0; e_p].
The last p entries of w evolve under K alone, so at t = s dt they are exactly
exp(t K) e_p, whose entry p-1-i is t^i / i!; each sub-step restarts from the
Krylov result for the first N entries and these exact last p entries.  (The
paper chooses sub-step sizes and dimensions adaptively as in KIOPS, whose
formulas it does not reproduce; this oracle uses equal steps and a fixed m.)
"""
from __future__ import annotations

import math

import numpy as np

from .krylov import phiv


def aug_tail(p: int, t: float) -> np.ndarray:
    """exp(t K) e_p: entry p-1-i is t^i / i! (K the p x p upper shift)."""
    xi = np.zeros(p)
    for i in range(p):
        xi[p - 1 - i] = t ** i / math.factorial(i)
    return xi


def aug_matvec(matvec, bs):
    """x -> Aaug x for x of length N+p (Eqs. 8-9): [A x_top + B x_bot; K x_bot]."""
    p = len(bs) - 1
    N = np.asarray(bs[0]).size
    cols = [np.asarray(bs[p - k], dtype=np.float64) for k in range(p)]   # B = [b_p, ..., b_1]

    def mv(x):
        top = np.asarray(matvec(x[:N]), dtype=np.float64).copy()
        for k in range(p):
            top += x[N + k] * cols[k]
        bot = np.zeros(p)
        bot[:p - 1] = x[N + 1:N + p]
        return np.concatenate([top, bot])

    return mv


def lincomb_krylov(matvec, bs, tau: float, m: int, nsub: int = 1, variant: str = "mgs"):
    """u = sum_j tau^j phi_j(tau A) b_j in nsub equal sub-steps, each an m-step
    Krylov projection of Aaug.  Returns (u, infos) with one info per sub-step."""
    bs = [np.asarray(b, dtype=np.float64) for b in bs]
    p = len(bs) - 1
    N = bs[0].size
    mv = aug_matvec(matvec, bs)
    dt = tau / nsub
    u = bs[0].copy()
    infos = []
    for s in range(nsub):
        w0 = np.concatenate([u, aug_tail(p, s * dt)])
        y, info = phiv(mv, w0, dt, 0, m, variant)
        u = y[0][:N].copy()
        infos.append(info)
    return u, infos


def step_factor(err: float, tol_abs: float, m: int) -> float:
    """Sub-step size factor of the adaptive control (this build's controller; the
    paper takes KIOPS's, which it does not reproduce): 0.9 (tol/err)^(1/(m+1)),
    clamped to [0.2, 4]; 4 when the estimate is zero (exact projection)."""
    if err <= 0.0:
        return 4.0
    return min(4.0, max(0.2, 0.9 * (tol_abs / err) ** (1.0 / (m + 1))))


def lincomb_adaptive(matvec, bs, tau: float, m: int, tol: float, nsub0: int = 1,
                     variant: str = "mgs", max_substeps: int = 100000):
    """u = sum_j tau^j phi_j(tau A) b_j in sub-steps chosen by the a-posteriori
    estimate err = beta dt H_{m+1,m} |e_m^T phi_1(dt H_m) e_1| of each projection:
    a sub-step is accepted when err <= tol * beta (beta the norm of its augmented
    start vector) and the next size is dt * step_factor; a rejected one is
    retried with dt * min(0.9, step_factor).  A sub-step shorter than
    tau * 2^-30 is accepted regardless (reported as not converged).  Starts with
    dt = tau / nsub0.  Returns (u, info) with the accepted sizes, the number of
    rejections and whether every accepted step met the tolerance."""
    bs = [np.asarray(b, dtype=np.float64) for b in bs]
    p = len(bs) - 1
    N = bs[0].size
    mv = aug_matvec(matvec, bs)
    m = min(m, N + p)
    u = bs[0].copy()
    t, dt = 0.0, tau / nsub0
    sizes, rejected, converged = [], 0, True
    floor = abs(tau) * 2.0 ** -30
    while len(sizes) + rejected < max_substeps:
        last = abs(dt) >= abs(tau - t)
        if last:
            dt = tau - t
        w0 = np.concatenate([u, aug_tail(p, t)])
        y, info = phiv(mv, w0, dt, 0, m, variant)
        err = 0.0 if info["breakdown"] else abs(float(info["err_est"]))
        tol_abs = tol * float(info["beta"])
        if err <= tol_abs or abs(dt) <= floor:
            if err > tol_abs:
                converged = False
            u = y[0][:N].copy()
            sizes.append(dt)
            if last:
                return u, dict(sizes=sizes, rejected=rejected, converged=converged)
            t += dt
            dt *= step_factor(err, tol_abs, m)
        else:
            rejected += 1
            dt *= min(0.9, step_factor(err, tol_abs, m))
    return u, dict(sizes=sizes, rejected=rejected, converged=False)


# --- sub-steps with adaptive size and adaptive Krylov dimension ---------------
#
# Sect. 2.2 chooses both the sub-step size and the Krylov dimension of every
# sub-step adaptively "as in KIOPS", whose formulas the paper does not give.
# The rule below is this build's own.  After a projection of dimension m over a
# sub-step dt with estimate err (the one of ``lincomb_adaptive``):
#
#   * error model: err(dt', m') = err kappa^(m - m') (dt'/dt)^(m'+1), the
#     power of dt' being the one ``step_factor`` assumes and kappa, the decay
#     of the error per Krylov dimension, measured on the same projection: its
#     estimate at the smaller dimension m - DM_PROBE gives
#     kappa = (err(m - DM_PROBE) / err)^(1 / DM_PROBE);
#   * for every m' in [m_min, m_max] the size factor that brings the model to
#     0.9^(m'+1) tol beta is f(m') = 0.9 (tol beta / (err kappa^(m - m')))^(1/(m'+1))
#     clamped to [0.2, 4]; at m' = m this is ``step_factor``.  After a
#     rejection only m' >= m is considered and f is capped at 0.9 (the retry
#     never takes a longer sub-step or a smaller space);
#   * the next sub-step takes the m' with the smallest modeled cost per unit of
#     time W(m') / (dt f(m')), W(m) = sum_{j=1..m} (j + 3) = m(m+1)/2 + 3m the
#     vectors of length N one m-step hybrid projection streams (step j reads j
#     basis columns and the source and writes two); m changes only when that
#     cost is below HYST times the cost of keeping m (against oscillation);
#   * when kappa cannot be measured (an exact projection, m - DM_PROBE < 1, a
#     breakdown) or kappa <= KAPPA_MIN (more dimensions would not pay), m stays
#     and only the size adapts, as in ``lincomb_adaptive``.

KAPPA_MIN = 1.05    # smallest useful error decay per added Krylov dimension
HYST = 0.9          # a new dimension must cut the modeled cost by 10 %
DM_PROBE = 2        # the decay is measured between m - DM_PROBE and m


def projection_cost(m: int) -> float:
    """W(m): vectors of length N streamed by one m-step hybrid projection."""
    return m * (m + 1) / 2.0 + 3.0 * m


def estimate_at(info, dt: float, mp: int) -> float:
    """The a-posteriori estimate of the same projection truncated to dimension
    mp: beta dt H_{mp+1,mp} |e_mp^T phi_1(dt H_mp) e_1| (Eq. 13's projection
    with the Hessenberg matrix's leading mp x mp block)."""
    from .krylov import small_phi_coeffs

    H = info["H"]
    c = small_phi_coeffs(H[:mp, :mp], dt, 0)
    return float(info["beta"]) * abs(dt) * float(H[mp, mp - 1]) * abs(float(c[1][mp - 1]))


def error_decay(info, dt: float, m: int, err: float):
    """kappa of the rule above, or None when it cannot be measured or is too weak."""
    mp = m - DM_PROBE
    if info["m_eff"] < m or not (err > 0.0) or mp < 1:
        return None
    e_p = estimate_at(info, dt, mp)
    if not (e_p > err):
        return None
    kappa = (e_p / err) ** (1.0 / DM_PROBE)
    return kappa if kappa > KAPPA_MIN else None


def plan_next(kappa, m: int, err: float, tol_abs: float, m_min: int, m_max: int, accepted: bool):
    """(m', f): the next dimension and the factor on the sub-step size."""
    def factor(mp):
        f = 0.9 * (tol_abs / (err * kappa ** (m - mp))) ** (1.0 / (mp + 1))
        f = min(4.0, max(0.2, f))
        return f if accepted else min(f, 0.9)

    f_keep = step_factor(err, tol_abs, m)
    f_keep = f_keep if accepted else min(0.9, f_keep)
    if kappa is None:
        return m, f_keep
    keep = projection_cost(m) / f_keep
    best = (keep, m, f_keep)
    for mp in range(m_min if accepted else m, m_max + 1):
        if mp == m:
            continue
        f = factor(mp)
        c = projection_cost(mp) / f
        if c < best[0]:
            best = (c, mp, f)
    return (best[1], best[2]) if best[0] < HYST * keep else (m, f_keep)


def lincomb_adaptive_m(matvec, bs, tau: float, m0: int, tol: float, m_min: int = 4, m_max: int = 64,
                       nsub0: int = 1, variant: str = "mgs", max_substeps: int = 100000):
    """u = sum_j tau^j phi_j(tau A) b_j in sub-steps whose size and Krylov
    dimension both adapt (the rule above).  Acceptance, the size floor and the
    first size tau / nsub0 are those of ``lincomb_adaptive``; the first
    dimension is m0.  Returns (u, info) with the accepted sizes and dimensions,
    the number of rejections and whether every accepted step met the tolerance."""
    bs = [np.asarray(b, dtype=np.float64) for b in bs]
    p = len(bs) - 1
    N = bs[0].size
    mv = aug_matvec(matvec, bs)
    m_max = min(m_max, N + p)
    m_min = max(1, min(m_min, m_max))
    m = int(min(m_max, max(m_min, m0)))
    u = bs[0].copy()
    t, dt = 0.0, tau / nsub0
    sizes, dims, rejected, converged = [], [], 0, True
    floor = abs(tau) * 2.0 ** -30
    while len(sizes) + rejected < max_substeps:
        last = abs(dt) >= abs(tau - t)
        if last:
            dt = tau - t
        w0 = np.concatenate([u, aug_tail(p, t)])
        y, info = phiv(mv, w0, dt, 0, m, variant)
        err = 0.0 if info["breakdown"] else abs(float(info["err_est"]))
        tol_abs = tol * float(info["beta"])
        accept = err <= tol_abs or abs(dt) <= floor
        kappa = error_decay(info, dt, m, err)
        if accept:
            if err > tol_abs:
                converged = False
            u = y[0][:N].copy()
            sizes.append(dt)
            dims.append(m)
            if last:
                return u, dict(sizes=sizes, dims=dims, rejected=rejected, converged=converged)
            t += dt
        else:
            rejected += 1
        m, f = plan_next(kappa, m, err, tol_abs, m_min, m_max, accept)
        dt *= f
    return u, dict(sizes=sizes, dims=dims, rejected=rejected, converged=False)
