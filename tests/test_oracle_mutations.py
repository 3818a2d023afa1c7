"""Planted mistakes in the oracle (on the CPU) must trip at least one pin.

Each case monkeypatches one plausible slip -- a dropped term, a wrong sign, a
wrong index, a transposed operand -- and checks that the pins which should
guard that spot report a large discrepancy."""
import numpy as np

from oracle import arnoldi as OA
from oracle import krylov as OK
from oracle import operators as OP
from tests import pins


def test_cwy_sign_slip_is_caught(monkeypatch):
    def bad_form(self, temp, j):
        T = self.T
        T[j - 1, :j - 1] = +(temp[:j - 1, 0] @ T[:j - 1, :j - 1])   # sign flipped
        return T[:j, :j] @ temp[:j, 1]
    monkeypatch.setattr(OA.CWY, "form", bad_form)
    assert pins.pin_cwy_projector_identity() > 1e-3
    assert pins.pin_t3_worked_example() > 1e-3


def test_cwy_dropped_product_is_caught(monkeypatch):
    # dropping the T_{j-1} factor turns CWY into NCWY: the T_3 example catches it
    monkeypatch.setattr(OA.CWY, "form", OA.NCWY.form)
    assert pins.pin_t3_worked_example() > 1e-4
    assert pins.pin_cwy_projector_identity() > 1e-4


def test_gsmgs_transposed_splitting_is_caught(monkeypatch):
    def bad_form(self, temp, j):
        M, Minv, N = self.M, self.Minv, self.N
        M[j - 1, :j - 1] = temp[:j - 1, 0]
        N[:j - 1, j - 1] = -temp[:j - 1, 0]
        Minv[j - 1, :j - 1] = -(temp[:j - 1, 0] @ Minv[:j - 1, :j - 1])
        pvec = temp[:j, 1] + N[:j, :j].T @ (Minv[:j, :j] @ temp[:j, 1])   # N transposed
        return np.linalg.solve(M[:j, :j], pvec)
    monkeypatch.setattr(OA.GSMGS, "form", bad_form)
    assert pins.pin_gsmgs_two_sweeps() > 1e-3


def test_hybrid_without_correction_is_caught(monkeypatch):
    # T left at the identity: the hybrid step becomes classical Gram-Schmidt once
    def no_correction(self, temp, j):
        return temp[:j, 1].copy()
    monkeypatch.setattr(OA.CWY, "form", no_correction)
    assert pins.pin_orthogonality_laws() > 10.0


def test_cgs2_single_pass_is_caught(monkeypatch):
    def cgs_once(matvec, b, m):
        b = np.asarray(b, dtype=np.float64)
        V = np.zeros((b.size, m + 1))
        H = np.zeros((m + 1, m))
        beta = np.linalg.norm(b)
        V[:, 0] = b / beta
        for j in range(1, m + 1):
            w = matvec(V[:, j - 1])
            H[:j, j - 1] = V[:, :j].T @ w      # the second projection left out
            w = w - V[:, :j] @ H[:j, j - 1]
            H[j, j - 1] = np.linalg.norm(w)
            V[:, j] = w / H[j, j - 1]
        return dict(V=V, H=H, beta=beta, m_eff=m, syncs=[2] * m, fallbacks=0, breakdown=False)
    monkeypatch.setitem(OA.VARIANTS, "cgs2", cgs_once)
    assert pins.pin_orthogonality_laws() > 10.0


def test_hybrid_missing_second_scaling_is_caught(monkeypatch):
    orig = OA.hybrid

    def bad_hybrid(matvec, b, m, variant="hcwy"):
        # scale A by the first true norm: models forgetting one 1/true_nrm on temp
        state = {}
        def mv(x):
            return matvec(x) * state.setdefault("s", 1.0 + 1e-3)
        return orig(mv, b, m, variant)
    monkeypatch.setattr(OA, "hybrid", bad_hybrid)
    monkeypatch.setitem(OA.VARIANTS, "hcwy", lambda f, b, m: bad_hybrid(f, b, m, "hcwy"))
    assert pins.pin_variants_equal_mgs(("hcwy",)) > 1e-4


def test_augmentation_index_slip_is_caught(monkeypatch):
    def bad_aug(H, h, p):
        m = H.shape[1]
        n = m + p + 1
        Hh = np.zeros((n, n))
        Hh[:m, :m] = h * H[:m, :m]
        Hh[m - 1, m] = 1.0                     # e_m instead of e_1
        for i in range(p):
            Hh[m + i, m + i + 1] = 1.0
        return Hh
    monkeypatch.setattr(OK, "augmented_hessenberg", bad_aug)
    assert pins.pin_krylov_vs_dense("mgs") > 1e-3
    assert pins.pin_krylov_vs_fft_config1("mgs") > 1e-3


def test_advection_sign_slip_is_caught(monkeypatch):
    orig = OP.central_difference
    monkeypatch.setattr(OP, "central_difference", lambda n, dx: -orig(n, dx))
    assert pins.pin_advdiff_fourier() > 1e-3


def test_grayscott_coupling_slip_is_caught(monkeypatch):
    import scipy.sparse as sp
    def bad(nx, ny, dx, Du, Dv, F, k, u0, v0):
        n = nx * ny
        lap = OP._axis_ops((nx, ny), [OP.second_difference(nx, dx), OP.second_difference(ny, dx)])
        I = sp.identity(n, format="csr")
        a, b = sp.diags(v0 * v0), sp.diags(2.0 * u0 * v0)
        return sp.bmat([[Du * lap - a - F * I, b], [a, Dv * lap + b - (F + k) * I]], format="csr")
    monkeypatch.setattr(OP, "grayscott2d", bad)
    assert pins.pin_grayscott_jacobian() > 1e-3


def test_adjoint_transpose_slip_is_caught(monkeypatch):
    from oracle import adjoint as OAD
    orig = OAD.grads_krylov

    def bad(A, dA, v, y_t, h, m, variant="mgs"):
        g = orig(A, dA, v, y_t, h, m, variant)
        y, _ = OK.phiv(lambda x: A @ x, g["r"], h, 1, m, variant)    # A instead of A^T
        g["dv"] = y[1]
        return g
    monkeypatch.setattr(OAD, "grads_krylov", bad)
    assert pins.pin_adjoint_finite_differences() > 1e-3


def test_adjoint_derivative_sign_slip_is_caught(monkeypatch):
    from oracle import adjoint as OAD
    orig = OAD.grayscott_parts

    def bad(cfg, inp, theta=None):
        A, dA = orig(cfg, inp, theta)
        dA[2] = -dA[2]                                                # dA/dF = +I
        return A, dA
    monkeypatch.setattr(OAD, "grayscott_parts", bad)
    # the dense reference shares dA with the Krylov gradients: the central
    # differences of the loss are the pin that sees this slip
    assert pins.pin_adjoint_finite_differences() > 1e-3


def test_adjoint_dF_closed_form_slips_are_caught(monkeypatch):
    from oracle import adjoint as OAD
    from oracle.krylov import phiv

    def plus(A, v, r, h, m, variant="mgs"):                          # phi_1 + phi_2
        y, _ = phiv(lambda x: A @ x, v, h, 2, m, variant)
        return -h * float(r @ (y[1] + y[2]))
    monkeypatch.setattr(OAD, "dF_closed_form", plus)
    assert pins.pin_adjoint_dF_closed_form() > 1e-3

    def no_h(A, v, r, h, m, variant="mgs"):                          # the factor h dropped
        y, _ = phiv(lambda x: A @ x, v, h, 2, m, variant)
        return -float(r @ (y[1] - y[2]))
    monkeypatch.setattr(OAD, "dF_closed_form", no_h)
    assert pins.pin_adjoint_dF_closed_form() > 1e-3


def test_uncounted_fallback_reduction_is_caught(monkeypatch):
    orig = OA.hybrid

    def bad(matvec, b, m, variant="hcwy"):
        r = orig(matvec, b, m, variant)
        r["syncs"] = [min(s, 1) for s in r["syncs"]]                   # fallbacks and final uncharged
        return r
    monkeypatch.setattr(OA, "hybrid", bad)
    for v in ("hcwy", "hncwy", "hgsmgs"):
        monkeypatch.setitem(OA.VARIANTS, v, lambda f, b, m, v=v: bad(f, b, m, v))
    assert pins.pin_sync_counts() > 0


def _adaptive_m_pin_fails():
    r = pins.pin_lincomb_adaptive_m()
    lo, hi = r[4], r[40]
    ok = (lo["converged"] and hi["converged"] and lo["err"] < 10.0 and hi["err"] < 10.0
          and lo["largest"] >= 10 and hi["last"] <= 20 and lo["cost_ratio"] < 0.5 and hi["cost_ratio"] < 1.0)
    return not ok


def test_adaptive_m_decay_sign_slip_is_caught(monkeypatch):
    from oracle import lincomb as OL
    orig = OL.plan_next

    def bad(kappa, m, err, tol_abs, m_min, m_max, accepted):
        return orig(None if kappa is None else 1.0 / kappa, m, err, tol_abs, m_min, m_max, accepted)
    monkeypatch.setattr(OL, "plan_next", bad)
    assert _adaptive_m_pin_fails()


def test_adaptive_m_probe_index_slip_is_caught(monkeypatch):
    from oracle import lincomb as OL
    from oracle.krylov import small_phi_coeffs

    def bad(info, dt, mp):                          # H_{mp,mp} instead of H_{mp+1,mp}
        H = info["H"]
        c = small_phi_coeffs(H[:mp, :mp], dt, 0)
        return float(info["beta"]) * abs(dt) * float(H[mp - 1, mp - 1]) * abs(float(c[1][mp - 1]))
    monkeypatch.setattr(OL, "estimate_at", bad)
    assert _adaptive_m_pin_fails()


def test_iocgs_window_slip_is_caught(monkeypatch):
    orig = OA.iocgs
    monkeypatch.setattr(OA, "iocgs", lambda f, b, m, nprev=2: orig(f, b, m, nprev=1))
    assert pins.pin_iocgs_symmetric_is_lanczos() > 1e-3 or pins.pin_iocgs_defining_properties() > 1e-3


def test_lincomb_tau_inside_augmented_matrix_is_caught(monkeypatch):
    # the printed Eq. 8 also scales A by tau inside the augmented matrix
    from oracle import lincomb as OL
    orig = OL.aug_matvec

    def bad(matvec, bs):
        return orig(lambda x: 0.7 * matvec(x), bs)
    monkeypatch.setattr(OL, "aug_matvec", bad)
    assert pins.pin_lincomb_solves_forced_ode() > 1e-3
    assert pins.pin_lincomb_substeps_vs_dense() > 1e-3


def test_lincomb_reversed_forcing_columns_are_caught(monkeypatch):
    # B = [b_1, ..., b_p] instead of [b_p, ..., b_1]
    from oracle import lincomb as OL
    orig = OL.aug_matvec
    monkeypatch.setattr(OL, "aug_matvec", lambda mv, bs: orig(mv, [bs[0]] + list(bs[1:])[::-1]))
    assert pins.pin_lincomb_solves_forced_ode() > 1e-3
    assert pins.pin_lincomb_diagonal() > 1e-3


def test_epi_coefficient_slip_is_caught(monkeypatch):
    from oracle import integrators as OI
    bad = OI.EPI_ALPHA[4].copy()
    bad[1, 0] *= 1.1
    monkeypatch.setitem(OI.EPI_ALPHA, 4, bad)
    pins._ORDER_CACHE.clear()
    try:
        assert pins.integrator_orders()["epi4"] < 3.5
    finally:
        pins._ORDER_CACHE.clear()


def test_srerk3_weight_slip_is_caught(monkeypatch):
    from oracle import integrators as OI
    orig = OI._combo

    def bad(lincomb, J, cs, h):
        if len(cs) == 4 and cs[3] is not None:
            cs = cs[:3] + [cs[3] * (3.0 / (32.0 / 9.0))]        # 3 instead of 32/9
        return orig(lincomb, J, cs, h)
    monkeypatch.setattr(OI, "_combo", bad)
    pins._ORDER_CACHE.clear()
    try:
        assert pins.integrator_orders()["srerk3"] < 2.5
    finally:
        pins._ORDER_CACHE.clear()


def test_lincomb_stale_tail_is_caught(monkeypatch):
    # sub-steps restarting the extra entries from e_p instead of exp(tK) e_p
    from oracle import lincomb as OL
    orig = OL.aug_tail
    monkeypatch.setattr(OL, "aug_tail", lambda p, t: orig(p, 0.0))
    assert pins.pin_lincomb_substeps_vs_dense() > 1e-3
    assert pins.pin_lincomb_adaptive()[0] > 1e3
