"""Pins of the CPU oracle against facts it does not itself compute.

Each function returns a scalar discrepancy (0 when the oracle is right) so that
``test_oracle_*`` assert it is small and ``test_oracle_mutations`` can check
that a planted mistake in the oracle makes at least one of them large.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import scipy.linalg
import scipy.sparse.linalg

import workloads as W
from oracle import adjoint as OAD
from oracle import arnoldi as OA
from oracle import exact as OE
from oracle import expm as OX
from oracle import krylov as OK
from oracle import integrators as OI
from oracle import lincomb as OL
from oracle import operators as OP
from oracle import phi as OPHI

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit_vectors(N, j, coupling, seed):
    """j random unit vectors with mutual inner products of order ``coupling``."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((N, j)))
    V = Q + coupling * rng.standard_normal((N, j)) / math.sqrt(N)
    return V / np.linalg.norm(V, axis=0)


def drive_correction(cls, V, b=None):
    """Feed the hybrid correction class the inner products of the columns of V
    step by step (temp column 1 = V_{1:j-1}^T v_j), as Alg. 4 would; at the
    last step column 2 is b.  Returns (object, result of the last form())."""
    j = V.shape[1]
    obj = cls(j)
    out = None
    for jj in range(2, j + 1):
        temp = np.zeros((jj + 1, 2))
        temp[:jj - 1, 0] = V[:, :jj - 1].T @ V[:, jj - 1]
        temp[:jj, 1] = b[:jj] if (b is not None and jj == j) else 0.0
        out = obj.form(temp, jj)
    return obj, out


# --- phi -------------------------------------------------------------------

def pin_phi_at_zero():
    return max(abs(OPHI.phi(k, 0.0) - 1.0 / math.factorial(k)) for k in range(8))


def pin_phi_quadrature():
    err = 0.0
    for z in [1e-6, -0.3, 0.9, 1.9, 2.1, -7.5, 3.0 + 4.0j, -0.5 + 0.1j, -12.0 - 6.0j]:
        for k in range(5):
            ref = OPHI.phi_quadrature(k, z)
            val = complex(OPHI.phi(k, np.array([z], dtype=complex))[0])
            err = max(err, abs(val - ref) / max(1e-300, abs(ref)))
    return err


# --- small exponential -----------------------------------------------------

def pin_expm_vs_scipy():
    rng = np.random.default_rng(7)
    err = 0.0
    for n, scale in [(5, 0.1), (12, 3.0), (33, 8.0), (41, 20.0)]:
        A = rng.standard_normal((n, n)) * scale / math.sqrt(n)
        E = OX.expm_taylor(A)
        R = scipy.linalg.expm(A)
        err = max(err, np.linalg.norm(E - R) / np.linalg.norm(R))
    return err


def pin_expm_nilpotent_shift():
    n = 7
    S = np.diag(np.ones(n - 1), 1)
    ref = sum(np.linalg.matrix_power(S, k) / math.factorial(k) for k in range(n))
    return np.abs(OX.expm_taylor(S) - ref).max()


def pin_expm_diagonal():
    lam = np.array([-30.0, -1.0, 0.0, 0.5, 4.0])
    return np.abs(OX.expm_taylor(np.diag(lam)) - np.diag(np.exp(lam))).max() / math.exp(4.0)


# --- operators ---------------------------------------------------------------

def pin_advdiff_fourier(cfg=None):
    cfg = cfg or W.advdiff2d(8, ny=6, vel=(1.0, -0.5))
    nx, ny = cfg["nx"], cfg["ny"]
    A = OP.advdiff2d(nx, ny, cfg["dx"], cfg["diff"], cfg["vel"])
    lam = OP.fourier_symbol_advdiff2d(nx, ny, cfg["dx"], cfg["diff"], cfg["vel"])
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    err = 0.0
    for kx in range(nx):
        for ky in range(ny):
            mode = np.exp(2j * np.pi * (kx * ix / nx + ky * iy / ny)).reshape(-1)
            err = max(err, np.abs(A @ mode - lam[ky, kx] * mode).max() / (1 + abs(lam[ky, kx])))
    return err


def pin_adr_fourier():
    nx, ny, nz, dx = 5, 4, 3, 0.2
    vel = (1.0, 0.5, -2.0)
    A = OP.adr3d(nx, ny, nz, dx, 0.03, vel, np.full(nx * ny * nz, -0.25))
    lam = OP.fourier_symbol_adr3d(nx, ny, nz, dx, 0.03, vel, -0.25)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    err = 0.0
    for kx in range(nx):
        for ky in range(ny):
            for kz in range(nz):
                mode = np.exp(2j * np.pi * (kx * ix / nx + ky * iy / ny + kz * iz / nz)).reshape(-1)
                err = max(err, np.abs(A @ mode - lam[kz, ky, kx] * mode).max())
    return err


def grayscott_rhs(u, v, nx, ny, dx, Du, Dv, F, k):
    """The Gray-Scott PDE right-hand side with a periodic 5-point Laplacian,
    written with np.roll on (ny, nx) fields."""
    def lap(f):
        f = f.reshape(ny, nx)
        return ((np.roll(f, 1, 0) + np.roll(f, -1, 0) + np.roll(f, 1, 1) + np.roll(f, -1, 1)
                 - 4 * f) / dx**2).reshape(-1)
    return (Du * lap(u) - u * v * v + F * (1 - u), Dv * lap(v) + u * v * v - (F + k) * v)


def pin_grayscott_jacobian():
    nx, ny, dx = 7, 5, 0.3
    Du, Dv, F, k = 2e-2, 1e-2, 0.04, 0.06
    rng = np.random.default_rng(3)
    u0, v0 = rng.uniform(0, 1, nx * ny), rng.uniform(0, 1, nx * ny)
    J = OP.grayscott2d(nx, ny, dx, Du, Dv, F, k, u0, v0)
    d = rng.uniform(-1, 1, 2 * nx * ny)
    eps = 1e-6
    n = nx * ny
    fp = np.concatenate(grayscott_rhs(u0 + eps * d[:n], v0 + eps * d[n:], nx, ny, dx, Du, Dv, F, k))
    fm = np.concatenate(grayscott_rhs(u0 - eps * d[:n], v0 - eps * d[n:], nx, ny, dx, Du, Dv, F, k))
    fd = (fp - fm) / (2 * eps)
    return np.abs(J @ d - fd).max() / np.abs(fd).max()


# --- correction matrices ------------------------------------------------------

def pin_t3_worked_example():
    with open(os.path.join(GOLDEN, "t3_worked_example.json")) as f:
        g = json.load(f)
    V = unit_vectors(40, 3, 0.3, 11)
    a = V.T @ V
    env = dict(a21=a[1, 0], a31=a[2, 0], a32=a[2, 1])
    err = 0.0
    for key, cls in [("cwy", OA.CWY), ("ncwy", OA.NCWY)]:
        ref = np.array([[eval(e, {}, env) for e in row] for row in g[key]], dtype=float)
        obj, _ = drive_correction(cls, V)
        err = max(err, np.abs(obj.T[:3, :3] - ref).max())
    return err


def pin_cwy_projector_identity():
    """Eq. 20: (I - v_j v_j^T) ... (I - v_1 v_1^T) = I - V_j T_j V_j^T with T_j
    from the recursion Eq. 21, for non-orthogonal unit vectors."""
    err = 0.0
    for j in (2, 5, 9):
        V = unit_vectors(30, j, 0.4, 20 + j)
        P = np.eye(30)
        for i in range(j):
            P = (np.eye(30) - np.outer(V[:, i], V[:, i])) @ P
        obj, _ = drive_correction(OA.CWY, V)
        err = max(err, np.abs(P - (np.eye(30) - V @ obj.T[:j, :j] @ V.T)).max())
    return err


def pin_gsmgs_two_sweeps():
    """Sect. 3.2.3: T_j b equals two Gauss-Seidel sweeps on V^T V x = b from
    x^0 = 0 (sweeps written element by element here)."""
    err = 0.0
    for j in (2, 4, 8):
        V = unit_vectors(50, j, 0.3, 40 + j)
        G = V.T @ V
        b = np.random.default_rng(j).standard_normal(j)
        x = np.zeros(j)
        for _ in range(2):
            xn = np.zeros(j)
            for i in range(j):
                s = b[i] - sum(G[i, l] * xn[l] for l in range(i)) \
                         - sum(G[i, l] * x[l] for l in range(i + 1, j))
                xn[i] = s / G[i, i]
            x = xn
        _, out = drive_correction(OA.GSMGS, V, b)
        err = max(err, np.abs(out - x).max())
    return err


def pin_norm_estimate_orthonormal():
    """Eq. 18 is exact for an orthonormal basis (Pythagoras)."""
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 9)))
    w = rng.standard_normal(60)
    est = math.sqrt(w @ w - np.sum((Q.T @ w) ** 2))
    return abs(est - np.linalg.norm(w - Q @ (Q.T @ w)))


# --- Arnoldi ----------------------------------------------------------------------

def small_problem(seed=0):
    cfg = W.advdiff2d(12, ny=10, diff=0.01, vel=(1.0, 0.5))
    cfg["seed"] = W.SEED_BASE + 100 + seed
    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    return cfg, inp, A


def pin_mgs_vs_qr():
    """The Arnoldi basis with positive subdiagonal is the Q factor (positive
    diagonal R) of the Krylov matrix [b, Ab, ..., A^{m-1} b]."""
    cfg, inp, A = small_problem()
    A = A / 50.0
    b = inp["v"]
    m = 6
    K = np.zeros((b.size, m))
    K[:, 0] = b
    for i in range(1, m):
        K[:, i] = A @ K[:, i - 1]
    Q, R = np.linalg.qr(K)
    Q = Q * np.sign(np.diag(R))
    res = OA.mgs(lambda x: A @ x, b, m)
    return np.abs(res["V"][:, :m] - Q).max()


def pin_variants_equal_mgs(variants=("cgs2", "hcwy", "hncwy", "hgsmgs")):
    cfg, inp, A = small_problem()
    ref = OA.mgs(lambda x: A @ x, inp["v"], 25)
    err = 0.0
    for var in variants:
        res = OA.arnoldi(lambda x: A @ x, inp["v"], 25, var)
        err = max(err, np.abs(res["H"] - ref["H"]).max() / np.abs(ref["H"]).max(),
                  np.abs(res["V"] - ref["V"]).max(), abs(res["beta"] - ref["beta"]) / ref["beta"])
    return err


def pin_arnoldi_relation(variant):
    cfg, inp, A = small_problem()
    res = OA.arnoldi(lambda x: A @ x, inp["v"], 25, variant)
    V, H = res["V"], res["H"]
    m = H.shape[1]
    R = A @ V[:, :m] - V @ H
    return np.linalg.norm(R) / (scipy.sparse.linalg.norm(A) * np.linalg.norm(V))


def prescribed_columns(N=200, n=31, kappa=1e7, seed=5):
    """X = U diag(1 .. 1/kappa) W^T (N x n, 2-norm condition number kappa) and
    a "matvec" that returns X's next column at each call, ignoring its input:
    driven by it, every Arnoldi variant becomes a Gram-Schmidt QR of X, where
    the textbook bounds on the loss of orthogonality apply."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((N, n)))
    W_, _ = np.linalg.qr(rng.standard_normal((n, n)))
    X = U @ np.diag(np.logspace(0, -np.log10(kappa), n)) @ W_.T
    calls = [0]

    def next_column(_v):
        calls[0] += 1
        return X[:, calls[0]].copy()
    return X, next_column, calls


def orthogonality_loss(variant, kappa):
    """||I - V^T V||_2 of the basis a variant computes from X (the QR reading
    above) and the column count driven; the start vector is X's first column."""
    X, f, calls = prescribed_columns(kappa=kappa)
    m = X.shape[1] - 1
    res = OA.arnoldi(f, X[:, 0], m, variant)
    V = res["V"]
    assert calls[0] == m and res["m_eff"] == m
    return np.linalg.norm(np.eye(V.shape[1]) - V.T @ V, 2)


def pin_orthogonality_laws(kappas=(1e4, 1e7)):
    """The loss of orthogonality against its textbook laws, as a ratio that
    is <= 1 when every law holds: modified Gram-Schmidt loses at most
    c eps kappa(X) (Bjorck 1967), and the hybrid corrections, which the paper
    says are as accurate as MGS, are held to the same law; classical
    Gram-Schmidt applied twice keeps O(eps) whatever kappa(X) is ("twice is
    enough": Giraud, Langou and Rozloznik 2005), held to 10 n eps here.
    Classical Gram-Schmidt once, which a dropped or wrong correction turns the
    hybrid step into, loses eps kappa^2 and fails the MGS law."""
    eps = np.finfo(float).eps
    n = 31
    worst = 0.0
    for kappa in kappas:
        for var in ("mgs", "hcwy", "hncwy", "hgsmgs"):
            worst = max(worst, orthogonality_loss(var, kappa) / (2.0 * eps * kappa))
        worst = max(worst, orthogonality_loss("cgs2", kappa) / (10.0 * n * eps))
    return worst


# --- phi products -------------------------------------------------------------------

def pin_krylov_vs_dense(variant="mgs"):
    cfg = W.advdiff2d(6, ny=5, diff=0.02, vel=(1.0, -0.7))
    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    ref = OE.phi_products_dense(A, inp["v"], 0.05, 3, expm=scipy.linalg.expm)
    y, _ = OK.phiv(lambda x: A @ x, inp["v"], 0.05, 3, 24, variant)
    return max(np.linalg.norm(y[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(4))


def pin_krylov_grayscott_vs_dense(variant="hcwy"):
    cfg = W.grayscott2d(12, Du=2e-3, Dv=1e-3)
    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    ref = OE.phi_products_dense(A, inp["v"], 1.0, 2, expm=scipy.linalg.expm)
    y, _ = OK.phiv(lambda x: A @ x, inp["v"], 1.0, 2, 40, variant)
    return max(np.linalg.norm(y[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(3))


def pin_krylov_vs_fft_config1(variant="mgs"):
    cfg = W.config(0)
    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    ref = OE.phi_products_fft_advdiff2d(cfg, inp["v"], cfg["h"], cfg["p"])
    y, _ = OK.phiv(lambda x: A @ x, inp["v"], cfg["h"], cfg["p"], cfg["m"], variant)
    return max(np.linalg.norm(y[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(cfg["p"] + 1))


def pin_krylov_vs_fft_adr(variant="hgsmgs"):
    cfg = W.adr3d(16, m=40)
    inp = W.make_inputs(cfg)
    r = np.full(16**3, -0.5)
    A = OP.adr3d(16, 16, 16, cfg["dx"], cfg["diff"], cfg["vel"], r)
    h = 0.02
    ref = OE.phi_products_fft_adr3d(cfg, inp["v"], h, 1, -0.5)
    y, _ = OK.phiv(lambda x: A @ x, inp["v"], h, 1, 40, variant)
    return max(np.linalg.norm(y[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(2))


def pin_diagonal_breakdown(variant):
    """Diagonal A with 3 distinct eigenvalues: the Krylov space is 3-dimensional,
    Arnoldi breaks down at step 3 and the product is exact."""
    rng = np.random.default_rng(9)
    lam = rng.choice([-3.0, -0.5, 1.2], size=200)
    v = rng.uniform(-1, 1, 200)
    y, info = OK.phiv(lambda x: lam * x, v, 0.7, 2, 10, variant)
    ref = OE.phi_products_diagonal(lam, v, 0.7, 2)
    err = max(np.linalg.norm(y[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(3))
    return err + abs(info["m_eff"] - 3)


def pin_zero_operator(variant):
    v = np.random.default_rng(2).uniform(-1, 1, 50)
    y, info = OK.phiv(lambda x: 0.0 * x, v, 0.3, 3, 8, variant)
    err = max(np.abs(y[k] - v / math.factorial(k)).max() for k in range(4))
    return err + abs(info["m_eff"] - 1)


def pin_h_zero(variant):
    cfg, inp, A = small_problem()
    y, _ = OK.phiv(lambda x: A @ x, inp["v"], 0.0, 3, 10, variant)
    return max(np.abs(y[k] - inp["v"] / math.factorial(k)).max() for k in range(4))


def pin_sync_counts():
    """Sect. 2.3 and Alg. 4 sync counts (tests/golden/sync_counts.json)."""
    cfg, inp, A = small_problem()
    mv = lambda x: A @ x
    m = 12
    bad = 0
    r = OA.mgs(mv, inp["v"], m)
    bad += sum(s != j + 1 for j, s in enumerate(r["syncs"], start=1))
    r = OA.cgs2(mv, inp["v"], m)
    bad += sum(s != 3 for s in r["syncs"])
    for var in ("hcwy", "hncwy", "hgsmgs"):
        r = OA.arnoldi(mv, inp["v"], m, var)
        bad += _hybrid_sync_mismatch(r, m)
    # a case that takes the explicit-norm fallback: the per-step counts must
    # still add up (one step charged 2, not 1) -- and the case must fall back
    op, b, mf = fallback_problem()
    for var in ("hcwy", "hncwy"):
        r = OA.arnoldi(op, b, mf, var)
        bad += _hybrid_sync_mismatch(r, mf) + (r["fallbacks"] < 1)
    return float(bad)


def _hybrid_sync_mismatch(r, m):
    """Alg. 4's count: one reduction at every step, one more at each step that
    took the explicit-norm fallback, one more for the final norm when the
    process ran all m steps.  Returns the number of mismatches (0 is good)."""
    syncs, f = r["syncs"], r["fallbacks"]
    full = r["m_eff"] == m and len(syncs) == m
    expect = [1 + (1 if (full and j == len(syncs)) else 0) for j in range(1, len(syncs) + 1)]
    extra = [s - e for s, e in zip(syncs, expect)]
    return sum(x not in (0, 1) for x in extra) + (sum(extra) != f)


def fallback_problem(n=12, seed=6):
    """A diagonal operator with three eigenvalue clusters of width 1e-11: the
    Krylov space is nearly exhausted after three steps and the Pythagorean
    radicand of Eq. 18 goes negative (Alg. 4's explicit-norm fallback)."""
    rng = np.random.default_rng(seed)
    lam = rng.choice([-1.0, -0.5, 0.0], n ** 3) + 1e-11 * rng.standard_normal(n ** 3)
    b = rng.uniform(-1, 1, n ** 3)
    return (lambda x: lam * x), b, 10


# --- adjoint (gradients of 1/2 ||phi_1(hA(theta))v - y_t||^2) ----------------

def _adjoint_case(n=4, Du=0.05, Dv=0.03, h=0.7, seed=7):
    cfg = W.grayscott2d(n, Du=Du, Dv=Dv, h=h, p=1, m=2 * 2 * n * n, seed=seed)
    inp = W.adjoint_inputs(cfg)
    A, dA = OAD.grayscott_parts(cfg, inp)
    return cfg, inp, A, dA


def pin_adjoint_vs_dense():
    """Krylov gradients (m = full dimension) against dense exponentials and
    scipy's Frechet derivative of exp on the Eq. 7 matrix (tiny grid)."""
    cfg, inp, A, dA = _adjoint_case()
    gk = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], cfg["h"], cfg["m"])
    gd = OAD.grads_dense(A, dA, inp["v"], inp["y_target"], cfg["h"])
    rel = lambda a, b: float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))
    return max(abs(gk["L"] - gd["L"]) / gd["L"], rel(gk["dv"], gd["dv"]), abs(gk["dh"] - gd["dh"]) / abs(gd["dh"]),
               rel(gk["dtheta"], gd["dtheta"]))


def pin_adjoint_dF_closed_form():
    """The closed form dL/dF = -h r.(phi_1 v - phi_2 v) against scipy's Frechet
    derivative of exp along dA/dF (tiny grid, no Krylov truncation: m = the
    full dimension) and against the Krylov block-operator product at the
    adjoint test size (m = 40 on 32 x 32)."""
    cfg, inp, A, dA = _adjoint_case()
    gd = OAD.grads_dense(A, dA, inp["v"], inp["y_target"], cfg["h"])
    r = gd["r"]
    e1 = abs(OAD.dF_closed_form(A, inp["v"], r, cfg["h"], cfg["m"]) - gd["dtheta"][2]) / abs(gd["dtheta"][2])
    cfg2 = W.grayscott2d(32, Du=2e-3, Dv=1e-3, h=0.5, p=1, m=40, seed=101)
    inp2 = W.adjoint_inputs(cfg2)
    A2, dA2 = OAD.grayscott_parts(cfg2, inp2)
    gf = OAD.grads_krylov(A2, dA2, inp2["v"], inp2["y_target"], cfg2["h"], 40)
    gc = OAD.grads_krylov(A2, dA2, inp2["v"], inp2["y_target"], cfg2["h"], 40, f_closed=True)
    e2 = abs(gc["dtheta"][2] - gf["dtheta"][2]) / abs(gf["dtheta"][2])
    return max(e1, e2)


def pin_adjoint_finite_differences(n=8, eps=1e-6, m=60):
    """Krylov gradients against central differences of the loss (step eps) in
    v (a random direction), h and each theta_k."""
    cfg, inp, A, dA = _adjoint_case(n=n, seed=11)
    v, yt, h = inp["v"], inp["y_target"], cfg["h"]
    g = OAD.grads_krylov(A, dA, v, yt, h, m)
    th = np.array([cfg["diff"], cfg["diff2"], cfg["F"], cfg["k"]])

    def L_at(theta=th, vv=v, hh=h):
        At, _ = OAD.grayscott_parts(cfg, inp, theta)
        return OAD.loss(At, vv, yt, hh, m)[0]

    d = np.random.default_rng(3).standard_normal(v.size)
    d /= np.linalg.norm(d)
    errs = [abs((L_at(vv=v + eps * d) - L_at(vv=v - eps * d)) / (2 * eps) - g["dv"] @ d) / np.linalg.norm(g["dv"]),
            abs((L_at(hh=h + eps) - L_at(hh=h - eps)) / (2 * eps) - g["dh"]) / abs(g["dh"])]
    for k in range(4):
        e = np.zeros(4)
        e[k] = eps
        fd = (L_at(theta=th + e) - L_at(theta=th - e)) / (2 * eps)
        errs.append(abs(fd - g["dtheta"][k]) / max(abs(g["dtheta"][k]), 1e-12))
    return max(errs)


# --- incomplete orthogonalisation (ioCGS) -----------------------------------

def pin_iocgs_symmetric_is_lanczos():
    """For a symmetric operator the two-vector incomplete process is Lanczos,
    which spans the same Krylov space with the same (tridiagonal) H as full
    orthogonalisation: ioCGS must match MGS (small m, little loss of
    orthogonality)."""
    cfg = W.advdiff2d(24, ny=20, vel=(0.0, 0.0), diff=0.02, m=12)
    A = OP.from_workload(cfg, {})
    b = np.random.default_rng(4).uniform(-1, 1, A.shape[0])
    r_io = OA.iocgs(lambda x: A @ x, b, cfg["m"])
    r_mg = OA.mgs(lambda x: A @ x, b, cfg["m"])
    return max(float(np.abs(r_io["H"] - r_mg["H"]).max() / np.abs(r_mg["H"]).max()),
               float(np.abs(r_io["V"] - r_mg["V"]).max()))


def pin_iocgs_defining_properties():
    """On a non-symmetric operator: unit basis vectors, each new vector
    orthogonal to the two it was orthogonalised against, the banded relation
    A v_j = sum_{i=j-1}^{j+1} H_ij v_i, and H zero outside that band."""
    cfg = W.advdiff2d(20, ny=18, m=15)
    A = OP.from_workload(cfg, {})
    b = np.random.default_rng(8).uniform(-1, 1, A.shape[0])
    r = OA.iocgs(lambda x: A @ x, b, cfg["m"])
    V, H, m = r["V"], r["H"], r["m_eff"]
    err = float(np.abs(np.linalg.norm(V, axis=0) - 1).max())
    for j in range(1, m + 1):
        for i in range(max(1, j - 1), j + 1):
            err = max(err, abs(float(V[:, j] @ V[:, i - 1])))
        band = slice(max(0, j - 2), j + 1)
        err = max(err, float(np.linalg.norm(A @ V[:, j - 1] - V[:, band] @ H[band, j - 1]))
                  / float(np.linalg.norm(A @ V[:, j - 1])))
        mask = np.ones(m + 1, bool)
        mask[band] = False
        err = max(err, float(np.abs(H[mask, j - 1]).max(initial=0.0)))
    # it is not full orthogonalisation: distant vectors do lose orthogonality
    return err


# ---------------------------------------------------------------------------
# Linear combinations sum_j tau^j phi_j(tau A) b_j (Sect. 2.1, Eqs. 7-9) with
# sub-stepping (Sect. 2.2).

def _lincomb_case(p, seed, n=6):
    cfg = W.advdiff2d(n, ny=n, diff=0.05, vel=(1.0, 0.5), m=20)
    A = OP.from_workload(cfg, {}).toarray()
    rng = np.random.default_rng(seed)
    bs = [rng.uniform(-1, 1, A.shape[0]) for _ in range(p + 1)]
    return A, bs


def pin_lincomb_diagonal(p=3, tau=0.7):
    """A = diag(lam): the combination is sum_j tau^j phi_j(tau lam_i) b_j,i
    entry by entry (scalar phi_k pinned separately); Krylov with m = N + p
    spans the whole augmented space, in one and in three sub-steps."""
    lam = np.array([-3.0, -1.2, -0.4, 0.0, 0.3, 1.1])
    rng = np.random.default_rng(21)
    bs = [rng.uniform(-1, 1, lam.size) for _ in range(p + 1)]
    ref = sum(tau ** j * OPHI.phi(j, tau * lam) * bs[j] for j in range(p + 1))
    err = 0.0
    for nsub in (1, 3):
        u, _ = OL.lincomb_krylov(lambda x: lam * x, bs, tau, lam.size + p, nsub)
        err = max(err, float(np.abs(u - ref).max() / np.abs(ref).max()))
    return err


def pin_lincomb_solves_forced_ode(p=3, tau=0.4, eps=1e-3):
    """u(t) = sum_j t^j phi_j(tA) b_j solves u' = A u + sum_{j>=1} t^{j-1}/(j-1)! b_j
    with u(0) = b_0: a fourth-order central difference in t of the Krylov
    result against the right-hand side (this fixes where tau enters Eq. 8)."""
    A, bs = _lincomb_case(p, 22)
    m = A.shape[0] + p
    u = lambda t: OL.lincomb_krylov(lambda x: A @ x, bs, t, m, 1)[0]
    du = (8 * (u(tau + eps) - u(tau - eps)) - (u(tau + 2 * eps) - u(tau - 2 * eps))) / (12 * eps)
    g = sum(tau ** (j - 1) / math.factorial(j - 1) * bs[j] for j in range(1, p + 1))
    rhs = A @ u(tau) + g
    e0 = float(np.abs(u(0.0) - bs[0]).max())
    return max(float(np.abs(du - rhs).max() / np.abs(rhs).max()), e0)


def pin_lincomb_substeps_vs_dense(p=2, tau=1.3):
    """Dense exponential of the augmented matrix (Eq. 7) against Krylov in 1,
    2 and 5 equal sub-steps on a non-symmetric operator."""
    A, bs = _lincomb_case(p, 23)
    ref = OE.phi_combination_dense(A, bs, tau, expm=scipy.linalg.expm)
    err = 0.0
    for nsub in (1, 2, 5):
        u, _ = OL.lincomb_krylov(lambda x: A @ x, bs, tau, A.shape[0] + p, nsub)
        err = max(err, float(np.abs(u - ref).max() / np.abs(ref).max()))
    return err


def pin_lincomb_single_vector(p=3, tau=0.9):
    """Only b_k nonzero: the combination is tau^k phi_k(tau A) b_k, the k-th
    phi product of the plain path; p = 0 is exp(tau A) b_0 (scipy)."""
    A, bs = _lincomb_case(p, 24)
    N = A.shape[0]
    y, _ = OK.phiv(lambda x: A @ x, bs[p], tau, p, N)
    zs = [np.zeros(N)] * p + [bs[p]]
    u, _ = OL.lincomb_krylov(lambda x: A @ x, zs, tau, N + p, 2)
    err = float(np.abs(u - tau ** p * y[p]).max() / np.abs(tau ** p * y[p]).max())
    u0, _ = OL.lincomb_krylov(lambda x: A @ x, [bs[0]], tau, N, 1)
    ref0 = scipy.linalg.expm(tau * A) @ bs[0]
    return max(err, float(np.abs(u0 - ref0).max() / np.abs(ref0).max()))


# ---------------------------------------------------------------------------
# Exponential integrators of Sect. 4 (SRERK3, EPI4, EPI5).

def pin_integrators_linear_exact(h=0.1, nsteps=6):
    """u' = A u: the remainder R vanishes and every method steps exactly with
    exp(hA), so nsteps steps equal exp(nsteps h A) u_0 (scipy)."""
    cfg = W.advdiff2d(6, diff=0.05, vel=(1.0, 0.5))
    A = OP.from_workload(cfg, {}).toarray()
    u0 = np.random.default_rng(31).uniform(-1, 1, A.shape[0])
    F, Jf = OI.linear_problem(A)
    ref = scipy.linalg.expm(nsteps * h * A) @ u0
    err = 0.0
    for meth in ("srerk3", "epi4", "epi5"):
        u = OI.integrate(meth, F, Jf, u0, h, nsteps, OI.dense_lincomb)
        err = max(err, float(np.abs(u - ref).max() / np.abs(ref).max()))
    return err


_ORDER_CACHE = {}


def integrator_orders(T=1.0, steps=(8, 16, 32)):
    """Observed convergence orders on a 6 x 6 Gray-Scott system (Radau
    reference at rtol 1e-13); the multistep methods start from reference
    values, so the order is the method's own.  Returns {method: order of the
    last halving}."""
    import scipy.integrate as si

    key = (T, steps)
    if key in _ORDER_CACHE:
        return _ORDER_CACHE[key]
    cfg = W.grayscott2d(6, Du=2e-2, Dv=1e-2)
    inp = W.make_inputs(cfg)
    u0 = np.concatenate([inp["u0"], inp["v0"]])
    F, Jf = OI.grayscott_problem(cfg)
    ref = si.solve_ivp(lambda t, y: F(y), (0, T), u0, method="Radau", rtol=1e-13, atol=1e-13,
                       jac=lambda t, y: Jf(y).toarray(), dense_output=True)
    uT = ref.y[:, -1]
    out = {}
    for meth in ("srerk3", "epi4", "epi5"):
        errs = []
        for nst in steps:
            h = T / nst
            if meth == "srerk3":
                u = OI.integrate(meth, F, Jf, u0, h, nst, OI.dense_lincomb)
            else:
                P = OI.EPI_ALPHA[int(meth[3:])].shape[1]
                hist = [ref.sol(i * h) for i in range(P, -1, -1)]
                u = OI.integrate(meth, F, Jf, hist[0], h, nst - P, OI.dense_lincomb, history=hist[1:])
            errs.append(float(np.abs(u - uT).max()))
        out[meth] = math.log2(errs[-2] / errs[-1])
    _ORDER_CACHE.clear()
    _ORDER_CACHE[key] = out
    return out


def pin_lincomb_adaptive(tol=1e-10, tau=2.0, m=12):
    """Adaptive sub-steps on a stiff non-symmetric operator where one m-step
    projection is far from the tolerance: the result is within a small multiple
    of tol of the dense augmented exponential, it took more than one sub-step,
    and every accepted sub-step met the tolerance.  Returns (error relative to
    tol, number of sub-steps, converged)."""
    cfg = W.advdiff2d(12, diff=0.05, vel=(1.0, 0.5))
    A = OP.from_workload(cfg, {}).toarray()
    rng = np.random.default_rng(25)
    bs = [rng.uniform(-1, 1, A.shape[0]) for _ in range(3)]
    ref = OE.phi_combination_dense(A, bs, tau, expm=scipy.linalg.expm)
    u, info = OL.lincomb_adaptive(lambda x: A @ x, bs, tau, m, tol)
    err = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    return err / tol, len(info["sizes"]), info["converged"]


def pin_lincomb_adaptive_m(tol=1e-10, tau=2.0):
    """Sub-steps with adaptive size and Krylov dimension (this build's rule) on
    the stiff operator of ``pin_lincomb_adaptive``: started with a dimension far
    too small (m0 = 4) the rule must raise it, started far too large (m0 = 40)
    it must lower it; both results are within a small multiple of tol of the
    dense augmented exponential and every accepted sub-step met the tolerance.
    Returns a dict per start: error relative to tol, first/largest/last
    dimension, sub-steps, converged, modeled cost against the fixed-m run."""
    cfg = W.advdiff2d(12, diff=0.05, vel=(1.0, 0.5))
    A = OP.from_workload(cfg, {}).toarray()
    rng = np.random.default_rng(25)
    bs = [rng.uniform(-1, 1, A.shape[0]) for _ in range(3)]
    ref = OE.phi_combination_dense(A, bs, tau, expm=scipy.linalg.expm)
    out = {}
    for m0 in (4, 40):
        u, info = OL.lincomb_adaptive_m(lambda x: A @ x, bs, tau, m0, tol)
        _, fixed = OL.lincomb_adaptive(lambda x: A @ x, bs, tau, m0, tol)
        cost = sum(OL.projection_cost(d) for d in info["dims"])
        cost_fixed = len(fixed["sizes"]) * OL.projection_cost(m0)
        out[m0] = dict(err=float(np.linalg.norm(u - ref) / np.linalg.norm(ref)) / tol,
                       first=info["dims"][0], largest=max(info["dims"]), last=info["dims"][-1],
                       substeps=len(info["sizes"]), converged=info["converged"],
                       cost_ratio=cost / cost_fixed)
    return out
