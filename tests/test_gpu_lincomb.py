"""phi-function linear combinations u = sum_j tau^j phi_j(tau A) b_j through the
CUDA path (lsa_phiv_lincomb: Krylov projection of the augmented operator of
Eqs. 7-9 in equal sub-steps) against the oracle's projection with the same m
and sub-steps, dense exponentials of the augmented matrix, and the plain phi
products."""
import numpy as np
import pytest

import workloads as W
from oracle import exact as OE
from oracle import lincomb as OL
from oracle import operators as OP
from tests.gpu_util import FP64_TOL, expected_syncs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def case(name, m=30):
    if name == "advdiff2d":
        return W.advdiff2d(48, ny=40, m=m, h=0.5, diff=0.01)        # ragged tiles in y
    if name == "grayscott2d":
        cfg = W.grayscott2d(32, Du=2e-3, Dv=1e-3, h=0.5, m=m, seed=105)
        cfg.update(ny=24, name="grayscott2d_32x24")
        return cfg
    cfg = W.adr3d(20, m=m, h=5e-3)
    cfg.update(ny=16, nz=12, name="adr3d_20x16x12")                    # ragged 3D tiles
    return cfg


def setup(cfg, p):
    import paper_2410_14917_gb300 as lsa

    inp = W.lincomb_inputs(cfg, p)
    fields = {k: torch.from_numpy(v).cuda() for k, v in inp.items() if k not in ("v", "b")}
    op = lsa.Operator.from_workload(cfg, fields)
    A = OP.from_workload(cfg, inp)
    return lsa, op, A, inp["b"], torch.from_numpy(inp["b"]).cuda().contiguous()


def rel(a, b):
    """The larger of the normwise and the element-wise (max-abs over max-abs) error."""
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = np.asarray(b)
    return float(max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b))))


@pytest.mark.parametrize("name", ["advdiff2d", "grayscott2d", "adr3d"])
@pytest.mark.parametrize("variant", ["hcwy", "mgs"])
@pytest.mark.parametrize("nsub", [1, 3])
def test_lincomb_matches_oracle(name, variant, nsub):
    p, tau = 3, 0.5 if name != "adr3d" else 5e-3
    cfg = case(name)
    lsa, op, A, b, bd = setup(cfg, p)
    ref, infos = OL.lincomb_krylov(lambda x: A @ x, list(b), tau, cfg["m"], nsub, "mgs")
    u, st = lsa.phiv_lincomb(op, bd, tau, cfg["m"], nsub, variant=variant)
    assert st["status"] >= 0
    assert rel(u, ref) < FP64_TOL
    m_eff = min(i["m_eff"] for i in infos)
    assert st["m_eff"] == m_eff
    assert st["grid_syncs"] == nsub * expected_syncs(variant, m_eff, 0) + (st["norm_fallbacks"] if variant != "mgs" else 0)


@pytest.mark.parametrize("variant", ["hncwy", "hgsmgs", "cgs2", "iocgs"])
def test_lincomb_other_variants(variant):
    p, tau = 2, 0.5
    cfg = case("grayscott2d")
    lsa, op, A, b, bd = setup(cfg, p)
    ref, _ = OL.lincomb_krylov(lambda x: A @ x, list(b), tau, cfg["m"], 2,
                               "iocgs" if variant == "iocgs" else "mgs")
    u, st = lsa.phiv_lincomb(op, bd, tau, cfg["m"], 2, variant=variant)
    assert rel(u, ref) < FP64_TOL


def test_lincomb_matches_dense_augmented_exponential():
    p, tau = 2, 1.3
    cfg = W.advdiff2d(16, m=48, diff=0.01)
    lsa, op, A, b, bd = setup(cfg, p)
    ref = OE.phi_combination_dense(A.toarray(), list(b), tau, expm=OE.scipy_expm)
    u, st = lsa.phiv_lincomb(op, bd, tau, 48, 2, variant="hcwy")
    assert rel(u, ref) < FP64_TOL


def test_lincomb_single_vector_is_the_phi_product():
    p, tau = 3, 0.5
    cfg = case("grayscott2d")
    lsa, op, A, b, bd = setup(cfg, p)
    z = torch.zeros_like(bd)
    z[p] = bd[p]
    u, _ = lsa.phiv_lincomb(op, z.contiguous(), tau, cfg["m"], 1, variant="hcwy")
    y, _ = lsa.phiv(op, bd[p].contiguous(), tau, p, cfg["m"], variant="hcwy")
    yp = (tau ** p) * y[p]
    assert rel(u, yp.cpu().numpy()) < 1e-11


def test_lincomb_p0_is_phiv_bit_for_bit():
    cfg = case("advdiff2d")
    lsa, op, A, b, bd = setup(cfg, 0)
    u, _ = lsa.phiv_lincomb(op, bd, 0.5, cfg["m"], 1, variant="hcwy")
    y, _ = lsa.phiv(op, bd[0].contiguous(), 0.5, 0, cfg["m"], variant="hcwy")
    assert torch.equal(u, y[0])


def test_lincomb_tau_zero_returns_b0():
    cfg = case("advdiff2d")
    lsa, op, A, b, bd = setup(cfg, 2)
    u, _ = lsa.phiv_lincomb(op, bd, 0.0, cfg["m"], 2, variant="hcwy")
    assert rel(u, b[0]) < 1e-14


def test_lincomb_in_place_on_b0():
    p, tau = 2, 0.5
    cfg = case("grayscott2d")
    lsa, op, A, b, bd = setup(cfg, p)
    ref, _ = OL.lincomb_krylov(lambda x: A @ x, list(b), tau, cfg["m"], 2, "mgs")
    u, _ = lsa.phiv_lincomb(op, bd, tau, cfg["m"], 2, variant="hcwy", u=bd[0])
    assert rel(bd[0], ref) < FP64_TOL


def test_lincomb_rejects_bad_arguments():
    import paper_2410_14917_gb300 as lsa
    from paper_2410_14917_gb300 import _binding as B

    cfg = case("advdiff2d")
    _, op, _, _, bd = setup(cfg, 1)
    u = torch.empty(bd.shape[1], dtype=torch.float64, device="cuda")
    work = lsa.Workspace.for_call(op, 30, 0, "fp64")
    lib = B.lib()
    import ctypes
    args = lambda nsub, prec: (ctypes.byref(op.c), ctypes.c_void_p(bd.data_ptr()), 1, 0.5, nsub, 30, 0.0,
                               B.VARIANTS["hcwy"], prec, ctypes.c_void_p(u.data_ptr()),
                               ctypes.c_void_p(work.ptr), work.nbytes, None, None)
    assert lib.lsa_phiv_lincomb(*args(0, B.PRECISIONS["fp64"])) == B.LSA_ERR_ARG
    assert lib.lsa_phiv_lincomb(*args(1, B.PRECISIONS["fp32"])) == B.LSA_ERR_ARG


def test_lincomb_zero_operator_closed_form():
    # A = 0: sum_j tau^j phi_j(0) b_j = sum_j tau^j / j! b_j; the Krylov process breaks
    # down inside the augmented space (dimension p + 1), exactly
    import math

    p, tau = 8, 0.7
    cfg = W.advdiff2d(32, diff=0.0, vel=(0.0, 0.0), m=64)
    lsa, op, A, b, bd = setup(cfg, p)
    ref = sum(tau ** j / math.factorial(j) * b[j] for j in range(p + 1))
    for variant in ("hcwy", "mgs"):
        u, st = lsa.phiv_lincomb(op, bd, tau, 64, 3, variant=variant)
        assert rel(u, ref) < 1e-13
        assert st["breakdown"] == 1 and st["m_eff"] <= p + 1


def test_lincomb_largest_p_and_m():
    p, tau = 8, 0.5
    cfg = case("grayscott2d", m=64)
    lsa, op, A, b, bd = setup(cfg, p)
    ref, _ = OL.lincomb_krylov(lambda x: A @ x, list(b), tau, 64, 1, "mgs")
    u, st = lsa.phiv_lincomb(op, bd, tau, 64, 1, variant="hcwy")
    assert rel(u, ref) < FP64_TOL


@pytest.mark.parametrize("variant", ["hcwy", "mgs"])
def test_lincomb_adaptive_matches_oracle(variant):
    p, tau, m, tol = 3, 2.0, 16, 1e-10
    cfg = case("grayscott2d")
    lsa, op, A, b, bd = setup(cfg, p)
    ref, info = OL.lincomb_adaptive(lambda x: A @ x, list(b), tau, m, tol)
    u, st = lsa.phiv_lincomb_adaptive(op, bd, tau, m, tol, variant=variant)
    assert st["status"] == 0 and info["converged"]
    assert abs(st["substeps"] - len(info["sizes"])) <= 1 and st["substeps"] > 1
    assert rel(u, ref) < 20 * tol


def test_lincomb_adaptive_against_dense_and_in_place():
    p, tau, m, tol = 2, 1.5, 12, 1e-9
    cfg = W.advdiff2d(16, m=m, diff=0.02)
    lsa, op, A, b, bd = setup(cfg, p)
    dense = OE.phi_combination_dense(A.toarray(), list(b), tau, expm=OE.scipy_expm)
    u, st = lsa.phiv_lincomb_adaptive(op, bd, tau, m, tol, u=bd[0])
    assert st["substeps"] > 1
    assert rel(bd[0], dense) < 20 * tol


def test_lincomb_adaptive_loose_tolerance_is_one_step():
    cfg = case("advdiff2d")
    lsa, op, A, b, bd = setup(cfg, 2)
    u1, st = lsa.phiv_lincomb_adaptive(op, bd, 0.5, cfg["m"], 1.0)
    u0, _ = lsa.phiv_lincomb(op, bd, 0.5, cfg["m"], 1, variant="hcwy")
    assert st["substeps"] == 1 and st["rejected"] == 0
    assert torch.equal(u0, u1)


def test_lincomb_adaptive_reports_the_substep_cap():
    p, tau, m, tol = 3, 2.0, 8, 1e-12
    cfg = case("grayscott2d")
    lsa, op, A, b, bd = setup(cfg, p)
    u, st = lsa.phiv_lincomb_adaptive(op, bd, tau, m, tol, max_substeps=2)
    assert st["status"] == 2          # LSA_NOT_CONVERGED: tau not reached within the cap


@pytest.mark.parametrize("name", ["grayscott2d", "adr3d"])
@pytest.mark.parametrize("m0", [4, 40])
def test_lincomb_adaptive_dimension_matches_oracle(name, m0):
    """Sub-steps with adaptive size and Krylov dimension (this library's rule,
    lsa_phiv_lincomb_adaptive_m) against the oracle running the same rule: the
    result, the first accepted dimension, and the direction the dimension moves
    from a start far too small (raised) or far too large (lowered)."""
    p, tau, tol = 3, 2.0, 1e-10
    cfg = case(name)
    lsa, op, A, b, bd = setup(cfg, p)
    ref, info = OL.lincomb_adaptive_m(lambda x: A @ x, list(b), tau, m0, tol)
    u, st = lsa.phiv_lincomb_adaptive_m(op, bd, tau, m0, tol, variant="hcwy")
    assert st["status"] == 0 and info["converged"]
    assert rel(u, ref) < 20 * tol
    assert st["dims"][0] == info["dims"][0]
    assert len(st["dims"]) == st["substeps"] and abs(st["substeps"] - len(info["sizes"])) <= max(2, len(info["sizes"]) // 5)
    if m0 == 4:
        assert max(st["dims"]) >= 8
    elif st["substeps"] > 1:
        assert min(st["dims"]) <= 20


def test_lincomb_adaptive_dimension_against_dense():
    p, tau, tol = 2, 1.5, 1e-9
    cfg = W.advdiff2d(16, m=12, diff=0.02)
    lsa, op, A, b, bd = setup(cfg, p)
    dense = OE.phi_combination_dense(A.toarray(), list(b), tau, expm=OE.scipy_expm)
    u, st = lsa.phiv_lincomb_adaptive_m(op, bd, tau, 6, tol, m_min=3, m_max=32)
    assert st["status"] == 0
    assert rel(u, dense) < 20 * tol
    assert all(3 <= d <= 32 for d in st["dims"])


def test_lincomb_adaptive_dimension_rejects_bad_arguments():
    import paper_2410_14917_gb300 as lsa
    from paper_2410_14917_gb300 import LsaError

    cfg = case("advdiff2d")
    _, op, A, b, bd = setup(cfg, 1)
    for kw in (dict(m_min=0), dict(m_min=10, m_max=5), dict(m_max=65)):
        with pytest.raises(LsaError):
            lsa.phiv_lincomb_adaptive_m(op, bd, 1.0, 8, 1e-8, **kw)
