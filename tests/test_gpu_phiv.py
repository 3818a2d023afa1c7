"""lsa_phiv parity: the CUDA path against the CPU oracle (O-Krylov, float64
MGS), per phi_k, for every variant and both precisions, on the benchmark
workloads (the 64x64 advection-diffusion case at full size, the others at
sizes the oracle finishes in seconds that still span many tiles and a ragged
tail), plus edge cases."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import exact as OE
from oracle import krylov as OK
from oracle import operators as OP
from tests.gpu_util import FP32_TOL, FP64_TOL, device_inputs, expected_syncs, oracle_phiv, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = ["mgs", "cgs2", "hcwy", "hncwy", "hgsmgs"]
CASES = [W.config(0), W.grayscott2d(72, m=64, p=2, Du=2e-3, Dv=1e-3, h=0.5),
         W.adr3d(40, m=40, p=1), W.advdiff2d(37, ny=29, m=25, p=2)]


def run(cfg, variant, precision, **kw):
    import paper_2410_14917_gb300 as lsa

    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    args = dict(h=cfg["h"], p=cfg["p"], m=cfg["m"])
    args.update(kw)
    y, st = lsa.phiv(op, v, variant=variant, precision=precision, **args)
    return y, st, inp


@pytest.mark.parametrize("cfg", CASES, ids=[c["name"] for c in CASES])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_phiv_parity(cfg, variant, precision):
    y, st, _ = run(cfg, variant, precision)
    ref, info = oracle_phiv(cfg)
    errs = rel_errors(y, ref)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    assert max(errs) < tol, errs
    assert st["status"] in (0, 1)
    assert st["m_eff"] == info["m_eff"]


@pytest.mark.parametrize("variant,precision", [("hcwy", "fp64"), ("mgs", "fp64"), ("cgs2", "fp64"),
                                               ("hcwy", "fp32")])
def test_phiv_grayscott512_full_size_matches_oracle(variant, precision):
    """The Gray-Scott 512^2 workload at full size (N = 524288, m = 64, phi_0..phi_2),
    each of its variants and the float32-basis form, against the oracle's
    float64 MGS product element by element and normwise."""
    cfg = W.config(1)
    y, st, _ = run(cfg, variant, precision)
    ref, info = oracle_phiv(cfg)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    errs = rel_errors(y, ref)
    assert max(errs) < tol, errs
    assert st["status"] == 0 and st["m_eff"] == info["m_eff"] == cfg["m"]
    assert st["grid_syncs"] == expected_syncs(variant, cfg["m"], st["norm_fallbacks"])


def test_phiv_advdiff64_matches_fft_exact():
    cfg = W.config(0)
    y, st, inp = run(cfg, "hcwy", "fp64")
    ref = OE.phi_products_fft_advdiff2d(cfg, inp["v"], cfg["h"], cfg["p"])
    assert max(rel_errors(y, ref)) < FP64_TOL


def test_phiv_h_zero_gives_v_over_factorial():
    cfg = W.advdiff2d(20, ny=12, m=10, p=3)
    y, st, inp = run(cfg, "hgsmgs", "fp64", h=0.0)
    yc = y.cpu().numpy()
    for k in range(4):
        assert np.abs(yc[k] - inp["v"] / math.factorial(k)).max() < 1e-13


@pytest.mark.parametrize("variant", VARIANTS)
def test_phiv_zero_operator_breaks_down_at_step_one(variant):
    cfg = W.advdiff2d(16, diff=0.0, vel=(0.0, 0.0), m=8, p=2)
    y, st, inp = run(cfg, variant, "fp64")
    yc = y.cpu().numpy()
    assert st["m_eff"] == 1 and st["breakdown"] == 1
    for k in range(3):
        assert np.abs(yc[k] - inp["v"] / math.factorial(k)).max() < 1e-14


def test_phiv_zero_vector():
    import paper_2410_14917_gb300 as lsa

    cfg = W.advdiff2d(16, m=8, p=1)
    op = lsa.Operator.from_workload(cfg, {})
    v = torch.zeros(256, dtype=torch.float64, device="cuda")
    y, st = lsa.phiv(op, v, 0.1, 1, 8, variant="hcwy")
    assert torch.count_nonzero(y).item() == 0 and st["m_eff"] == 0


@pytest.mark.parametrize("n,ny", [(1, 1), (3, 5), (2, 2)])
def test_phiv_tiny_grids_cap_m(n, ny):
    cfg = W.advdiff2d(n, ny=ny, m=30, p=2, h=0.01)
    y, st, inp = run(cfg, "hcwy", "fp64")
    A = OP.from_workload(cfg, inp).toarray()
    ref = OE.phi_products_dense(A, inp["v"], cfg["h"], cfg["p"])
    assert max(rel_errors(y, ref)) < 1e-10


def test_phiv_argument_errors():
    import paper_2410_14917_gb300 as lsa
    from paper_2410_14917_gb300 import LsaError

    cfg = W.advdiff2d(16, m=8, p=1)
    op = lsa.Operator.from_workload(cfg, {})
    v = torch.ones(256, dtype=torch.float64, device="cuda")
    with pytest.raises(LsaError):
        lsa.phiv(op, v, float("nan"), 1, 8)
    with pytest.raises(LsaError):
        lsa.phiv(op, v, 0.1, 1, 65)
    small = lsa.Workspace(1024)
    with pytest.raises(LsaError):
        lsa.phiv(op, v, 0.1, 1, 8, work=small)


def test_barrier_timeout_returns_error_and_context_survives():
    import paper_2410_14917_gb300 as lsa

    assert lsa.selftest_barrier_timeout(0.2) == -3          # LSA_ERR_TIMEOUT
    cfg = W.advdiff2d(16, m=8, p=1)
    y, st, inp = run(cfg, "hcwy", "fp64")                  # the context is still usable
    ref, _ = oracle_phiv(cfg)
    assert max(rel_errors(y, ref)) < FP64_TOL


def test_norm_estimate_fallback_path():
    """Diagonal operators (3D ADR with no diffusion or advection) with three
    eigenvalue clusters of width delta: the Krylov space is nearly exhausted
    after three steps, the Pythagorean radicand of Eq. 18 goes negative and
    Alg. 4 falls back to an explicit norm (one extra reduction each time), or
    the process ends in a detected breakdown.  Whether the radicand of a given
    step rounds below zero depends on the summation order, so each variant
    runs on several widths and must take the fallback (or the breakdown it
    leads to) on at least one; every run matches the oracle and its sync count
    includes the fallbacks (after a detected breakdown there is no final
    reduction)."""
    import paper_2410_14917_gb300 as lsa
    from oracle import operators as OPS

    n, m, p, h = 16, 10, 1, 0.5
    degenerate = {"hcwy": 0, "hncwy": 0, "hgsmgs": 0}
    for delta, seed in ((1e-11, 6), (1e-10, 7), (3e-12, 8), (1e-11, 9)):
        rng = np.random.default_rng(seed)
        r = rng.choice([-1.0, -0.5, 0.0], n ** 3) + delta * rng.standard_normal(n ** 3)
        b = rng.uniform(-1, 1, n ** 3)
        A = OPS.adr3d(n, n, n, 1.0 / n, 0.0, (0.0, 0.0, 0.0), r)
        ref, _ = OK.phiv(lambda x: A @ x, b, h, p, m, "mgs")
        op = lsa.Operator.adr3d(n, n, n, 1.0 / n, 0.0, (0.0, 0.0, 0.0), torch.from_numpy(r).cuda())
        for variant in degenerate:
            y, st = lsa.phiv(op, torch.from_numpy(b).cuda(), h, p, m, variant=variant)
            assert max(rel_errors(y, ref)) < FP64_TOL, (variant, delta)
            f = st["norm_fallbacks"]
            if st["breakdown"]:
                # detected at step j: by the estimate (m_eff = j) or lagged (m_eff = j - 1)
                assert st["grid_syncs"] - f in (st["m_eff"], st["m_eff"] + 1)
            else:
                assert st["grid_syncs"] == expected_syncs(variant, st["m_eff"], f)
            degenerate[variant] += f + st["breakdown"]
    for variant, count in degenerate.items():
        assert count >= 1, variant       # each variant met the degenerate case at least once
