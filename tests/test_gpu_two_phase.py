"""The two-phase hybrid step of the grid Arnoldi kernel (Alg. 4 with Algs.
5/6/7: project every value once over equal flat shares, grid barrier, then
stencil and inner products) against the one-pass step, which projects each
tile's halo again.  Both apply the same operations in the same order to every
value, so basis, H and phi products must agree bit for bit; the two-phase form
is also checked against the oracle, on ragged grids (partial tiles and flat
shares), 2D and 3D operators, both precisions and each hybrid correction, and
the step-form tuner's choice is the form later calls report."""
import os

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import FP32_TOL, FP64_TOL, device_inputs, oracle_phiv, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [W.advdiff2d(64, m=30, p=2), W.advdiff2d(40, ny=23, m=24, p=1),
         W.grayscott2d(40, m=32, p=2), W.adr3d(20, m=24, p=1),
         W.advdiff2d(3, ny=5, m=6, p=1)]
VARIANTS = ["hcwy", "hncwy", "hgsmgs"]


class env:
    """Set environment variables for the duration of a block."""

    def __init__(self, **kw):
        self.kw = kw

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kw}
        os.environ.update({k: str(v) for k, v in self.kw.items()})

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _op(cfg):
    import paper_2410_14917_gb300 as lsa

    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    return lsa.Operator.from_workload(cfg, fields), v


def _grid_kernel_env(two):
    # the float32-basis form would otherwise run the TMA or streaming kernels
    return env(LSA_TWO_PHASE=int(two), LSA_TMA=0, LSA_STREAM=0, LSA_CLUSTER=0)


@pytest.mark.parametrize("cfg", CASES, ids=[c["name"] for c in CASES])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_phase_arnoldi_bitwise_equal_to_one_pass(cfg, variant, precision):
    import paper_2410_14917_gb300 as lsa

    op, v = _op(cfg)
    m = min(cfg["m"], op.N)
    out = {}
    for two in (0, 1):
        with _grid_kernel_env(two):
            V, H, st = lsa.arnoldi(op, v, m, variant=variant, precision=precision)
        out[two] = (V.cpu().numpy(), H.cpu().numpy(), st)
    (V0, H0, s0), (V1, H1, s1) = out[0], out[1]
    assert s0["arnoldi_kernel"] == 0 and s1["arnoldi_kernel"] == 4
    assert s0["status"] == s1["status"] == 0 and s0["m_eff"] == s1["m_eff"] == m
    assert np.array_equal(H0, H1)
    assert np.array_equal(V0, V1)
    assert s0["norm_fallbacks"] == s1["norm_fallbacks"]
    for s in (s0, s1):
        assert s["grid_syncs"] == m + 1 + s["norm_fallbacks"]
    # one barrier without a reduction per step, plus one per reduction
    assert s1["grid_barriers"] == s1["grid_syncs"] + m
    assert s0["grid_barriers"] == s0["grid_syncs"]


@pytest.mark.parametrize("cfg", CASES[:4], ids=[c["name"] for c in CASES[:4]])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_phase_phiv_matches_oracle(cfg, precision):
    import paper_2410_14917_gb300 as lsa

    op, v = _op(cfg)
    with _grid_kernel_env(1):
        y1, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy", precision=precision)
    with _grid_kernel_env(0):
        y0, _ = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy", precision=precision)
    assert st["arnoldi_kernel"] == 4
    ref, info = oracle_phiv(cfg, "hcwy")
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    assert torch.equal(y0, y1)
    assert max(rel_errors(y1, ref)) < tol
    assert st["m_eff"] == info["m_eff"]
    assert st["grid_syncs"] == cfg["m"] + 1 + st["norm_fallbacks"]


def test_two_phase_headline_shape_sampled():
    """Gray-Scott 512^2 with m = 64 (the full-size float64 workload): both
    forms agree bit for bit, and the Arnoldi relation holds on sampled
    columns of the two-phase basis."""
    import paper_2410_14917_gb300 as lsa

    cfg = W.config(1)
    op, v = _op(cfg)
    m = cfg["m"]
    res = {}
    for two in (0, 1):
        with _grid_kernel_env(two):
            V, H, st = lsa.arnoldi(op, v, m, variant="hcwy")
        res[two] = (V, H, st)
    assert res[1][2]["arnoldi_kernel"] == 4
    assert torch.equal(res[0][1], res[1][1]) and torch.equal(res[0][0], res[1][0])
    V, H = res[1][0], res[1][1]
    for j in (0, 17, m - 1):
        Av = lsa.matvec(op, V[:, j].contiguous())
        r = Av - V @ H[:, j]
        assert float(r.norm() / Av.norm()) < 1e-11


def test_tune_step_records_choice():
    import paper_2410_14917_gb300 as lsa

    cfg = W.grayscott2d(128, m=24, p=1)
    op, v = _op(cfg)
    os.environ.pop("LSA_TWO_PHASE", None)
    two, ms1, ms2 = lsa.tune_step(op, v, cfg["m"], variant="hcwy", precision="fp64", reps=2)
    assert two in (0, 1, 2) and ms1 > 0 and ms2 > 0
    assert (two != 0) == (ms2 < ms1)
    _, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy")
    assert st["arnoldi_kernel"] == (3 + two if two else 0)
    # the environment overrides the recorded choice
    other = 0 if two else 1
    with env(LSA_TWO_PHASE=other):
        _, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy")
    assert st["arnoldi_kernel"] == (3 + other if other else 0)
    # variants without the hybrid step: nothing to choose
    assert lsa.tune_step(op, v, cfg["m"], variant="mgs") == (0, 0.0, 0.0)


def test_two_phase_3d_large_grid_matches_one_pass_and_oracle():
    """The 3D ADR operator at 128^3 with m = 40 in float64 (the two-phase
    step is the default form on 3D grids): several z-segments per tile column
    and many flat shares per plane; both forms agree bit for bit, and the
    two-phase phi product matches the oracle (its H-CWY form) element by
    element."""
    import paper_2410_14917_gb300 as lsa

    cfg = W.adr3d(128, m=40, p=1)
    op, v = _op(cfg)
    out = {}
    for two in (0, 1):
        with _grid_kernel_env(two):
            out[two] = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy")
    (y0, s0), (y1, s1) = out[0], out[1]
    assert s0["arnoldi_kernel"] == 0 and s1["arnoldi_kernel"] == 4
    assert torch.equal(y0, y1)
    ref, info = oracle_phiv(cfg, "hcwy")
    assert max(rel_errors(y1, ref)) < FP64_TOL
    assert s1["m_eff"] == info["m_eff"] == cfg["m"]


def test_two_phase_adr256_full_size_matches_oracle():
    """The 3D ADR 256^3 workload (N = 16.7M, m = 40) in float64, where the
    two-phase step is the default form: the phi product against the oracle's
    H-CWY form (the same oracle product the streaming float32 test compares
    with; the oracle's pins hold H-CWY equal to MGS) element by element."""
    import paper_2410_14917_gb300 as lsa

    cfg = W.config(2)
    op, v = _op(cfg)
    with _grid_kernel_env(1):
        y, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy")
    assert st["arnoldi_kernel"] == 4 and st["status"] == 0
    ref, info = oracle_phiv(cfg, "hcwy")
    assert max(rel_errors(y, ref)) < FP64_TOL
    assert st["m_eff"] == info["m_eff"] == cfg["m"]


def _box3d(nx, ny, nz, **kw):
    cfg = W.adr3d(nx, **kw)
    cfg.update(ny=ny, nz=nz, name=f"adr3d_{nx}x{ny}x{nz}")
    return cfg


# ragged shares and chunks: N not a multiple of the 512-point chunk or of 32;
# a two-plane z extent (both z neighbours are the other plane)
FLAT_CASES = [W.adr3d(20, m=24, p=1), _box3d(33, 17, 9, m=20, p=2), _box3d(16, 8, 3, m=12, p=1),
              _box3d(7, 5, 2, m=10, p=1), W.adr3d(64, m=40, p=1),
              W.advdiff2d(40, ny=23, m=24, p=1), W.advdiff2d(3, ny=5, m=6, p=1),
              W.grayscott2d(40, m=32, p=2), W.grayscott2d(96, m=40, p=1)]


@pytest.mark.parametrize("cfg", FLAT_CASES, ids=[c["name"] for c in FLAT_CASES])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flat_two_phase_matches_tile_form_and_oracle(cfg, variant, precision):
    """The flat two-phase step (both passes over equal flat shares): w is
    the tile passes' value, the inner products sum the points in other
    groups, so basis and H agree with the tile form to rounding; the phi
    product matches the oracle element by element, and the step takes one
    barrier without a reduction besides its reduction."""
    import paper_2410_14917_gb300 as lsa

    op, v = _op(cfg)
    m = min(cfg["m"], op.N)
    out = {}
    for two in (1, 2):
        with _grid_kernel_env(two):
            V, H, st = lsa.arnoldi(op, v, m, variant=variant, precision=precision)
        out[two] = (V.cpu().numpy().astype(np.float64), H.cpu().numpy(), st)
    (V1, H1, s1), (V2, H2, s2) = out[1], out[2]
    assert s1["arnoldi_kernel"] == 4 and s2["arnoldi_kernel"] == 5
    assert s2["status"] == 0 and s2["m_eff"] == s1["m_eff"] == m
    tol = 1e-10 if precision == "fp64" else 1e-4
    assert np.max(np.abs(H1 - H2)) <= tol * np.max(np.abs(H1))
    assert np.max(np.abs(V1 - V2)) <= tol * np.max(np.abs(V1))
    assert s2["grid_syncs"] == m + 1 + s2["norm_fallbacks"]
    assert s2["grid_barriers"] == s2["grid_syncs"] + m
    with _grid_kernel_env(2):
        y, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant=variant, precision=precision)
    assert st["arnoldi_kernel"] == 5 and st["status"] == 0
    ref, info = oracle_phiv(cfg, variant)
    assert max(rel_errors(y, ref)) < (FP64_TOL if precision == "fp64" else FP32_TOL)
    assert st["m_eff"] == info["m_eff"]


def test_flat_two_phase_headline_shape():
    """Gray-Scott 512^2 with m = 64 in float64: the flat form agrees with the
    tile two-phase form to rounding, and the Arnoldi relation holds on sampled
    columns of its basis."""
    import paper_2410_14917_gb300 as lsa

    cfg = W.config(1)
    op, v = _op(cfg)
    m = cfg["m"]
    res = {}
    for two in (1, 2):
        with _grid_kernel_env(two):
            res[two] = lsa.arnoldi(op, v, m, variant="hcwy")
    assert res[1][2]["arnoldi_kernel"] == 4 and res[2][2]["arnoldi_kernel"] == 5
    (V1, H1, _), (V2, H2, _) = res[1], res[2]
    assert float((H1 - H2).abs().max() / H1.abs().max()) < 1e-10
    for j in (0, 17, m - 1):
        Av = lsa.matvec(op, V2[:, j].contiguous())
        r = Av - V2 @ H2[:, j]
        assert float(r.norm() / Av.norm()) < 1e-11


def test_flat_two_phase_adr256_fp32_matches_oracle():
    """The flat form on the 3D ADR 256^3 workload with the float32 basis
    (N = 16.7M, m = 40): the phi product against the oracle's H-CWY form,
    element by element and normwise."""
    import paper_2410_14917_gb300 as lsa

    cfg = W.config(2)
    op, v = _op(cfg)
    with _grid_kernel_env(2):
        y, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy", precision="fp32")
    assert st["arnoldi_kernel"] == 5 and st["status"] == 0
    ref, info = oracle_phiv(cfg, "hcwy")
    assert max(rel_errors(y, ref)) < FP32_TOL
    assert st["m_eff"] == info["m_eff"] == cfg["m"]


def test_tune_step_3d_times_three_forms():
    """On the 3D ADR operator in float64 the tuner also times the flat form;
    later calls run the recorded form, and the float64 default (nothing
    recorded) is the flat form."""
    import paper_2410_14917_gb300 as lsa

    cfg = W.adr3d(40, m=16, p=1)
    op, v = _op(cfg)
    os.environ.pop("LSA_TWO_PHASE", None)
    with env(LSA_TMA=0, LSA_STREAM=0, LSA_CLUSTER=0):
        _, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy")
        assert st["arnoldi_kernel"] == 5
        two, ms1, ms2 = lsa.tune_step(op, v, cfg["m"], variant="hcwy", precision="fp64", reps=1)
        assert two in (0, 1, 2) and ms1 > 0 and ms2 > 0
        _, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="hcwy")
        assert st["arnoldi_kernel"] == (3 + two if two else 0)
