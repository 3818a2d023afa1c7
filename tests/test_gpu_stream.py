"""The streaming float32-basis Arnoldi kernel (interior-only TMA stages, halo
by plain loads, a ring of stages sized per pass) against the oracle and
against the plain-load kernel, on single-species operators whose grids are
whole tiles: several z-segments, non-cubic boxes, the largest m (fewest
stages), and each hybrid correction (Algs. 5/6/7)."""
import os

import pytest

import workloads as W
from tests.gpu_util import FP32_TOL, device_inputs, oracle_phiv, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def box3d(nx, ny, nz, **kw):
    cfg = W.adr3d(nx, **kw)
    cfg.update(ny=ny, nz=nz, name=f"adr3d_{nx}x{ny}x{nz}")
    return cfg


CASES = [W.adr3d(16, m=20, p=1), W.adr3d(48, m=40, p=1), box3d(32, 48, 64, m=30, p=2),
         W.adr3d(32, m=48, p=1), W.advdiff2d(64, m=30, p=3), W.advdiff2d(80, ny=48, m=24, p=2)]


def run(cfg, variant, stream):
    import paper_2410_14917_gb300 as lsa

    old = {k: os.environ.get(k) for k in ("LSA_TMA", "LSA_STREAM")}
    os.environ["LSA_STREAM"] = "1" if stream else "0"
    os.environ["LSA_TMA"] = "0"
    try:
        inp = W.make_inputs(cfg)
        v, fields = device_inputs(cfg, inp, torch)
        op = lsa.Operator.from_workload(cfg, fields)
        y, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant=variant, precision="fp32")
        return y.cpu().numpy(), st
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("cfg", CASES, ids=[c["name"] for c in CASES])
@pytest.mark.parametrize("variant", ["hcwy", "hncwy", "hgsmgs"])
def test_stream_kernel_matches_oracle_and_plain_kernel(cfg, variant):
    y_s, st_s = run(cfg, variant, True)
    y_p, st_p = run(cfg, variant, False)
    assert st_s["arnoldi_kernel"] == 2 and st_p["arnoldi_kernel"] in (0, 4, 5)
    ref, info = oracle_phiv(cfg)
    assert max(rel_errors(y_s, ref)) < FP32_TOL
    assert max(rel_errors(y_p, ref)) < FP32_TOL
    assert max(rel_errors(y_s, y_p)) < FP32_TOL
    assert st_s["m_eff"] == st_p["m_eff"] == info["m_eff"]
    assert st_s["grid_syncs"] == cfg["m"] + 1 + st_s["norm_fallbacks"]


def test_stream_kernel_arnoldi_relation():
    """lsa_arnoldi through the streaming kernel: orthonormal basis and the
    Arnoldi relation A V_m = V_{m+1} H (Eq. 12) within float32 accuracy."""
    import numpy as np

    import paper_2410_14917_gb300 as lsa
    from oracle import operators as OP

    cfg = W.adr3d(32, m=24, p=1)
    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    V, H, st = lsa.arnoldi(op, v, cfg["m"], variant="hcwy", precision="fp32")
    assert st["arnoldi_kernel"] == 2
    V = V.double().cpu().numpy()
    H = H.cpu().numpy()
    m = cfg["m"]
    A = OP.from_workload(cfg, inp)
    G = V.T @ V
    assert np.linalg.norm(G - np.eye(m + 1)) < 1e-4
    R = (A @ V[:, :m]) - V @ H
    assert np.linalg.norm(R) / np.linalg.norm(A @ V[:, :m]) < 1e-5


@pytest.mark.parametrize("n", [128, 256])
def test_stream_kernel_large_grids_match_oracle(n):
    """The 3D ADR workload's kernel at 128^3 and at the full 256^3 (m = 40):
    many z-segments per tile column, every pass's stage ring at its working
    depth, against the oracle (its H-CWY form, which the oracle pins equal to
    MGS) element by element."""
    cfg = W.adr3d(n, m=40, p=1) if n != 256 else W.config(2)
    y_s, st_s = run(cfg, "hcwy", True)
    assert st_s["arnoldi_kernel"] == 2 and st_s["m_eff"] == 40
    ref, info = oracle_phiv(cfg, "hcwy")
    assert max(rel_errors(y_s, ref)) < FP32_TOL
    assert st_s["grid_syncs"] == cfg["m"] + 1 + st_s["norm_fallbacks"]
