"""The TMA-staged hybrid kernel (float32 basis, shapes that meet the TMA
alignment rules) against the plain-load kernel and the oracle."""
import os

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import FP32_TOL, device_inputs, oracle_phiv, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [W.adr3d(16, m=20, p=1), W.adr3d(48, m=40, p=1), W.advdiff2d(64, m=30, p=3),
         W.advdiff2d(80, ny=48, m=24, p=2), W.grayscott2d(48, m=20, p=2, Du=2e-3, Dv=1e-3, h=0.5)]


def run(cfg, variant, tma):
    import paper_2410_14917_gb300 as lsa

    old = {k: os.environ.get(k) for k in ("LSA_TMA", "LSA_STREAM")}
    os.environ["LSA_TMA"] = "1" if tma else "0"
    os.environ["LSA_STREAM"] = "0"
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
def test_tma_kernel_matches_plain_kernel_and_oracle(cfg, variant):
    y_tma, st_tma = run(cfg, variant, True)
    y_plain, st_plain = run(cfg, variant, False)
    ref, _ = oracle_phiv(cfg)
    assert max(rel_errors(y_tma, ref)) < FP32_TOL
    assert max(rel_errors(y_plain, ref)) < FP32_TOL
    assert max(rel_errors(y_tma, y_plain)) < FP32_TOL
    # the TMA-staged kernel needs rows of whole 16-byte units and ny >= TY + 2
    staged = cfg["ny"] >= 18 and (cfg["nx"] * 4) % 16 == 0 and cfg["nx"] >= 16
    # (the grid kernel runs any step form: 0 one-pass, 4 two-phase, 5 flat two-phase)
    assert st_tma["arnoldi_kernel"] in ((1,) if staged else (0, 4, 5)) and st_plain["arnoldi_kernel"] in (0, 4, 5)
    assert st_tma["grid_syncs"] == st_plain["grid_syncs"] == cfg["m"] + 1 + st_tma["norm_fallbacks"]
