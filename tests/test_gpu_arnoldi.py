"""lsa_arnoldi: every Gram-Schmidt variant against the oracle's MGS (Alg. 1):
same basis and Hessenberg matrix (unique with positive subdiagonal), the
Arnoldi relation, orthonormality and the grid-sync counts of each method."""
import numpy as np
import pytest

import workloads as W
from oracle import arnoldi as OA
from oracle import operators as OP
from tests.gpu_util import device_inputs, expected_syncs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = ["mgs", "cgs2", "hcwy", "hncwy", "hgsmgs"]
CASES = [(W.advdiff2d(24, ny=20), 20), (W.grayscott2d(20, Du=2e-3, Dv=1e-3), 30),
         (W.adr3d(12), 24), (W.advdiff2d(64), 30)]


@pytest.mark.parametrize("case", CASES, ids=[c[0]["name"] for c in CASES])
@pytest.mark.parametrize("variant", VARIANTS)
def test_arnoldi_fp64_matches_mgs_oracle(case, variant):
    import paper_2410_14917_gb300 as lsa

    cfg, m = case
    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    V, H, st = lsa.arnoldi(op, v, m, variant=variant)
    V = V.cpu().numpy()
    H = H.cpu().numpy()
    A = OP.from_workload(cfg, inp)
    ref = OA.mgs(lambda x: A @ x, inp["v"], m)
    assert st["m_eff"] == m and st["status"] == 0
    assert abs(st["beta"] - ref["beta"]) / ref["beta"] < 1e-13
    assert np.abs(H - ref["H"]).max() / np.abs(ref["H"]).max() < 1e-10
    assert np.abs(V - ref["V"]).max() < 1e-9
    R = A @ V[:, :m] - V @ H
    assert np.linalg.norm(R) / np.linalg.norm(H) < 1e-12
    orth = np.linalg.norm(np.eye(m + 1) - V.T @ V)
    orth_mgs = np.linalg.norm(np.eye(m + 1) - ref["V"].T @ ref["V"])
    assert orth < max(10 * orth_mgs, 1e-13), (orth, orth_mgs)
    assert st["grid_syncs"] == expected_syncs(variant, m, st["norm_fallbacks"])


@pytest.mark.parametrize("variant", VARIANTS)
def test_arnoldi_fp32_basis(variant):
    import paper_2410_14917_gb300 as lsa

    cfg = W.adr3d(16)
    m = 20
    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    V, H, st = lsa.arnoldi(op, v, m, variant=variant, precision="fp32")
    H = H.cpu().numpy()
    V = V.cpu().numpy().astype(np.float64)
    A = OP.from_workload(cfg, inp)
    ref = OA.mgs(lambda x: A @ x, inp["v"], m)
    assert np.abs(H - ref["H"]).max() / np.abs(ref["H"]).max() < 1e-4
    assert np.linalg.norm(np.eye(m + 1) - V.T @ V) < 1e-4
