"""The incomplete-orthogonalisation variant (ioCGS, the paper's reference
baseline) through the CUDA path against the oracle's ioCGS: phi products in
both precisions, the Arnoldi output (banded H, locally orthogonal V), sync
counts, and the batched form."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import FP32_TOL, FP64_TOL, device_inputs, expected_syncs, oracle_phiv, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [W.config(0), W.grayscott2d(72, m=40, p=2, Du=2e-3, Dv=1e-3, h=0.5),
         W.adr3d(40, m=30, p=1), W.advdiff2d(37, ny=29, m=25, p=2)]


@pytest.mark.parametrize("cfg", CASES, ids=[c["name"] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_iocgs_phiv_matches_oracle_iocgs(cfg, precision):
    import paper_2410_14917_gb300 as lsa

    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    y, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant="iocgs", precision=precision)
    ref, info = oracle_phiv(cfg, variant="iocgs")
    assert max(rel_errors(y, ref)) < (FP64_TOL if precision == "fp64" else FP32_TOL)
    assert st["m_eff"] == info["m_eff"]
    assert st["grid_syncs"] == expected_syncs("iocgs", st["m_eff"])


def test_iocgs_arnoldi_output_matches_oracle():
    import paper_2410_14917_gb300 as lsa
    from oracle import arnoldi as OA
    from oracle import operators as OP

    cfg = W.advdiff2d(40, ny=36, m=20)
    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    V, H, st = lsa.arnoldi(op, v, cfg["m"], variant="iocgs")
    A = OP.from_workload(cfg, inp)
    ref = OA.iocgs(lambda x: A @ x, inp["v"], cfg["m"])
    V, H = V.cpu().numpy(), H.cpu().numpy()
    assert np.abs(H - ref["H"]).max() / np.abs(ref["H"]).max() < 1e-11
    assert np.abs(V - ref["V"]).max() < 1e-10
    assert st["grid_syncs"] == 1 + 2 * cfg["m"]


def test_iocgs_batched_matches_single_calls():
    import paper_2410_14917_gb300 as lsa

    cfgs = [W.advdiff2d(n, m=m, p=2, seed=500 + n) for n, m in ((32, 16), (48, 24), (64, 30), (40, 20))]
    ops, vs = [], []
    for c in cfgs:
        inp = W.make_inputs(c)
        ops.append(lsa.Operator.from_workload(c, {}))
        vs.append(torch.from_numpy(inp["v"]).cuda())
    h, p = cfgs[0]["h"], 2
    b = lsa.Batch(ops, [c["m"] for c in cfgs], h, p, variant="iocgs")
    v = torch.cat(vs)
    y = torch.empty(b.y_elems, dtype=torch.float64, device="cuda")
    b.run(v, y, graph=False)
    parts = b.split(y)
    for i, c in enumerate(cfgs):
        ref, _ = oracle_phiv(c, variant="iocgs")
        assert max(rel_errors(parts[i], ref)) < FP64_TOL
    b.close()
