"""S1: the stencil matvec of the CUDA tile engine against the oracle's sparse
matrices (float64: ~1 ulp level; float32 basis: float rounding)."""
import numpy as np
import pytest

import workloads as W
from oracle import operators as OP
from tests.gpu_util import device_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    W.advdiff2d(64), W.advdiff2d(17, ny=33), W.advdiff2d(3, ny=5), W.advdiff2d(1, ny=1),
    W.advdiff2d(40, ny=16, vel=(-2.0, 3.0)),
    W.grayscott2d(16), W.grayscott2d(33, Du=2e-3, Dv=1e-3), W.grayscott2d(5),
    W.adr3d(16), W.adr3d(20), W.adr3d(3), W.adr3d(33, vel=(1.0, -0.5, 2.0)),
]


@pytest.mark.parametrize("cfg", CASES, ids=[c["name"] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_matvec_matches_sparse_operator(cfg, precision):
    import paper_2410_14917_gb300 as lsa

    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    A = OP.from_workload(cfg, inp)
    if precision == "fp64":
        y = lsa.matvec(op, v).cpu().numpy()
        ref = A @ inp["v"]
        err = np.abs(y - ref).max() / max(np.abs(ref).max(), 1.0)
        assert err < 1e-13, err
    else:
        x32 = v.float()
        y = lsa.matvec(op, x32, precision="fp32").cpu().numpy().astype(np.float64)
        ref = A @ x32.cpu().numpy().astype(np.float64)
        err = np.abs(y - ref).max() / max(np.abs(ref).max(), 1.0)
        assert err < 2e-6, err
