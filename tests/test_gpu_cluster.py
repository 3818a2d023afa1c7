"""The single-cluster kernel (basis in the CTAs' shared memory, halo over
distributed shared memory, cluster barriers) for small 2D advection-diffusion
grids in float64: against the oracle and against the grid-wide kernel, for
every hybrid correction (Algs. 5/6/7), on 1 to 16 tiles, through lsa_phiv and
lsa_arnoldi (basis, Hessenberg matrix, Arnoldi relation)."""
import os

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import FP64_TOL, device_inputs, expected_syncs, oracle_phiv, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [W.config(0), W.advdiff2d(32, ny=48, m=24, p=2), W.advdiff2d(16, m=12, p=1),
         W.advdiff2d(48, ny=64, m=64, p=3, h=0.05)]


def run(cfg, variant, cluster, fn="phiv"):
    import paper_2410_14917_gb300 as lsa

    old = os.environ.get("LSA_CLUSTER")
    os.environ["LSA_CLUSTER"] = "1" if cluster else "0"
    try:
        inp = W.make_inputs(cfg)
        v, fields = device_inputs(cfg, inp, torch)
        op = lsa.Operator.from_workload(cfg, fields)
        if fn == "phiv":
            y, st = lsa.phiv(op, v, cfg["h"], cfg["p"], cfg["m"], variant=variant)
            return y.cpu().numpy(), st
        V, H, st = lsa.arnoldi(op, v, cfg["m"], variant=variant)
        return (V.cpu().numpy(), H.cpu().numpy()), st
    finally:
        if old is None:
            os.environ.pop("LSA_CLUSTER", None)
        else:
            os.environ["LSA_CLUSTER"] = old


@pytest.mark.parametrize("cfg", CASES, ids=[f"{c['name']}_m{c['m']}" for c in CASES])
@pytest.mark.parametrize("variant", ["hcwy", "hncwy", "hgsmgs"])
def test_cluster_kernel_matches_oracle_and_grid_kernel(cfg, variant):
    y_c, st_c = run(cfg, variant, True)
    y_g, st_g = run(cfg, variant, False)
    assert st_c["arnoldi_kernel"] == 3 and st_g["arnoldi_kernel"] in (0, 4, 5)
    ref, info = oracle_phiv(cfg)
    assert max(rel_errors(y_c, ref)) < FP64_TOL
    assert max(rel_errors(y_c, y_g)) < FP64_TOL
    assert st_c["m_eff"] == st_g["m_eff"] == info["m_eff"]
    assert st_c["grid_syncs"] == expected_syncs(variant, st_c["m_eff"], st_c["norm_fallbacks"])


def test_cluster_kernel_arnoldi_basis_and_relation():
    """lsa_arnoldi through the cluster kernel: the orthonormal basis and H
    against the oracle's MGS, and the Arnoldi relation A V_m = V_{m+1} H (Eq. 12)."""
    from oracle import arnoldi as OA
    from oracle import operators as OP

    cfg = W.config(0)
    (V, H), st = run(cfg, "hcwy", True, fn="arnoldi")
    assert st["arnoldi_kernel"] == 3
    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    m = cfg["m"]
    ref = OA.arnoldi(lambda x: A @ x, inp["v"], m, "mgs")
    assert np.abs(H - ref["H"]).max() / np.abs(ref["H"]).max() < 1e-10
    assert np.abs(V - ref["V"]).max() < 1e-9
    R = (A @ V[:, :m]) - V @ H
    assert np.linalg.norm(R) / np.linalg.norm(H) < 1e-12
