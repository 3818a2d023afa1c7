"""The exponential integrators of Sect. 4 (SRERK3, EPI4, EPI5) on the GPU path
(paper_2410_14917_gb300.integrators over lsa_phiv_lincomb, lsa_rhs,
lsa_matvec and lsa_axpby) against the oracle's integrators with the same
Krylov dimension and sub-steps, and the two new kernels against the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import integrators as OI

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gs_case(n=32, ny=24):
    cfg = W.grayscott2d(n, Du=2e-3, Dv=1e-3, h=0.5, seed=107)
    cfg.update(ny=ny, name=f"grayscott2d_{n}x{ny}")
    inp = W.make_inputs(cfg)
    return cfg, np.concatenate([inp["u0"], inp["v0"]])


def make(cfg, u0, m=30, nsub=1, variant="hcwy"):
    from paper_2410_14917_gb300.integrators import GrayScottIntegrator

    return GrayScottIntegrator(cfg["nx"], cfg["ny"], cfg["dx"], cfg["diff"], cfg["diff2"], cfg["F"],
                               cfg["k"], torch.from_numpy(u0).cuda(), m=m, nsub=nsub, variant=variant)


def rel(a, b):
    """The larger of the normwise and the element-wise (max-abs over max-abs) error."""
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = np.asarray(b)
    return float(max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b))))


def test_rhs_kernel_matches_oracle():
    cfg, u0 = gs_case(40, 24)
    it = make(cfg, u0)
    F, _ = OI.grayscott_problem(cfg)
    w = np.random.default_rng(3).uniform(0, 1, u0.size)
    f = it.rhs(torch.from_numpy(w).cuda(), torch.empty(u0.size, dtype=torch.float64, device="cuda"))
    assert rel(f, F(w)) < 1e-13


def test_axpby_kernel():
    cfg, u0 = gs_case()
    it = make(cfg, u0)
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(u0.size), rng.standard_normal(u0.size)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    w = it.axpby(0.3, xd, -1.7, yd, xd)          # in place on x
    assert rel(w, 0.3 * x - 1.7 * y) < 1e-15


@pytest.mark.parametrize("method,nsteps", [("srerk3", 3), ("epi4", 5), ("epi5", 6)])
@pytest.mark.parametrize("variant", ["hcwy", "mgs"])
def test_integrator_matches_oracle(method, nsteps, variant):
    cfg, u0 = gs_case()
    h, m, nsub = 0.5, 30, 2
    F, Jf = OI.grayscott_problem(cfg)
    ref = OI.integrate(method, F, Jf, u0, h, nsteps, OI.krylov_lincomb(m, nsub, "mgs"))
    it = make(cfg, u0, m=m, nsub=nsub, variant=variant)
    u = it.run(method, h, nsteps)
    assert rel(u, ref) < 1e-10
    assert it.stats["steps"] == nsteps
    # one linear combination per SRERK3 stage and step, one per EPI step (Sect. 4)
    P = {"srerk3": 0, "epi4": 2, "epi5": 3}[method]
    start = min(P, nsteps)
    assert it.stats["lincomb_calls"] == 2 * start + (nsteps - start) if P else 2 * nsteps
