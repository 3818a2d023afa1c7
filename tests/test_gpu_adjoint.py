"""Gradients of 1/2 ||phi_1(h A(theta)) v - y_t||^2 on the Gray-Scott Jacobian
through the CUDA path (lsa_phiv_vjp and the autograd function) against the
oracle's gradients, central differences of the GPU loss (step 1e-6), and the
two operators the gradient needs (transpose, Frechet block operator)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import adjoint as OAD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_case(n=32, ny=None, m=40, h=0.5):
    cfg = W.grayscott2d(n, Du=2e-3, Dv=1e-3, h=h, p=1, m=m, seed=101)
    if ny:
        cfg.update(ny=ny, name=f"grayscott2d_{n}x{ny}")
    return cfg


def setup(cfg):
    import paper_2410_14917_gb300 as lsa

    inp = W.adjoint_inputs(cfg)
    dev = {k: torch.from_numpy(v).cuda() for k, v in inp.items()}
    op = lsa.Operator.from_workload(cfg, dev)
    return lsa, inp, dev, op


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


GRAD_TOL = 1e-10    # the float64 contract, element-wise (max-abs over max-abs)


def check_grads(gv, gs, ref, ref_frechet):
    """dv, dh and each dtheta_k against the oracle: like for like (the oracle's
    closed form for dL/dF, the form the library evaluates), and the F
    component also against the oracle's block-operator (Frechet) product."""
    assert rel(gv, ref["dv"]) < GRAD_TOL
    assert abs(gs[0] - ref["dh"]) / abs(ref["dh"]) < GRAD_TOL
    for k in range(4):
        assert abs(gs[1 + k] - ref["dtheta"][k]) / abs(ref["dtheta"][k]) < GRAD_TOL, k
    assert abs(gs[3] - ref_frechet["dtheta"][2]) / abs(ref_frechet["dtheta"][2]) < GRAD_TOL


def test_transposed_operator_is_the_adjoint():
    cfg = small_case(24, ny=40)
    lsa, inp, dev, op = setup(cfg)
    rng = np.random.default_rng(5)
    N = 2 * cfg["nx"] * cfg["ny"]
    x = torch.from_numpy(rng.standard_normal(N)).cuda()
    y = torch.from_numpy(rng.standard_normal(N)).cuda()
    Ax = lsa.matvec(op, x)
    Aty = lsa.matvec(op.derived(kind="grayscott2d_t"), y)
    lhs, rhs = float(Ax @ y), float(x @ Aty)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
    A, _ = OAD.grayscott_parts(cfg, inp)
    assert rel(Aty.cpu().numpy(), A.T @ y.cpu().numpy()) < 1e-13


@pytest.mark.parametrize("k", range(4))
def test_frechet_block_operator_matches_oracle(k):
    cfg = small_case(24, ny=40)
    lsa, inp, dev, op = setup(cfg)
    A, dA = OAD.grayscott_parts(cfg, inp)
    K = sp.bmat([[A, dA[k]], [None, A]], format="csr")
    z = np.random.default_rng(9 + k).standard_normal(K.shape[0])
    Kz = lsa.matvec(op.derived(kind="grayscott2d_frechet", aux=k), torch.from_numpy(z).cuda())
    assert rel(Kz.cpu().numpy(), K @ z) < 1e-13


@pytest.mark.parametrize("variant", ["mgs", "hcwy", "hgsmgs"])
def test_vjp_matches_oracle_gradient(variant):
    import paper_2410_14917_gb300 as lsa

    cfg = small_case(32, m=40)
    lsa, inp, dev, op = setup(cfg)
    h, m = cfg["h"], cfg["m"]
    A, dA = OAD.grayscott_parts(cfg, inp)
    ref = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], h, m, f_closed=True)
    ref_f = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], h, m)
    y, _ = lsa.phiv(op, dev["v"], h, 2, m, variant=variant)
    r = y[1] - dev["y_target"]
    gv, gs, st = lsa.phiv_vjp(op, dev["v"], h, m, r, y, variant=variant, stats=True)
    assert st["status"] in (0, 1)
    check_grads(gv.cpu().numpy(), gs.cpu().numpy(), ref, ref_f)


def test_autograd_function_matches_vjp_and_central_differences():
    import paper_2410_14917_gb300 as lsa

    cfg = small_case(32, m=40)
    lsa, inp, dev, op = setup(cfg)
    m = cfg["m"]
    yt = dev["y_target"]

    def loss(v, h, theta):
        y = lsa.Phi1GrayScott.apply(v, h, theta, op, m, "hcwy")
        return 0.5 * ((y - yt) ** 2).sum()

    v = dev["v"].clone().requires_grad_(True)
    h = torch.tensor(cfg["h"], dtype=torch.float64, requires_grad=True)
    theta = torch.tensor([cfg["diff"], cfg["diff2"], cfg["F"], cfg["k"]], dtype=torch.float64,
                         requires_grad=True)
    L = loss(v, h, theta)
    L.backward()
    A, dA = OAD.grayscott_parts(cfg, inp)
    ref = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], cfg["h"], m, f_closed=True)
    ref_f = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], cfg["h"], m)
    assert abs(float(L.detach()) - ref["L"]) / ref["L"] < 1e-10
    gs = np.concatenate([[float(h.grad)], theta.grad.numpy()])
    check_grads(v.grad.cpu().numpy(), gs, ref, ref_f)
    # central differences of the GPU loss, step 1e-6
    eps = 1e-6
    with torch.no_grad():
        for kk in range(4):
            e = torch.zeros(4, dtype=torch.float64)
            e[kk] = eps
            fd = (float(loss(dev["v"], h.detach(), theta.detach() + e))
                  - float(loss(dev["v"], h.detach(), theta.detach() - e))) / (2 * eps)
            assert abs(fd - float(theta.grad[kk])) / abs(float(theta.grad[kk])) < 1e-5
        fd = (float(loss(dev["v"], h.detach() + eps, theta.detach()))
              - float(loss(dev["v"], h.detach() - eps, theta.detach()))) / (2 * eps)
        assert abs(fd - float(h.grad)) / abs(float(h.grad)) < 1e-5
        d = torch.from_numpy(np.random.default_rng(2).standard_normal(v.numel())).cuda()
        d /= d.norm()
        fd = (float(loss(dev["v"] + eps * d, h.detach(), theta.detach()))
              - float(loss(dev["v"] - eps * d, h.detach(), theta.detach()))) / (2 * eps)
        assert abs(fd - float(v.grad @ d)) / float(v.grad.norm()) < 1e-5


def test_vjp_rejects_bad_arguments():
    import paper_2410_14917_gb300 as lsa
    from paper_2410_14917_gb300 import LsaError

    cfg = small_case(16, m=10)
    lsa, inp, dev, op = setup(cfg)
    y, _ = lsa.phiv(op, dev["v"], cfg["h"], 2, 10)
    with pytest.raises(LsaError):
        lsa.phiv_vjp(op, dev["v"], 0.0, 10, dev["v"], y)                   # h = 0
    with pytest.raises(LsaError):
        lsa.phiv_vjp(op.derived(kind="grayscott2d_t"), dev["v"], 0.5, 10, dev["v"], y)
    with pytest.raises(LsaError):                                          # float32 basis form
        lsa.phiv(op.derived(kind="grayscott2d_t"), dev["v"], 0.5, 1, 10, precision="fp32")


def test_adjoint_workload_full_size_matches_oracle():
    """The 256 x 256 adjoint workload (m = 48), GPU (H-CWY) against the oracle (MGS)."""
    import paper_2410_14917_gb300 as lsa

    cfg = W.config(4)
    lsa, inp, dev, op = setup(cfg)
    h, m = cfg["h"], cfg["m"]
    y, _ = lsa.phiv(op, dev["v"], h, 2, m, variant="hcwy")
    r = y[1] - dev["y_target"]
    gv, gs, _ = lsa.phiv_vjp(op, dev["v"], h, m, r, y, variant="hcwy")
    A, dA = OAD.grayscott_parts(cfg, inp)
    ref = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], h, m, f_closed=True)
    ref_f = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], h, m)
    check_grads(gv.cpu().numpy(), gs.cpu().numpy(), ref, ref_f)
