"""Batched phi products (lsa_batch_* / lsa_phiv_batched) against the oracle.

Each instance of a batch is the computation of lsa_phiv; its result must match
the oracle's Krylov product O-Krylov of the same (operator, v, h, p, m,
variant) within the tolerance of the single call, whatever the CTA tiling:
one CTA per instance, CTA groups for the costliest instances, or the whole
grid per instance.  The full 512-instance workload is checked on a sample of
instances the oracle computes one by one."""
import numpy as np
import pytest

import workloads as W
from oracle import exact as OE
from oracle import operators as OP
from tests.gpu_util import FP32_TOL, FP64_TOL, expected_syncs, oracle_phiv, rel_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lsa():
    import paper_2410_14917_gb300 as lsa
    return lsa


# small batch: ragged tiles (6, 24, 40, 72, 100 are not multiples of 16) and
# uneven m, plus one 5 x 5 instance whose m = 40 exceeds N = 25 (capped at N;
# the Krylov space is then the whole space and the product is exact)
SMALL = W.batched_advdiff2d(18, seed=W.SEED_BASE + 31, sides=(6, 16, 24, 40, 72, 100),
                            m_range=(8, 40))
SMALL["instances"].append(W.advdiff2d(5, diff=0.01, h=SMALL["h"], p=SMALL["p"], m=40,
                                      seed=W.SEED_BASE + 99, name="batch_tiny_5"))


def _batch(bcfg, variant="hcwy", precision="fp64", zero=()):
    lsa = _lsa()
    insts = bcfg["instances"]
    ops = [lsa.Operator.from_workload(c, {}) for c in insts]
    ms = [c["m"] for c in insts]
    vs = W.batched_inputs(bcfg)
    for i in zero:
        vs[i] = np.zeros_like(vs[i])
    v = torch.from_numpy(np.concatenate(vs)).cuda()
    b = lsa.Batch(ops, ms, bcfg["h"], bcfg["p"], variant=variant, precision=precision)
    return b, v, vs


def _reference(bcfg, i, variant, vs=None):
    c = bcfg["instances"][i]
    N = W.n_dof(c)
    m = min(c["m"], N)
    if vs is not None and not np.any(vs[i]):
        return np.zeros((bcfg["p"] + 1, N)), m
    if c["m"] >= N:      # full Krylov space: the dense exact products
        inp = W.make_inputs(c)
        A = OP.from_workload(c, inp).toarray()
        return OE.phi_products_dense(A, inp["v"], bcfg["h"], bcfg["p"]), m
    y, _ = oracle_phiv(c, variant=variant, m=m, p=bcfg["p"], h=bcfg["h"])
    return y, m


def _check_instances(b, y, bcfg, variant, tol, idx=None, vs=None):
    st, fin, stats = b.stats()
    assert st >= 0, st
    assert fin == b.count
    parts = b.split(y)
    idx = range(b.count) if idx is None else idx
    for i in idx:
        ref, m = _reference(bcfg, i, variant, vs)
        errs = rel_errors(parts[i], ref) if np.any(ref) else [float(parts[i].abs().max())]
        assert max(errs) < tol, (i, errs)
        s = stats[i]
        if np.any(ref):
            assert s["m_eff"] == m or s["breakdown"], (i, s)
            if not s["breakdown"]:
                assert s["grid_syncs"] == expected_syncs(variant, m, s["norm_fallbacks"]), (i, s)


@pytest.mark.parametrize("variant", ["hcwy", "hncwy", "hgsmgs", "mgs", "cgs2"])
def test_batched_each_tiling_matches_oracle(variant):
    b, v, _ = _batch(SMALL, variant)
    n = b.count
    for gs, nl in [(1, 0), (4, n // 3), (b.ctas, n)]:
        b.set_tiling(gs, nl)
        y = b.run(v, graph=False)
        torch.cuda.synchronize()
        _check_instances(b, y, SMALL, variant, FP64_TOL)
    b.close()


def test_batched_fp32_basis_matches_oracle():
    b, v, _ = _batch(SMALL, "hcwy", "fp32")
    for gs, nl in [(1, 0), (8, 6)]:
        b.set_tiling(gs, nl)
        y = b.run(v, graph=False)
        torch.cuda.synchronize()
        _check_instances(b, y, SMALL, "hcwy", FP32_TOL)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_two_phase_step_bitwise_equal_and_matches_oracle(precision):
    """The two-phase hybrid step inside the batched kernel (its extra barrier
    counted over an instance's group, or a single CTA): bitwise the one-pass
    result on each tiling, and within tolerance of the oracle."""
    b, v, _ = _batch(SMALL, "hcwy", precision)
    n = b.count
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    for gs, nl in [(1, 0), (4, n // 2), (8, n)]:
        b.set_tiling(gs, nl)
        out = []
        for two in (0, 1):
            b.set_step_form(two)
            assert b.step_form == two
            out.append(b.run(v, graph=False).clone())
            torch.cuda.synchronize()
        assert torch.equal(out[0], out[1]), (gs, nl)
        _check_instances(b, out[1], SMALL, "hcwy", tol)
    b.close()


def test_graph_replay_is_bitwise_equal_to_direct_launch():
    b, v, _ = _batch(SMALL, "hcwy")
    b.set_tiling(4, 5)
    y0 = b.run(v, graph=False).clone()
    y1 = b.run(v, graph=True)
    y2 = b.run(v, y=y1, graph=True)          # replay of the captured graph
    torch.cuda.synchronize()
    assert torch.equal(y0, y2)
    st, fin, _ = b.stats()
    assert st >= 0 and fin == b.count
    b.close()


def test_batched_equals_loop_of_single_calls():
    lsa = _lsa()
    b, v, vs = _batch(SMALL, "hcwy")
    b.set_tiling(1, 0)
    y = b.run(v, graph=True)
    torch.cuda.synchronize()
    parts = b.split(y)
    for i, c in enumerate(SMALL["instances"]):
        op = lsa.Operator.from_workload(c, {})
        ys, _ = lsa.phiv(op, torch.from_numpy(vs[i]).cuda(), SMALL["h"], SMALL["p"], c["m"],
                         variant="hcwy")
        err = rel_errors(parts[i], ys.cpu().numpy())
        assert max(err) < 1e-12, (i, err)
    b.close()


def test_zero_start_vector_instance_gives_zero():
    b, v, vs = _batch(SMALL, "hcwy", zero=(2, 7))
    b.set_tiling(2, 9)
    y = b.run(v, graph=False)
    torch.cuda.synchronize()
    _check_instances(b, y, SMALL, "hcwy", FP64_TOL, vs=vs)
    b.close()


def test_tuner_picks_a_valid_tiling_and_keeps_parity():
    b, v, _ = _batch(SMALL, "hcwy")
    gs, nl, ms = b.tune(v, reps=1)
    assert 1 <= gs <= b.ctas and 0 <= nl <= b.count and ms > 0
    assert b.tiling == (gs, nl) and b.step_form in (0, 1)
    y = b.run(v, graph=True)
    torch.cuda.synchronize()
    _check_instances(b, y, SMALL, "hcwy", FP64_TOL)
    b.close()


def test_one_shot_entry_point():
    lsa = _lsa()
    insts = SMALL["instances"]
    ops = [lsa.Operator.from_workload(c, {}) for c in insts]
    v = torch.from_numpy(np.concatenate(W.batched_inputs(SMALL))).cuda()
    y, st, stats = lsa.phiv_batched(ops, v, SMALL["h"], SMALL["p"], [c["m"] for c in insts])
    assert st >= 0
    off = 0
    for i, c in enumerate(insts):
        N = W.n_dof(c)
        ref, _ = _reference(SMALL, i, "hcwy")
        part = y[off:off + (SMALL["p"] + 1) * N].view(SMALL["p"] + 1, N)
        assert max(rel_errors(part, ref)) < FP64_TOL, i
        off += (SMALL["p"] + 1) * N


def test_argument_errors():
    import ctypes
    lsa = _lsa()
    from paper_2410_14917_gb300 import _binding as B
    a = lsa.Operator.advdiff2d(32, 32, 1 / 32, 0.01, (1.0, 0.5))
    u0 = torch.rand(64, dtype=torch.float64, device="cuda")
    g = lsa.Operator.grayscott2d(8, 8, 0.1, 1e-3, 1e-3, 0.04, 0.06, u0, u0)
    with pytest.raises(lsa.LsaError):          # mixed operator families
        lsa.Batch([a, g], [8, 8], 0.01, 1)
    with pytest.raises(lsa.LsaError):          # m out of range
        lsa.Batch([a], [0], 0.01, 1)
    with pytest.raises(lsa.LsaError):          # p out of range
        lsa.Batch([a], [8], 0.01, 9)
    b = lsa.Batch([a, a], [8, 8], 0.01, 1)
    with pytest.raises(lsa.LsaError):
        b.set_tiling(0, 0)
    with pytest.raises(lsa.LsaError):
        b.set_tiling(2, 3)
    with pytest.raises(lsa.LsaError):
        b.set_tiling(b.ctas + 1, 1)
    b.close()
    # workspace too small
    ops = lsa._op_array([a])
    mm = (ctypes.c_int * 1)(8)
    need = B.lib().lsa_batch_workspace_bytes(ops, mm, 1, 1, 0)
    w = lsa.Workspace(need)
    h = ctypes.c_void_p()
    st = B.lib().lsa_batch_create(ops, mm, 1, 0.01, 1, 0.0, 2, 0, ctypes.c_void_p(w.ptr), need - 256,
                                  ctypes.byref(h), None)
    assert st == B.LSA_ERR_WORKSPACE


def test_full_workload_sampled_against_oracle():
    """The 512-instance workload at full size, tuned tiling, graph replay;
    sampled instances (smallest, largest, cheapest, costliest, three seeded
    picks) against the oracle one by one, all instances complete with m_eff = m."""
    bcfg = W.config(3)
    b, v, _ = _batch(bcfg, "hcwy")
    b.tune(v, reps=1)
    y = b.run(v, graph=True)
    y = b.run(v, y=y, graph=True)
    torch.cuda.synchronize()
    st, fin, stats = b.stats()
    assert st >= 0 and fin == b.count
    insts = bcfg["instances"]
    assert all(s["m_eff"] == c["m"] for s, c in zip(stats, insts))
    N = np.array([W.n_dof(c) for c in insts])
    cost = np.array([W.n_dof(c) * c["m"] * (c["m"] + 7) for c in insts])
    rng = np.random.default_rng(W.SEED_BASE + 77)
    sample = sorted(set([int(N.argmin()), int(N.argmax()), int(cost.argmin()), int(cost.argmax())]
                        + [int(x) for x in rng.choice(len(insts), 3, replace=False)]))
    _check_instances(b, y, bcfg, "hcwy", FP64_TOL, idx=sample)
    b.close()


@pytest.mark.parametrize("variant", ["hcwy", "mgs"])
def test_batched_default_step_form(variant):
    """A new plan runs the two-phase step for the hybrid variants (the one
    that the tuner picks on the benchmark batch) and the one-pass passes of
    the other variants."""
    b, v, _ = _batch(SMALL, variant)
    assert b.step_form == (1 if variant == "hcwy" else 0)
    y = b.run(v, graph=False)
    torch.cuda.synchronize()
    _check_instances(b, y, SMALL, variant, FP64_TOL)
    b.close()
