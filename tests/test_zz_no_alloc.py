"""lsa_phiv_noalloc -- the entry point for callers that cannot allocate device
memory (plugins inside an application that owns the device memory pool,
latency-critical code that must not call cudaMalloc/cudaFree) -- gives the same
phi products as lsa_phiv with a caller-provided workspace, on two calls in a
row, through the C ABI.

The file is collected last (its name sorts last) so that a run that stops at
the first failure has run every other GPU test before this one.  No other test
depends on it or on the order: the test passes alone in a fresh process and
after the others (the static array is only touched here, and each call
re-initialises what must start at zero)."""
import ctypes

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import FP32_TOL, FP64_TOL, device_inputs, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg,variant,precision",
                         [(W.config(0), "hcwy", "fp64"), (W.grayscott2d(64, m=48, p=2), "hgsmgs", "fp64"),
                          (W.adr3d(24, m=30, p=1), "mgs", "fp32")],
                         ids=["advdiff2d_64-hcwy", "grayscott2d_64-hgsmgs", "adr3d_24-mgs-fp32"])
def test_noalloc_matches_phiv_on_two_calls(cfg, variant, precision):
    import paper_2410_14917_gb300 as lsa
    from paper_2410_14917_gb300 import _binding as B

    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    h, p, m = cfg["h"], cfg["p"], cfg["m"]
    ref, _ = lsa.phiv(op, v, h, p, m, variant=variant, precision=precision)
    ref = ref.cpu().numpy()
    lib = B.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    for _ in range(2):
        y = torch.full((p + 1, v.numel()), float("nan"), dtype=torch.float64, device="cuda")
        st = B.LsaStats()
        rc = lib.lsa_phiv_noalloc(ctypes.byref(op.c), ctypes.c_void_p(v.data_ptr()), h, p, m, 0.0,
                                  B.VARIANTS[variant], B.PRECISIONS[precision],
                                  ctypes.c_void_p(y.data_ptr()), ctypes.byref(st), stream)
        assert rc == 0, B.status_string(rc)
        assert st.status == 0 and st.m_eff == m
        assert max(rel_errors(y, ref)) < tol


def test_noalloc_rejects_problems_beyond_its_fixed_size():
    import paper_2410_14917_gb300 as lsa
    from paper_2410_14917_gb300 import _binding as B

    cfg = W.config(1)                     # 512^2 Gray-Scott, m = 64: ~290 MB of workspace
    inp = W.make_inputs(cfg)
    v, fields = device_inputs(cfg, inp, torch)
    op = lsa.Operator.from_workload(cfg, fields)
    y = torch.zeros((cfg["p"] + 1, v.numel()), dtype=torch.float64, device="cuda")
    rc = B.lib().lsa_phiv_noalloc(ctypes.byref(op.c), ctypes.c_void_p(v.data_ptr()), cfg["h"],
                                  cfg["p"], cfg["m"], 0.0, 2, 0, ctypes.c_void_p(y.data_ptr()),
                                  None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == B.LSA_ERR_WORKSPACE
    assert torch.count_nonzero(y).item() == 0
