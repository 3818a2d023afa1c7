"""Guard words around every caller-owned buffer a call writes (outputs and
workspace): the bytes before and after each buffer must be untouched after the
call, for the plain, streaming, augmented-operator and gradient kernels on
grids whose sizes are not multiples of the tile."""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PATTERN = 0xA5
GUARD = 4096            # bytes on each side; keeps the 256-byte alignment of the interior


class Guarded:
    def __init__(self, nbytes):
        self.nbytes = int(nbytes)
        self.buf = torch.full((GUARD + self.nbytes + GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
        self.ptr = self.buf.data_ptr() + GUARD
        assert self.ptr % 256 == 0

    def f64(self, n):
        return self.buf[GUARD:GUARD + 8 * n].view(torch.float64)

    def intact(self):
        torch.cuda.synchronize()
        return bool((self.buf[:GUARD] == PATTERN).all()) and bool((self.buf[GUARD + self.nbytes:] == PATTERN).all())


def lib():
    from paper_2410_14917_gb300 import _binding as B
    return B, B.lib()


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def gs_case(nx=40, ny=24, m=24):
    import paper_2410_14917_gb300 as lsa

    cfg = W.grayscott2d(nx, Du=2e-3, Dv=1e-3, h=0.5, m=m, seed=109)
    cfg.update(ny=ny, name=f"grayscott2d_{nx}x{ny}")
    inp = W.make_inputs(cfg)
    fields = {k: torch.from_numpy(v).cuda() for k, v in inp.items() if k != "v"}
    return lsa, cfg, inp, lsa.Operator.from_workload(cfg, fields), torch.from_numpy(inp["v"]).cuda()


@pytest.mark.parametrize("variant", ["hcwy", "mgs"])
def test_phiv_writes_only_its_buffers(variant):
    lsa, cfg, inp, op, v = gs_case()
    B, L = lib()
    N, p, m = v.numel(), 2, cfg["m"]
    y = Guarded((p + 1) * N * 8)
    work = Guarded(lsa.workspace_bytes(op, m, p, "fp64"))
    st = L.lsa_phiv(ctypes.byref(op.c), ctypes.c_void_p(v.data_ptr()), cfg["h"], p, m, 0.0, B.VARIANTS[variant],
                    B.PRECISIONS["fp64"], ctypes.c_void_p(y.ptr), ctypes.c_void_p(work.ptr), work.nbytes, None, stream())
    assert st == 0 and y.intact() and work.intact()
    ref, _ = lsa.phiv(op, v, cfg["h"], p, m, variant=variant)
    assert torch.equal(y.f64((p + 1) * N).view(p + 1, N), ref)


def test_arnoldi_writes_only_its_buffers():
    import paper_2410_14917_gb300 as lsa

    cfg = W.advdiff2d(48, ny=40, m=20)
    inp = W.make_inputs(cfg)
    op = lsa.Operator.from_workload(cfg, {})
    v = torch.from_numpy(inp["v"]).cuda()
    B, L = lib()
    N, m = v.numel(), cfg["m"]
    V = Guarded(N * (m + 1) * 8)
    H = Guarded((m + 1) * m * 8)
    work = Guarded(lsa.workspace_bytes(op, m, 0, "fp64"))
    st = L.lsa_arnoldi(ctypes.byref(op.c), ctypes.c_void_p(v.data_ptr()), m, B.VARIANTS["hcwy"], B.PRECISIONS["fp64"],
                       ctypes.c_void_p(V.ptr), ctypes.c_void_p(H.ptr), ctypes.c_void_p(work.ptr), work.nbytes,
                       None, stream())
    assert st == 0 and V.intact() and H.intact() and work.intact()


def test_streaming_kernel_writes_only_its_buffers():
    import paper_2410_14917_gb300 as lsa

    cfg = W.adr3d(32, m=20)
    inp = W.make_inputs(cfg)
    op = lsa.Operator.from_workload(cfg, {"r": torch.from_numpy(inp["r"]).cuda()})
    v = torch.from_numpy(inp["v"]).cuda()
    B, L = lib()
    N, p, m = v.numel(), 1, cfg["m"]
    y = Guarded((p + 1) * N * 8)
    work = Guarded(lsa.workspace_bytes(op, m, p, "fp32"))
    s = B.LsaStats()
    st = L.lsa_phiv(ctypes.byref(op.c), ctypes.c_void_p(v.data_ptr()), cfg["h"], p, m, 0.0, B.VARIANTS["hcwy"],
                    B.PRECISIONS["fp32"], ctypes.c_void_p(y.ptr), ctypes.c_void_p(work.ptr), work.nbytes,
                    ctypes.byref(s), stream())
    assert st in (0, 1) and s.arnoldi_kernel == 2
    assert y.intact() and work.intact()


def test_linear_combination_writes_only_its_buffers():
    lsa, cfg, inp, op, v = gs_case()
    B, L = lib()
    N, p, m = v.numel(), 3, cfg["m"]
    b = torch.from_numpy(W.lincomb_inputs(cfg, p)["b"]).cuda().contiguous()
    u = Guarded(N * 8)
    work = Guarded(lsa.workspace_bytes(op, min(m, N + p), 0, "fp64"))
    st = L.lsa_phiv_lincomb(ctypes.byref(op.c), ctypes.c_void_p(b.data_ptr()), p, 0.5, 2, m, 0.0,
                            B.VARIANTS["hcwy"], B.PRECISIONS["fp64"], ctypes.c_void_p(u.ptr),
                            ctypes.c_void_p(work.ptr), work.nbytes, None, stream())
    assert st == 0 and u.intact() and work.intact()
    ref, _ = lsa.phiv_lincomb(op, b, 0.5, m, 2, variant="hcwy")
    assert torch.equal(u.f64(N), ref)


def test_gradient_writes_only_its_buffers():
    lsa, cfg, inp, op, v = gs_case(32, 16)
    B, L = lib()
    N, m, h = v.numel(), cfg["m"], cfg["h"]
    y, _ = lsa.phiv(op, v, h, 2, m)
    r = (y[1] - 0.5).contiguous()
    gv = Guarded(N * 8)
    gs = Guarded(5 * 8)
    work = Guarded(lsa.vjp_workspace_bytes(op, m))
    st = L.lsa_phiv_vjp(ctypes.byref(op.c), ctypes.c_void_p(v.data_ptr()), h, m, B.VARIANTS["hcwy"],
                        ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(gv.ptr),
                        ctypes.c_void_p(gs.ptr), ctypes.c_void_p(work.ptr), work.nbytes, None, stream())
    assert st == 0 and gv.intact() and gs.intact() and work.intact()
    assert np.isfinite(gs.f64(5).cpu().numpy()).all()
