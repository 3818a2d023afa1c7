"""lsarnoldi for GB300: Krylov phi-function products with low-synchronisation
Arnoldi (arXiv 2410.14917), as hand-written CUDA for sm_103a behind a C ABI.

The Python layer only marshals arguments to the C entry points of
``include/lsarnoldi.h`` (same names without the ``lsa_`` prefix) and uses
PyTorch for device memory and streams.

    import paper_2410_14917_gb300 as lsa
    op = lsa.Operator.grayscott2d(512, 512, dx=2.5/512, Du=2e-5, Dv=1e-5, F=0.04, k=0.06,
                                  u0=u0_cuda, v0=v0_cuda)
    y, stats = lsa.phiv(op, v_cuda, h=1.0, p=2, m=64, variant="hcwy")
"""
from __future__ import annotations

import ctypes

import torch

from . import _binding as B
from ._binding import LsaError, LsaOp, LsaStats, PRECISIONS, VARIANTS, KINDS

__all__ = ["Operator", "phiv", "phiv_lincomb", "phiv_lincomb_adaptive", "axpby", "phiv_noalloc", "arnoldi", "matvec", "expm_phi", "workspace_bytes", "read_stats",
           "selftest_barrier_timeout", "max_m", "LsaError", "Workspace", "Batch", "phiv_batched",
           "phiv_vjp", "Phi1GrayScott"]


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Operator:
    """Operator descriptor; keeps the device field tensors alive."""

    def __init__(self, kind, nx, ny, nz, dx, diff=0.0, diff2=0.0, vel=(0.0, 0.0, 0.0), F=0.0,
                 k=0.0, field0=None, field1=None, aux=0):
        self.kind = kind
        self.args = dict(nx=nx, ny=ny, nz=nz, dx=dx, diff=diff, diff2=diff2, vel=vel, F=F, k=k,
                         field0=field0, field1=field1, aux=aux)
        self.fields = [f for f in (field0, field1) if f is not None]
        for f in self.fields:
            if f.dtype != torch.float64 or not f.is_cuda or not f.is_contiguous():
                raise ValueError("operator fields must be contiguous float64 CUDA tensors")
        v = (list(vel) + [0.0, 0.0, 0.0])[:3]
        self.c = LsaOp(KINDS[kind], int(nx), int(ny), int(nz), float(dx), float(diff),
                       float(diff2), (ctypes.c_double * 3)(*v), float(F), float(k),
                       ctypes.c_void_p(field0.data_ptr() if field0 is not None else None),
                       ctypes.c_void_p(field1.data_ptr() if field1 is not None else None), int(aux))

    def derived(self, kind=None, aux=0, **changes):
        """A descriptor of another kind (e.g. the transpose) or with changed
        coefficients, sharing the field tensors."""
        args = dict(self.args, aux=aux)
        args.update(changes)
        return Operator(kind or self.kind, **args)

    @property
    def N(self) -> int:
        n = B.lib().lsa_op_dof(ctypes.byref(self.c))
        if n < 0:
            raise LsaError(B.LSA_ERR_ARG, "invalid operator")
        return int(n)

    @classmethod
    def advdiff2d(cls, nx, ny, dx, diff, vel):
        return cls("advdiff2d", nx, ny, 1, dx, diff=diff, vel=vel)

    @classmethod
    def grayscott2d(cls, nx, ny, dx, Du, Dv, F, k, u0, v0):
        return cls("grayscott2d", nx, ny, 1, dx, diff=Du, diff2=Dv, F=F, k=k, field0=u0, field1=v0)

    @classmethod
    def adr3d(cls, nx, ny, nz, dx, eps, vel, r):
        return cls("adr3d", nx, ny, nz, dx, diff=eps, vel=vel, field0=r)

    @classmethod
    def from_workload(cls, cfg, fields):
        """Build from a workload dict and a dict of float64 CUDA field tensors."""
        kind = cfg["kind"]
        if kind == "advdiff2d":
            return cls.advdiff2d(cfg["nx"], cfg["ny"], cfg["dx"], cfg["diff"], cfg["vel"])
        if kind == "grayscott2d":
            return cls.grayscott2d(cfg["nx"], cfg["ny"], cfg["dx"], cfg["diff"], cfg["diff2"],
                                   cfg["F"], cfg["k"], fields["u0"], fields["v0"])
        if kind == "adr3d":
            return cls.adr3d(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["diff"], cfg["vel"],
                             fields["r"])
        raise ValueError(kind)


def max_m() -> int:
    return int(B.lib().lsa_max_m())


def workspace_bytes(op: Operator, m: int, p: int = 0, precision: str = "fp64") -> int:
    n = B.lib().lsa_workspace_bytes(ctypes.byref(op.c), int(m), int(p), PRECISIONS[precision])
    if n == 0:
        raise LsaError(B.LSA_ERR_ARG, "lsa_workspace_bytes")
    return int(n)


class Workspace:
    """A 256-byte aligned device buffer (torch-allocated)."""

    def __init__(self, nbytes: int, device="cuda"):
        self.nbytes = int(nbytes)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = self.buf.data_ptr() + off

    @classmethod
    def for_call(cls, op, m, p=0, precision="fp64"):
        return cls(workspace_bytes(op, m, p, precision))


def _check(st, what, ok=(B.LSA_OK, B.LSA_BREAKDOWN, B.LSA_NOT_CONVERGED)):
    if st not in ok:
        raise LsaError(st, what)
    return st


def _basis_dtype(precision):
    return torch.float64 if precision == "fp64" else torch.float32


def matvec(op: Operator, x: torch.Tensor, precision="fp64", y=None, work=None, stream=None):
    dt = _basis_dtype(precision)
    if x.dtype != dt or not x.is_cuda:
        raise ValueError(f"x must be a CUDA tensor of {dt}")
    y = torch.empty_like(x) if y is None else y
    work = work or Workspace.for_call(op, 1, 0, precision)
    st = B.lib().lsa_matvec(ctypes.byref(op.c), _ptr(x), _ptr(y), PRECISIONS[precision],
                            ctypes.c_void_p(work.ptr), work.nbytes, _stream_ptr(stream))
    _check(st, "lsa_matvec", ok=(B.LSA_OK,))
    return y


def arnoldi(op: Operator, v: torch.Tensor, m: int, variant="hcwy", precision="fp64", work=None,
            stream=None, stats=True):
    """Returns (V, H, stats): V is N x (m+1) (column j = v_{j+1}), H is (m+1) x m."""
    N = op.N
    dt = _basis_dtype(precision)
    V = torch.empty((m + 1, N), dtype=dt, device=v.device)        # column-major N x (m+1)
    H = torch.empty((m, m + 1), dtype=torch.float64, device=v.device)  # column-major (m+1) x m
    work = work or Workspace.for_call(op, m, 0, precision)
    s = LsaStats()
    st = B.lib().lsa_arnoldi(ctypes.byref(op.c), _ptr(v), int(m), VARIANTS[variant],
                             PRECISIONS[precision], _ptr(V), _ptr(H), ctypes.c_void_p(work.ptr),
                             work.nbytes, ctypes.byref(s) if stats else None, _stream_ptr(stream))
    _check(st, "lsa_arnoldi")
    return V.T, H.T, (s.as_dict() if stats else None)


def _check_vector_and_output(v: torch.Tensor, p: int, y):
    """v: contiguous float64 on the current CUDA device (the library launches on
    the current device); y, when given, a contiguous float64 (p+1, N) tensor on
    the same device.  Returns y (allocated when None)."""
    if v.dtype != torch.float64 or not v.is_cuda or not v.is_contiguous():
        raise ValueError("v must be a contiguous float64 CUDA tensor")
    if v.device.index != torch.cuda.current_device():
        raise ValueError(f"v is on {v.device}, but cuda:{torch.cuda.current_device()} is the current device")
    N = v.numel()
    if y is None:
        return torch.empty((p + 1, N), dtype=torch.float64, device=v.device)
    if (y.dtype != torch.float64 or y.device != v.device or not y.is_contiguous()
            or tuple(y.shape) != (p + 1, N)):
        raise ValueError(f"y must be a contiguous float64 ({p + 1}, {N}) tensor on {v.device}")
    return y


def phiv(op: Operator, v: torch.Tensor, h: float, p: int, m: int, tol: float = 0.0,
         variant="hcwy", precision="fp64", y=None, work=None, stream=None, stats=True):
    """y[k] = phi_k(h A) v for k = 0..p; returns (y, stats dict or None)."""
    y = _check_vector_and_output(v, p, y)
    N = v.numel()
    work = work or Workspace.for_call(op, min(m, N), p, precision)
    s = LsaStats()
    st = B.lib().lsa_phiv(ctypes.byref(op.c), _ptr(v), float(h), int(p), int(m), float(tol),
                          VARIANTS[variant], PRECISIONS[precision], _ptr(y),
                          ctypes.c_void_p(work.ptr), work.nbytes,
                          ctypes.byref(s) if stats else None, _stream_ptr(stream))
    _check(st, "lsa_phiv")
    return y, (s.as_dict() if stats else None)


def phiv_host(op: Operator, v_host: torch.Tensor, h: float, p: int, m: int, y_host: torch.Tensor,
              v_dev: torch.Tensor, y_dev: torch.Tensor, tol: float = 0.0, variant="hcwy", precision="fp64",
              work=None, stream=None):
    """phiv from and to host memory (lsa_phiv_host): v_host (N,) and y_host (p+1, N)
    float64 CPU tensors (pinned for overlap), v_dev and y_dev device staging
    tensors of the same shapes.  Enqueues H2D, the phi product and D2H on the
    stream; returns the status (synchronise before reading y_host)."""
    for t_, name, dev in ((v_host, "v_host", False), (y_host, "y_host", False), (v_dev, "v_dev", True),
                          (y_dev, "y_dev", True)):
        if t_.dtype != torch.float64 or not t_.is_contiguous() or t_.is_cuda != dev:
            raise ValueError(f"{name} must be a contiguous float64 {'CUDA' if dev else 'CPU'} tensor")
    N = v_host.numel()
    if v_dev.numel() != N or y_host.numel() != (p + 1) * N or y_dev.numel() != (p + 1) * N:
        raise ValueError("v and y buffers must hold N and (p+1) N values")
    work = work or Workspace.for_call(op, min(m, N), p, precision)
    st = B.lib().lsa_phiv_host(ctypes.byref(op.c), ctypes.c_void_p(v_host.data_ptr()), float(h), int(p), int(m),
                               float(tol), VARIANTS[variant], PRECISIONS[precision],
                               ctypes.c_void_p(y_host.data_ptr()), _ptr(v_dev), _ptr(y_dev),
                               ctypes.c_void_p(work.ptr), work.nbytes, _stream_ptr(stream))
    return _check(st, "lsa_phiv_host")


def tune_step(op: Operator, v: torch.Tensor, m: int, variant="hcwy", precision="fp64", reps: int = 3,
              work=None, stream=None):
    """Times the step forms of the grid Arnoldi kernel's hybrid variants (0
    one-pass; 1 two-phase, its second pass over tiles; 2 flat two-phase, on
    the ADR 3D, advection-diffusion and Gray-Scott operators) on (op, m,
    variant, precision) (lsa_tune_step) and records the fastest for later
    calls with that shape.  Returns (form, ms of form 0, ms of the fastest
    two-phase form); (0, 0.0, 0.0) when the forms do not apply."""
    if v.dtype != torch.float64 or not v.is_cuda or not v.is_contiguous() or v.numel() != op.N:
        raise ValueError("v must be a contiguous float64 CUDA tensor of N values")
    m = min(int(m), op.N)
    work = work or Workspace.for_call(op, m, 0, precision)
    two, a, b = ctypes.c_int(), ctypes.c_float(), ctypes.c_float()
    st = B.lib().lsa_tune_step(ctypes.byref(op.c), _ptr(v), m, VARIANTS[variant], PRECISIONS[precision],
                               ctypes.c_void_p(work.ptr), work.nbytes, int(reps), ctypes.byref(two),
                               ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream))
    _check(st, "lsa_tune_step", ok=(B.LSA_OK,))
    return two.value, a.value, b.value


def probe_fp64_fma_tflops(iters: int = 2000, reps: int = 10, device="cuda"):
    """Measured float64 FMA throughput (TFLOP/s, best of reps) of
    lsa_probe_fp64_fma, timed with CUDA events on the current stream."""
    out = torch.zeros(1, dtype=torch.float64, device=device)
    flops = ctypes.c_double(0.0)
    stream = torch.cuda.current_stream()
    best = 0.0
    for r in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _check(B.lib().lsa_probe_fp64_fma(int(iters), _ptr(out), ctypes.byref(flops), _stream_ptr(None)),
               "lsa_probe_fp64_fma", ok=(B.LSA_OK,))
        b.record(stream)
        b.synchronize()
        if r > 0:                      # the first launch is a warm-up
            best = max(best, flops.value / (a.elapsed_time(b) / 1e3) / 1e12)
    return best


def phiv_lincomb(op: Operator, b: torch.Tensor, tau: float, m: int, nsub: int = 1, tol: float = 0.0,
                 variant="hcwy", u=None, work=None, stream=None, stats=True):
    """u = sum_j tau^j phi_j(tau A) b[j] (b: (p+1, N) float64 CUDA tensor) by Krylov
    projection of the augmented operator in nsub equal sub-steps, each of
    dimension m; returns (u, stats dict or None)."""
    if b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous() or b.dim() != 2:
        raise ValueError("b must be a contiguous (p+1, N) float64 CUDA tensor")
    p = b.shape[0] - 1
    N = b.shape[1]
    u = torch.empty(N, dtype=torch.float64, device=b.device) if u is None else u
    work = work or Workspace.for_call(op, min(m, N + p), 0, "fp64")
    s = LsaStats()
    st = B.lib().lsa_phiv_lincomb(ctypes.byref(op.c), _ptr(b), int(p), float(tau), int(nsub), int(m),
                                  float(tol), VARIANTS[variant], PRECISIONS["fp64"], _ptr(u),
                                  ctypes.c_void_p(work.ptr), work.nbytes,
                                  ctypes.byref(s) if stats else None, _stream_ptr(stream))
    _check(st, "lsa_phiv_lincomb")
    return u, (s.as_dict() if stats else None)


def phiv_lincomb_adaptive(op: Operator, b: torch.Tensor, tau: float, m: int, tol: float, nsub0: int = 1,
                          max_substeps: int = 10000, variant="hcwy", u=None, work=None, stream=None):
    """phiv_lincomb with sub-steps chosen by the a-posteriori estimate of each
    projection (lsa_phiv_lincomb_adaptive); returns (u, stats dict with the
    accepted and rejected sub-step counts)."""
    if b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous() or b.dim() != 2:
        raise ValueError("b must be a contiguous (p+1, N) float64 CUDA tensor")
    p = b.shape[0] - 1
    N = b.shape[1]
    u = torch.empty(N, dtype=torch.float64, device=b.device) if u is None else u
    scratch = torch.empty(N, dtype=torch.float64, device=b.device)
    work = work or Workspace.for_call(op, min(m, N + p), 0, "fp64")
    s = LsaStats()
    nacc, nrej = ctypes.c_int(0), ctypes.c_int(0)
    st = B.lib().lsa_phiv_lincomb_adaptive(ctypes.byref(op.c), _ptr(b), int(p), float(tau), float(tol),
                                           int(m), int(nsub0), int(max_substeps), VARIANTS[variant],
                                           PRECISIONS["fp64"], _ptr(u), _ptr(scratch),
                                           ctypes.c_void_p(work.ptr), work.nbytes, ctypes.byref(s),
                                           ctypes.byref(nacc), ctypes.byref(nrej), _stream_ptr(stream))
    _check(st, "lsa_phiv_lincomb_adaptive")
    d = s.as_dict()
    d.update(substeps=nacc.value, rejected=nrej.value)
    return u, d


def phiv_lincomb_adaptive_m(op: Operator, b: torch.Tensor, tau: float, m0: int, tol: float, m_min: int = 4,
                            m_max: int = 64, nsub0: int = 1, max_substeps: int = 10000, variant="hcwy",
                            u=None, work=None, stream=None):
    """phiv_lincomb with the size and the Krylov dimension of every sub-step
    adaptive (lsa_phiv_lincomb_adaptive_m); returns (u, stats dict with the
    accepted and rejected sub-step counts and the dimension of each accepted one)."""
    if b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous() or b.dim() != 2:
        raise ValueError("b must be a contiguous (p+1, N) float64 CUDA tensor")
    p = b.shape[0] - 1
    N = b.shape[1]
    u = torch.empty(N, dtype=torch.float64, device=b.device) if u is None else u
    scratch = torch.empty(N, dtype=torch.float64, device=b.device)
    if work is None:
        nbytes = B.lib().lsa_lincomb_adaptive_m_workspace_bytes(ctypes.byref(op.c), int(m_max))
        if nbytes == 0:
            raise LsaError(B.LSA_ERR_ARG, "lsa_lincomb_adaptive_m_workspace_bytes")
        work = Workspace(nbytes, device=b.device)
    s = LsaStats()
    nacc, nrej = ctypes.c_int(0), ctypes.c_int(0)
    cap = int(max_substeps)
    dims = (ctypes.c_int * cap)()
    st = B.lib().lsa_phiv_lincomb_adaptive_m(ctypes.byref(op.c), _ptr(b), int(p), float(tau), float(tol),
                                             int(m0), int(m_min), int(m_max), int(nsub0), cap,
                                             VARIANTS[variant], _ptr(u), _ptr(scratch),
                                             ctypes.c_void_p(work.ptr), work.nbytes, ctypes.byref(s),
                                             ctypes.byref(nacc), ctypes.byref(nrej), dims, cap,
                                             _stream_ptr(stream))
    _check(st, "lsa_phiv_lincomb_adaptive_m")
    d = s.as_dict()
    d.update(substeps=nacc.value, rejected=nrej.value, dims=list(dims[:min(nacc.value, cap)]))
    return u, d


def axpby(a: float, x: torch.Tensor, b: float, y: torch.Tensor, out=None, stream=None):
    """out = a x + b y over float64 CUDA tensors of one size (lsa_axpby)."""
    for t_, name in ((x, "x"), (y, "y")):
        if t_.dtype != torch.float64 or not t_.is_cuda or not t_.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if x.numel() != y.numel():
        raise ValueError("x and y must have the same size")
    out = torch.empty_like(x) if out is None else out
    _check(B.lib().lsa_axpby(x.numel(), float(a), _ptr(x), float(b), _ptr(y), _ptr(out),
                             _stream_ptr(stream)), "lsa_axpby", ok=(B.LSA_OK,))
    return out


def phiv_noalloc(op: Operator, v: torch.Tensor, h: float, p: int, m: int, tol: float = 0.0,
                 variant="hcwy", precision="fp64", y=None, stream=None, stats=True):
    """phiv through lsa_phiv_noalloc: the library's fixed static device workspace
    is used instead of a caller-provided one (for callers that cannot allocate)."""
    y = _check_vector_and_output(v, p, y)
    s = LsaStats()
    st = B.lib().lsa_phiv_noalloc(ctypes.byref(op.c), _ptr(v), float(h), int(p), int(m), float(tol),
                                  VARIANTS[variant], PRECISIONS[precision], _ptr(y),
                                  ctypes.byref(s) if stats else None, _stream_ptr(stream))
    _check(st, "lsa_phiv_noalloc")
    return y, (s.as_dict() if stats else None)


def expm_phi(H: torch.Tensor, m: int, h: float, p: int, stream=None):
    """C (p+2, m): row k = phi_k(h H_m) e_1 from one exponential of the augmented matrix.
    H: float64 CUDA tensor holding H_m in its leading m x m block (row-major torch
    view of a column-major matrix is handled here)."""
    Hc = H[:m, :m].T.contiguous()        # column-major storage, ldh = m
    C = torch.empty((p + 2, m), dtype=torch.float64, device=H.device)
    work = Workspace(1 << 20, device=H.device)
    st = B.lib().lsa_expm_phi(_ptr(Hc), int(m), int(m), float(h), int(p), _ptr(C),
                              ctypes.c_void_p(work.ptr), work.nbytes, _stream_ptr(stream))
    _check(st, "lsa_expm_phi", ok=(B.LSA_OK,))
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return C


def read_stats(work: Workspace, stream=None):
    s = LsaStats()
    st = B.lib().lsa_read_stats(ctypes.c_void_p(work.ptr), ctypes.byref(s), _stream_ptr(stream))
    return st, s.as_dict()


def selftest_barrier_timeout(seconds: float = 0.5, stream=None) -> int:
    work = Workspace(1 << 16)
    return int(B.lib().lsa_selftest_barrier_timeout(ctypes.c_void_p(work.ptr), work.nbytes,
                                                    float(seconds), _stream_ptr(stream)))


def _op_array(ops):
    arr = (LsaOp * len(ops))()
    for i, op in enumerate(ops):
        arr[i] = op.c
    return arr


class Batch:
    """A plan for many independent phi products in one persistent launch
    (lsa_batch_* entry points).  Inputs and outputs are packed: v is the
    concatenation of the N_i-vectors, y of the (p+1) x N_i outputs; `voff` and
    `yoff` give each instance's element offset."""

    def __init__(self, ops, m, h, p, tol=0.0, variant="hcwy", precision="fp64", stream=None):
        self.ops = list(ops)               # keeps the operators' field tensors alive
        self.count = len(self.ops)
        self.p = int(p)
        self._ops_c = _op_array(self.ops)
        self._m_c = (ctypes.c_int * self.count)(*[int(x) for x in m])
        nb = B.lib().lsa_batch_workspace_bytes(self._ops_c, self._m_c, self.count, self.p,
                                               PRECISIONS[precision])
        if nb == 0:
            raise LsaError(B.LSA_ERR_ARG, "lsa_batch_workspace_bytes")
        self.work = Workspace(nb)
        h_ = ctypes.c_void_p()
        st = B.lib().lsa_batch_create(self._ops_c, self._m_c, self.count, float(h), self.p,
                                      float(tol), VARIANTS[variant], PRECISIONS[precision],
                                      ctypes.c_void_p(self.work.ptr), self.work.nbytes,
                                      ctypes.byref(h_), _stream_ptr(stream))
        _check(st, "lsa_batch_create", ok=(B.LSA_OK,))
        self._h = h_
        ctas, gs, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nv, ny = ctypes.c_longlong(), ctypes.c_longlong()
        vo = (ctypes.c_longlong * self.count)()
        yo = (ctypes.c_longlong * self.count)()
        _check(B.lib().lsa_batch_info(self._h, ctypes.byref(ctas), ctypes.byref(gs), ctypes.byref(nl),
                                      ctypes.byref(nv), ctypes.byref(ny), vo, yo), "lsa_batch_info",
               ok=(B.LSA_OK,))
        self.ctas = ctas.value
        self.v_elems, self.y_elems = nv.value, ny.value
        self.voff, self.yoff = list(vo), list(yo)

    @property
    def tiling(self):
        gs, nl = ctypes.c_int(), ctypes.c_int()
        B.lib().lsa_batch_info(self._h, None, ctypes.byref(gs), ctypes.byref(nl), None, None, None, None)
        return gs.value, nl.value

    def set_tiling(self, group_size: int, nlarge: int):
        _check(B.lib().lsa_batch_set_tiling(self._h, int(group_size), int(nlarge)),
               "lsa_batch_set_tiling", ok=(B.LSA_OK,))

    @property
    def step_form(self):
        """1 when the plan runs the two-phase hybrid step, 0 for the one-pass step."""
        return int(B.lib().lsa_batch_step_form(self._h))

    def set_step_form(self, two_phase: int):
        _check(B.lib().lsa_batch_set_step_form(self._h, int(two_phase)), "lsa_batch_set_step_form",
               ok=(B.LSA_OK,))

    def _check_v(self, v, y):
        if v.dtype != torch.float64 or not v.is_cuda or not v.is_contiguous() or v.numel() != self.v_elems:
            raise ValueError("v must be a contiguous float64 CUDA tensor of the packed size")
        if y is None:
            y = torch.empty(self.y_elems, dtype=torch.float64, device=v.device)
        elif y.dtype != torch.float64 or not y.is_contiguous() or y.numel() != self.y_elems:
            raise ValueError("y must be a contiguous float64 CUDA tensor of the packed size")
        return y

    def run(self, v, y=None, graph=True, stream=None):
        """Enqueue one evaluation (no synchronisation); returns y."""
        y = self._check_v(v, y)
        st = B.lib().lsa_batch_run(self._h, _ptr(v), _ptr(y), 1 if graph else 0, _stream_ptr(stream))
        _check(st, "lsa_batch_run", ok=(B.LSA_OK,))
        return y

    def tune(self, v, y=None, reps=2, stream=None):
        """Time candidate tilings on (v, y) and keep the fastest; returns
        (group_size, nlarge, ms)."""
        y = self._check_v(v, y)
        gs, nl, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        st = B.lib().lsa_batch_tune(self._h, _ptr(v), _ptr(y), int(reps), ctypes.byref(gs),
                                    ctypes.byref(nl), ctypes.byref(ms), _stream_ptr(stream))
        _check(st, "lsa_batch_tune")
        return gs.value, nl.value, ms.value

    def stats(self, stream=None):
        """(status, finished, [per-instance stats dicts]) of the last run."""
        arr = (LsaStats * self.count)()
        fin = ctypes.c_int()
        st = B.lib().lsa_batch_read_stats(self._h, arr, ctypes.byref(fin), _stream_ptr(stream))
        return int(st), fin.value, [a.as_dict() for a in arr]

    def split(self, y):
        """Per-instance (p+1, N_i) views of a packed output."""
        out = []
        for i, op in enumerate(self.ops):
            n = op.N
            out.append(y[self.yoff[i]:self.yoff[i] + (self.p + 1) * n].view(self.p + 1, n))
        return out

    def close(self):
        if getattr(self, "_h", None):
            B.lib().lsa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def phiv_batched(ops, v, h, p, m, tol=0.0, variant="hcwy", precision="fp64", stream=None):
    """One-shot batched call (lsa_phiv_batched, default tiling, no graph).
    v packed as in Batch; returns (y packed, status, per-instance stats)."""
    ops = list(ops)
    n = len(ops)
    ops_c = _op_array(ops)
    m_c = (ctypes.c_int * n)(*[int(x) for x in m])
    nb = B.lib().lsa_batch_workspace_bytes(ops_c, m_c, n, int(p), PRECISIONS[precision])
    if nb == 0:
        raise LsaError(B.LSA_ERR_ARG, "lsa_batch_workspace_bytes")
    work = Workspace(nb)
    ny = sum((int(p) + 1) * op.N for op in ops)
    y = torch.empty(ny, dtype=torch.float64, device=v.device)
    arr = (LsaStats * n)()
    st = B.lib().lsa_phiv_batched(ops_c, m_c, n, _ptr(v), float(h), int(p), float(tol),
                                  VARIANTS[variant], PRECISIONS[precision], _ptr(y),
                                  ctypes.c_void_p(work.ptr), work.nbytes, arr, _stream_ptr(stream))
    _check(st, "lsa_phiv_batched")
    return y, int(st), [a.as_dict() for a in arr]


# ---------------------------------------------------------------------------
# Gradients of the phi_1 product on the Gray-Scott Jacobian

def vjp_workspace_bytes(op: Operator, m: int) -> int:
    n = B.lib().lsa_phiv_vjp_workspace_bytes(ctypes.byref(op.c), int(m))
    if n == 0:
        raise LsaError(B.LSA_ERR_ARG, "lsa_phiv_vjp_workspace_bytes")
    return int(n)


def phiv_vjp(op: Operator, v: torch.Tensor, h: float, m: int, r: torch.Tensor, y: torch.Tensor,
             variant="hcwy", work=None, stream=None, stats=False):
    """Vector-Jacobian product of y1 = phi_1(h A(theta)) v (Gray-Scott, float64)
    for the cotangent r: returns (dL/dv, tensor of dL/dh, dL/dDu, dL/dDv, dL/dF,
    dL/dk on the device, stats or None).  y is the (3, N) output of
    phiv(op, v, h, p=2, m) -- the phi_0, phi_1 and phi_2 products."""
    N = v.numel()
    for t, name in ((v, "v"), (r, "r"), (y, "y")):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if r.numel() != N or y.numel() != 3 * N:
        raise ValueError("r must have N elements and y 3N (phiv with p = 2)")
    grad_v = torch.empty_like(v)
    grad_s = torch.empty(5, dtype=torch.float64, device=v.device)
    work = work or Workspace(vjp_workspace_bytes(op, m), device=v.device)
    s = LsaStats()
    st = B.lib().lsa_phiv_vjp(ctypes.byref(op.c), _ptr(v), float(h), int(m), VARIANTS[variant], _ptr(r),
                              _ptr(y), _ptr(grad_v), _ptr(grad_s), ctypes.c_void_p(work.ptr), work.nbytes,
                              ctypes.byref(s) if stats else None, _stream_ptr(stream))
    _check(st, "lsa_phiv_vjp")
    return grad_v, grad_s, (s.as_dict() if stats else None)


class Phi1GrayScott(torch.autograd.Function):
    """y = phi_1(h A(theta)) v for the Gray-Scott Jacobian A(theta), theta =
    (Du, Dv, F, k), differentiable in v (CUDA float64), h and theta (CPU
    float64 tensors).  The forward keeps v, h, theta and the phi_0 / phi_1 /
    phi_2 products; the backward recomputes every Krylov basis it needs through
    lsa_phiv_vjp (no basis is stored).

        y = Phi1GrayScott.apply(v, h, theta, op, m, variant)

    op supplies the grid, spacing and fields (its own coefficients are replaced
    by theta)."""

    @staticmethod
    def forward(ctx, v, h, theta, op, m, variant="hcwy"):
        hh = float(h)
        Du, Dv, F, k = (float(t) for t in theta)
        opt = op.derived(kind="grayscott2d", diff=Du, diff2=Dv, F=F, k=k)
        y, _ = phiv(opt, v.contiguous(), hh, 2, m, variant=variant, stats=False)
        ctx.save_for_backward(v, y)
        ctx.opt, ctx.h, ctx.m, ctx.variant = opt, hh, m, variant
        ctx.theta_dev = theta.device
        return y[1].clone()

    @staticmethod
    def backward(ctx, g):
        v, y = ctx.saved_tensors
        gv, gs, _ = phiv_vjp(ctx.opt, v, ctx.h, ctx.m, g.contiguous(), y, variant=ctx.variant)
        gs = gs.to(ctx.theta_dev)
        return gv, gs[0], gs[1:5], None, None, None
