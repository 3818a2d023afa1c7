"""Exponential integrators of Sect. 4 (SRERK3, EPI4, EPI5) for the Gray-Scott
system u' = F(u), on the GPU path.

Each phi-function combination of a stage or step is one call of
``lsa_phiv_lincomb`` (Sect. 2.1, Eqs. 7-9: sum_k tau^k phi_k(tau J_n) b_k),
the right-hand side is ``lsa_rhs``, Jacobian products are ``lsa_matvec`` on
the Gray-Scott operator at the current state (the descriptor borrows the
state tensor, so it is J_n at every step), and every vector update is
``lsa_axpby``.  This module only sequences those calls.

  SRERK3:  z_1 = u_n + phi_1(3/4 h J_n) 3/4 h f_n,
           u_{n+1} = u_n + phi_1(h J_n) h f_n + phi_3(h J_n) 32/9 h R_n(z_1);
  EPIk:    u_{n+1} = u_n + phi_1(h J_n) h f_n + sum_k phi_k(h J_n) v_k,
           v_k = sum_{i=1}^{P} alpha_{k,i} h R_n(u_{n-i}),
with R_n(z) = F(z) - f_n - J_n (z - u_n) (Sect. 2) and the A_4, A_5
coefficient matrices of Sect. 4.  The multistep methods take their first P
steps with SRERK3 (the paper does not say how they start).
"""
from __future__ import annotations

import ctypes

import torch

from . import _binding as B
from . import Operator, Workspace, _check, _ptr, _stream_ptr, phiv_lincomb

EPI_ALPHA = {
    4: ((0.0, 0.0),
        (-3.0 / 10.0, 3.0 / 40.0),
        (32.0 / 5.0, -11.0 / 10.0)),
    5: ((0.0, 0.0, 0.0),
        (-4.0 / 5.0, 2.0 / 5.0, -4.0 / 45.0),
        (12.0, -9.0 / 2.0, 8.0 / 9.0),
        (3.0, 0.0, -1.0 / 3.0)),
}


class GrayScottIntegrator:
    """State u = [u; v] (2*nx*ny float64 on the GPU) of the Gray-Scott system
    and the exponential integrators that advance it.  m, nsub and variant are
    those of every phi combination (Krylov dimension per sub-step, equal
    sub-steps, Gram-Schmidt variant)."""

    def __init__(self, nx, ny, dx, Du, Dv, F, k, state: torch.Tensor, m=30, nsub=1,
                 variant="hcwy", tol=0.0, stream=None, collect_stats=True):
        if state.dtype != torch.float64 or not state.is_cuda or state.numel() != 2 * nx * ny:
            raise ValueError("state must be a float64 CUDA tensor of 2*nx*ny entries")
        self.n = nx * ny
        self.N = 2 * self.n
        self.u = torch.empty(2 * nx * ny, dtype=torch.float64, device=state.device)
        _check(B.lib().lsa_axpby(self.u.numel(), 1.0, _ptr(state), 0.0, _ptr(state), _ptr(self.u),
                                 _stream_ptr(stream)), "lsa_axpby", ok=(B.LSA_OK,))
        self.op = Operator.grayscott2d(nx, ny, dx, Du, Dv, F, k, self.u[:self.n], self.u[self.n:])
        self.m, self.nsub, self.variant, self.tol, self.stream = m, nsub, variant, tol, stream
        self.work_lc = Workspace.for_call(self.op, min(m, self.N + 4), 0)
        self.work_mv = Workspace.for_call(self.op, 1, 0)
        self.hist = []          # u_{n-1}, u_{n-2}, ... of the multistep methods
        self.collect_stats = collect_stats    # False: no per-call synchronisation
        self.stats = dict(lincomb_calls=0, grid_syncs=0, steps=0, launches=0)
        dev = self.u.device
        self._b = torch.empty((5, self.N), dtype=torch.float64, device=dev)
        self._t = [torch.empty(self.N, dtype=torch.float64, device=dev) for _ in range(4)]
        self._zero = torch.zeros(self.N, dtype=torch.float64, device=dev)

    # -- kernels ------------------------------------------------------------
    def rhs(self, w, out):
        self.stats["launches"] += 1
        _check(B.lib().lsa_rhs(ctypes.byref(self.op.c), _ptr(w), _ptr(out), _stream_ptr(self.stream)),
               "lsa_rhs", ok=(B.LSA_OK,))
        return out

    def axpby(self, a, x, b, y, out):
        self.stats["launches"] += 1
        _check(B.lib().lsa_axpby(self.N, float(a), _ptr(x), float(b), _ptr(y), _ptr(out),
                                 _stream_ptr(self.stream)), "lsa_axpby", ok=(B.LSA_OK,))
        return out

    def jv(self, x, out):
        self.stats["launches"] += 2          # operator set-up and the stencil
        _check(B.lib().lsa_matvec(ctypes.byref(self.op.c), _ptr(x), _ptr(out), B.PRECISIONS["fp64"],
                                  ctypes.c_void_p(self.work_mv.ptr), self.work_mv.nbytes,
                                  _stream_ptr(self.stream)), "lsa_matvec", ok=(B.LSA_OK,))
        return out

    def remainder(self, z, f, out):
        """out = R_n(z) = F(z) - f_n - J_n (z - u_n)."""
        d, jd = self._t[2], self._t[3]
        self.axpby(1.0, z, -1.0, self.u, d)
        self.jv(d, jd)
        self.rhs(z, out)
        self.axpby(1.0, out, -1.0, f, out)
        return self.axpby(1.0, out, -1.0, jd, out)

    def combo(self, cs, h, out):
        """out = sum_k phi_k(h J_n) c_k for cs = [(k, [(coef, vector), ...]), ...]
        (k >= 1), as one linear combination with b_0 = 0 and b_k = c_k / h^k."""
        p = max(k for k, _ in cs)
        b = self._b[:p + 1]
        for k in range(p + 1):
            self.axpby(0.0, self._zero, 0.0, self._zero, b[k])
        for k, terms in cs:
            for coef, vec in terms:
                self.axpby(1.0, b[k], coef / h ** k, vec, b[k])
        _, st = phiv_lincomb(self.op, b, h, self.m, self.nsub, self.tol, self.variant, u=out,
                             work=self.work_lc, stream=self.stream, stats=self.collect_stats)
        self.stats["lincomb_calls"] += 1
        self.stats["launches"] += 4 * self.nsub
        if st is not None:
            self.stats["grid_syncs"] += st["grid_syncs"]
        return out

    # -- methods ------------------------------------------------------------
    def copy(self, x):
        return self.axpby(1.0, x, 0.0, self._zero, torch.empty_like(x))

    def _advance(self, du):
        self.hist.insert(0, self.copy(self.u))
        del self.hist[max(len(a[0]) for a in EPI_ALPHA.values()):]
        self.axpby(1.0, self.u, 1.0, du, self.u)       # in place: the operator borrows u
        self.stats["steps"] += 1

    def step_srerk3(self, h):
        f = self.rhs(self.u, torch.empty_like(self.u))
        z1 = torch.empty_like(self.u)
        self.combo([(1, [(0.75 * h, f)])], 0.75 * h, z1)
        self.axpby(1.0, self.u, 1.0, z1, z1)
        r1 = self.remainder(z1, f, torch.empty_like(self.u))
        du = torch.empty_like(self.u)
        self.combo([(1, [(h, f)]), (3, [((32.0 / 9.0) * h, r1)])], h, du)
        self._advance(du)

    def step_epi(self, order, h):
        alpha = EPI_ALPHA[order]
        P = len(alpha[0])
        if len(self.hist) < P:
            return self.step_srerk3(h)
        f = self.rhs(self.u, torch.empty_like(self.u))
        R = [self.remainder(self.hist[i], f, torch.empty_like(self.u)) for i in range(P)]
        cs = [(1, [(h, f)])]
        for k in range(1, len(alpha) + 1):
            terms = [(alpha[k - 1][i] * h, R[i]) for i in range(P) if alpha[k - 1][i] != 0.0]
            if terms:
                cs.append((k, terms))
        du = torch.empty_like(self.u)
        self.combo(cs, h, du)
        self._advance(du)
        del self.hist[P:]

    def run(self, method: str, h: float, nsteps: int) -> torch.Tensor:
        """nsteps steps of 'srerk3', 'epi4' or 'epi5'; returns the state."""
        for _ in range(nsteps):
            if method == "srerk3":
                self.step_srerk3(h)
            elif method in ("epi4", "epi5"):
                self.step_epi(int(method[3:]), h)
            else:
                raise ValueError(method)
        return self.u
