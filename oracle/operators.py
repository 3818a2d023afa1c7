"""Sparse-matrix forms of the synthetic stencil operators (oracle side).

The paper applies its Jacobians matrix-free (Sect. 2.1: only products J v are
needed).  The oracle instead assembles each operator as a scipy.sparse matrix
from Kronecker products of periodic 1D difference matrices, so that it shares
no code path with the CUDA stencils.  Grid index: i = ix + nx*(iy + ny*iz),
x fastest; Gray-Scott stacks the species as [u-block; v-block].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _periodic_1d(n: int, taps) -> sp.csr_matrix:
    """n x n periodic matrix with (M v)_i = sum_(off, val) val * v_{(i+off) mod n}.
    Coinciding offsets (n <= 2) add up, as the periodic stencil requires."""
    rows = np.arange(n)
    M = sp.csr_matrix((n, n))
    for off, val in taps:
        M = M + sp.csr_matrix((np.full(n, float(val)), (rows, (rows + off) % n)), shape=(n, n))
    return M.tocsr()


def second_difference(n: int, dx: float) -> sp.csr_matrix:
    """(v_{i-1} - 2 v_i + v_{i+1}) / dx^2, periodic."""
    return _periodic_1d(n, [(-1, 1.0), (0, -2.0), (1, 1.0)]) / dx**2


def central_difference(n: int, dx: float) -> sp.csr_matrix:
    """(v_{i+1} - v_{i-1}) / (2 dx), periodic."""
    return _periodic_1d(n, [(1, 1.0), (-1, -1.0)]) / (2.0 * dx)


def upwind_difference(n: int, dx: float, vel: float) -> sp.csr_matrix:
    """First-order upwind approximation of d/dx for advection speed ``vel``:
    backward (v_i - v_{i-1})/dx when vel >= 0, forward (v_{i+1} - v_i)/dx otherwise."""
    if vel >= 0:
        return _periodic_1d(n, [(0, 1.0), (-1, -1.0)]) / dx
    return _periodic_1d(n, [(1, 1.0), (0, -1.0)]) / dx


def _axis_ops(shape, ops):
    """Sum over axes of (I x ... x op_axis x ... x I) for index x-fastest.

    shape = (nx, ny[, nz]); ops = per-axis 1D matrices (None to skip)."""
    dims = list(shape)
    total = None
    for a, op in enumerate(ops):
        if op is None:
            continue
        # Kronecker order: slowest axis first -> kron(I_z, kron(I_y, op_x)) etc.
        factors = []
        for b in reversed(range(len(dims))):
            factors.append(op if b == a else sp.identity(dims[b], format="csr"))
        K = factors[0]
        for f in factors[1:]:
            K = sp.kron(K, f, format="csr")
        total = K if total is None else total + K
    return total


def advdiff2d(nx: int, ny: int, dx: float, diff: float, vel) -> sp.csr_matrix:
    """A = diff * (D2x + D2y) - vel_x Dx - vel_y Dy (central), periodic 2D."""
    lap = _axis_ops((nx, ny), [second_difference(nx, dx), second_difference(ny, dx)])
    adv = _axis_ops((nx, ny), [vel[0] * central_difference(nx, dx),
                               vel[1] * central_difference(ny, dx)])
    return (diff * lap - adv).tocsr()


def grayscott2d(nx: int, ny: int, dx: float, Du: float, Dv: float, F: float, k: float,
                u0: np.ndarray, v0: np.ndarray) -> sp.csr_matrix:
    """Jacobian of the Gray-Scott right-hand side
         f_u = Du Lap u - u v^2 + F (1 - u),   f_v = Dv Lap v + u v^2 - (F + k) v
    at (u0, v0):  [[Du Lap - diag(v0^2) - F,  -diag(2 u0 v0)],
                   [diag(v0^2),  Dv Lap + diag(2 u0 v0) - (F + k)]]."""
    n = nx * ny
    lap = _axis_ops((nx, ny), [second_difference(nx, dx), second_difference(ny, dx)])
    I = sp.identity(n, format="csr")
    a = sp.diags(v0 * v0)
    b = sp.diags(2.0 * u0 * v0)
    J = sp.bmat([[Du * lap - a - F * I, -b],
                 [a, Dv * lap + b - (F + k) * I]], format="csr")
    return J


def adr3d(nx: int, ny: int, nz: int, dx: float, eps: float, vel, r: np.ndarray) -> sp.csr_matrix:
    """A = eps (D2x + D2y + D2z) - sum_a vel_a * Upwind_a + diag(r), periodic 3D."""
    shape = (nx, ny, nz)
    lap = _axis_ops(shape, [second_difference(n, dx) for n in shape])
    adv = _axis_ops(shape, [vel[a] * upwind_difference(shape[a], dx, vel[a]) for a in range(3)])
    return (eps * lap - adv + sp.diags(r)).tocsr()


def from_workload(cfg: dict, inputs: dict) -> sp.csr_matrix:
    """Assemble the operator of a workload dict (see the ``workloads`` module)."""
    kind = cfg["kind"]
    if kind == "advdiff2d":
        return advdiff2d(cfg["nx"], cfg["ny"], cfg["dx"], cfg["diff"], cfg["vel"])
    if kind == "grayscott2d":
        return grayscott2d(cfg["nx"], cfg["ny"], cfg["dx"], cfg["diff"], cfg["diff2"],
                           cfg["F"], cfg["k"], inputs["u0"], inputs["v0"])
    if kind == "adr3d":
        return adr3d(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["diff"], cfg["vel"],
                     inputs["r"])
    raise ValueError(kind)


def fourier_symbol_advdiff2d(nx, ny, dx, diff, vel):
    """Eigenvalues of the periodic advdiff2d operator on the Fourier modes
    exp(i(theta_x ix + theta_y iy)), theta = 2 pi k / n, arranged as a
    (ny, nx) array matching numpy.fft.fft2 of a (ny, nx)-shaped field."""
    tx = 2 * np.pi * np.fft.fftfreq(nx) ; ty = 2 * np.pi * np.fft.fftfreq(ny)
    TX, TY = np.meshgrid(tx, ty)  # shape (ny, nx)
    lam = diff * ((2 * np.cos(TX) - 2) + (2 * np.cos(TY) - 2)) / dx**2
    lam = lam - 1j * (vel[0] * np.sin(TX) + vel[1] * np.sin(TY)) / dx
    return lam


def fourier_symbol_adr3d(nx, ny, nz, dx, eps, vel, r_const=0.0):
    """Eigenvalues of the periodic adr3d operator with a constant reaction,
    as an (nz, ny, nx) array matching numpy.fft.fftn of an (nz, ny, nx) field."""
    thetas = [2 * np.pi * np.fft.fftfreq(n) for n in (nx, ny, nz)]
    TX, TY, TZ = np.meshgrid(thetas[0], thetas[1], thetas[2], indexing="xy")
    # meshgrid 'xy' for 3 inputs gives shape (ny, nx, nz); reorder to (nz, ny, nx)
    TX, TY, TZ = (np.transpose(T, (2, 0, 1)) for T in (TX, TY, TZ))
    lam = np.zeros(TX.shape, dtype=complex) + r_const
    for T, u in zip((TX, TY, TZ), vel):
        lam += eps * (2 * np.cos(T) - 2) / dx**2
        if u >= 0:
            lam -= u * (1 - np.exp(-1j * T)) / dx
        else:
            lam -= u * (np.exp(1j * T) - 1) / dx
    return lam
