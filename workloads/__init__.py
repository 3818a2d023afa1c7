"""Seeded synthetic workloads for the phi-product hot path.

This module only *describes* workloads and draws their random inputs.  It holds
none of the method's arithmetic: no operator application, no orthogonalisation,
no exponential.  Both the CPU oracle (``oracle/``) and the CUDA path (through
the tests and ``bench.py``) take their inputs from here, so that the two sides
see identical bytes.

The paper's own experiments (Allen-Cahn, ADR and Burgers at 2000^2, shallow
water at ~8.3M DOF; Sect. 4) use applications whose code is not public.  These
synthetic stencil operators stand in for them: periodic 2D advection-diffusion,
the Jacobian of 2D Gray-Scott at a random state, and 3D advection-diffusion-
reaction (the ADR family of Sect. 4.2 lifted to 3D and made periodic).

Every workload is a plain dict.  Random draws use ``numpy.random.default_rng``
with the workload's seed, in the fixed order documented in ``make_inputs``.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20241014

# Operator kinds, shared names with the C header's lsa_op_kind enum values.
ADVDIFF2D = "advdiff2d"
GRAYSCOTT2D = "grayscott2d"
ADR3D = "adr3d"


def advdiff2d(n=64, *, ny=None, diff=0.01, vel=(1.0, 0.5), h=1e-2, p=3, m=30,
              seed=SEED_BASE + 0, name=None):
    """2D periodic advection-diffusion on an n x ny grid with spacing 1/n.

    A v = diff * Lap5 v - (vel_x Dx v + vel_y Dy v), central differences."""
    ny = n if ny is None else ny
    return dict(name=name or f"advdiff2d_{n}x{ny}", kind=ADVDIFF2D, nx=n, ny=ny, nz=1,
                dx=1.0 / n, diff=diff, diff2=0.0, vel=(float(vel[0]), float(vel[1]), 0.0),
                F=0.0, k=0.0, h=h, p=p, m=m, seed=seed)


def grayscott2d(n=512, *, Du=2e-5, Dv=1e-5, F=0.04, k=0.06, length=2.5, h=1.0, p=2, m=64,
                seed=SEED_BASE + 1, name=None):
    """Jacobian of 2D Gray-Scott at a random state (u0, v0) ~ U[0,1]^2, periodic,
    domain length 2.5 (spacing 2.5/n), N = 2 n^2 in species-major order."""
    return dict(name=name or f"grayscott2d_{n}", kind=GRAYSCOTT2D, nx=n, ny=n, nz=1,
                dx=length / n, diff=Du, diff2=Dv, vel=(0.0, 0.0, 0.0), F=F, k=k,
                h=h, p=p, m=m, seed=seed)


def adr3d(n=256, *, eps=1e-3, vel=(1.0, 1.0, 1.0), h=5e-3, p=1, m=40,
          seed=SEED_BASE + 2, name=None):
    """3D periodic advection-diffusion-reaction, n^3 grid with spacing 1/n:
    A v = eps Lap7 v - sum_a vel_a * (upwind difference along a) + r .* v,
    with the reaction field r ~ U[-1, 0]."""
    return dict(name=name or f"adr3d_{n}", kind=ADR3D, nx=n, ny=n, nz=n, dx=1.0 / n,
                diff=eps, diff2=0.0, vel=tuple(float(x) for x in vel), F=0.0, k=0.0,
                h=h, p=p, m=m, seed=seed)


# The five benchmark workloads, in the order the project's configuration list
# gives them.  Index i uses seed SEED_BASE + i.
def config(i: int) -> dict:
    if i == 0:
        return advdiff2d(64, name="advdiff2d_64")
    if i == 1:
        return grayscott2d(512, name="grayscott2d_512")
    if i == 2:
        return adr3d(256, name="adr3d_256")
    if i == 3:
        return batched_advdiff2d(512)
    if i == 4:
        return grayscott2d(256, m=48, p=1, seed=SEED_BASE + 4, name="adjoint_grayscott2d_256")
    raise IndexError(i)


def n_dof(cfg: dict) -> int:
    ns = 2 if cfg["kind"] == GRAYSCOTT2D else 1
    return ns * cfg["nx"] * cfg["ny"] * cfg["nz"]


def make_inputs(cfg: dict) -> dict:
    """Draw the random inputs of a workload (float64 numpy arrays).

    Draw order, from ``default_rng(cfg['seed'])``:
      advdiff2d:   v ~ U[-1,1]^N
      grayscott2d: u0 ~ U[0,1]^(nx*ny), v0 ~ U[0,1]^(nx*ny), v ~ U[-1,1]^N
      adr3d:       r ~ U[-1,0]^N, v ~ U[-1,1]^N
    """
    rng = np.random.default_rng(cfg["seed"])
    N = n_dof(cfg)
    out = {}
    kind = cfg["kind"]
    if kind == ADVDIFF2D:
        out["v"] = rng.uniform(-1.0, 1.0, N)
    elif kind == GRAYSCOTT2D:
        npts = cfg["nx"] * cfg["ny"]
        out["u0"] = rng.uniform(0.0, 1.0, npts)
        out["v0"] = rng.uniform(0.0, 1.0, npts)
        out["v"] = rng.uniform(-1.0, 1.0, N)
    elif kind == ADR3D:
        out["r"] = rng.uniform(-1.0, 0.0, N)
        out["v"] = rng.uniform(-1.0, 1.0, N)
    else:
        raise ValueError(kind)
    return out


def adjoint_inputs(cfg: dict) -> dict:
    """Inputs of the adjoint workload (a Gray-Scott configuration): those of
    ``make_inputs`` followed, from the same generator, by the target
    y_t ~ U[-1,1]^N of the loss 1/2 ||phi_1(hA)v - y_t||^2."""
    if cfg["kind"] != GRAYSCOTT2D:
        raise ValueError("the adjoint workload is a Gray-Scott configuration")
    rng = np.random.default_rng(cfg["seed"])
    npts = cfg["nx"] * cfg["ny"]
    out = {"u0": rng.uniform(0.0, 1.0, npts), "v0": rng.uniform(0.0, 1.0, npts)}
    out["v"] = rng.uniform(-1.0, 1.0, 2 * npts)
    out["y_target"] = rng.uniform(-1.0, 1.0, 2 * npts)
    return out


def lincomb_inputs(cfg: dict, p: int) -> dict:
    """Inputs of a phi-function linear combination sum_j tau^j phi_j(tau A) b_j:
    those of ``make_inputs`` (the operator's fields) and the vectors
    b_0..b_p ~ U[-1,1]^N as a (p+1, N) array from a second generator seeded
    with the configuration's seed + 7919."""
    out = make_inputs(cfg)
    rng = np.random.default_rng(cfg["seed"] + 7919)
    out["b"] = rng.uniform(-1.0, 1.0, (p + 1, n_dof(cfg)))
    return out


# ---------------------------------------------------------------------------
# Batched workload: 512 independent 2D advection-diffusion instances.

BATCH_SIDES = tuple(range(32, 257, 16))  # {32, 48, ..., 256}: 15 values


def batched_advdiff2d(count=512, *, seed=SEED_BASE + 3, vel=(1.0, 0.5), h=1e-2, p=2,
                      m_range=(16, 48), diff_range=(1e-4, 1e-1), sides=BATCH_SIDES):
    """Instance table of the batched workload: sides drawn uniformly from
    {32, 48, ..., 256}, diffusion log-uniform in [1e-4, 1e-1], m uniform in
    [16, 48].  Draw order from ``default_rng(seed)``: sides, diffusions, m's;
    then each instance's v ~ U[-1,1]^(side^2) from ``default_rng(seed + 1 + i)``.
    ``sides`` replaces the side set (smaller test batches)."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.array(sides), size=count)
    lo, hi = math.log(diff_range[0]), math.log(diff_range[1])
    diffs = np.exp(rng.uniform(lo, hi, size=count))
    ms = rng.integers(m_range[0], m_range[1] + 1, size=count)
    inst = [advdiff2d(int(s), diff=float(c), vel=vel, h=h, p=p, m=int(mm), seed=seed + 1 + i,
                      name=f"batch{i}_{int(s)}")
            for i, (s, c, mm) in enumerate(zip(sides, diffs, ms))]
    return dict(name=f"batched_advdiff2d_{count}", kind="batched", instances=inst, h=h, p=p)


def batched_inputs(bcfg: dict) -> list:
    """Start vectors of every instance of a batched workload (in order)."""
    return [make_inputs(c)["v"] for c in bcfg["instances"]]
