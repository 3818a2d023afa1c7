"""Helpers for the GPU parity tests: device inputs from the seeded workloads,
oracle references (cached), and the comparison metrics."""
from __future__ import annotations

import functools

import numpy as np

import workloads as W
from oracle import arnoldi as OA
from oracle import krylov as OK
from oracle import operators as OP

FP64_TOL = 1e-10     # relative 2-norm error per phi_k, float64 form
FP32_TOL = 1e-5      # relative 2-norm error per phi_k, float32-basis form


def device_inputs(cfg, inp, torch, dev="cuda"):
    fields = {k: torch.from_numpy(v).to(dev) for k, v in inp.items() if k != "v"}
    v = torch.from_numpy(inp["v"]).to(dev)
    return v, fields


@functools.lru_cache(maxsize=64)
def _cached(key):
    cfg, variant, m, p, h = key
    cfg = dict(cfg)
    cfg["vel"] = tuple(cfg["vel"])
    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    y, info = OK.phiv(lambda x: A @ x, inp["v"], h, p, m, variant)
    return y, info


def oracle_phiv(cfg, variant="mgs", m=None, p=None, h=None):
    m = cfg["m"] if m is None else m
    p = cfg["p"] if p is None else p
    h = cfg["h"] if h is None else h
    key = (tuple(sorted((k, v if not isinstance(v, list) else tuple(v)) for k, v in cfg.items())),
           variant, m, p, h)
    return _cached(key)


def norm_errors(y_gpu, y_ref):
    """Per phi_k: ||y_k - ref_k||_2 / ||ref_k||_2 (the normwise parity metric)."""
    y = y_gpu.detach().cpu().numpy() if hasattr(y_gpu, "detach") else np.asarray(y_gpu)
    return [float(np.linalg.norm(y[k] - y_ref[k]) / max(np.linalg.norm(y_ref[k]), 1e-300))
            for k in range(y_ref.shape[0])]


def elem_errors(y_gpu, y_ref):
    """Per phi_k: max_i |y_k[i] - ref_k[i]| / max_i |ref_k[i]| (element by
    element, so a few wrong points at a tile edge cannot hide under a small norm)."""
    y = y_gpu.detach().cpu().numpy() if hasattr(y_gpu, "detach") else np.asarray(y_gpu)
    return [float(np.max(np.abs(y[k] - y_ref[k])) / max(np.max(np.abs(y_ref[k])), 1e-300))
            for k in range(y_ref.shape[0])]


def rel_errors(y_gpu, y_ref):
    """Per phi_k, the larger of the normwise and the element-wise error: every
    parity assertion holds both to the same bound."""
    return [max(a, b) for a, b in zip(norm_errors(y_gpu, y_ref), elem_errors(y_gpu, y_ref))]


def expected_syncs(variant, m_eff, fallbacks=0):
    if variant == "mgs":
        return 1 + sum(j + 1 for j in range(1, m_eff + 1))
    if variant == "cgs2":
        return 1 + 3 * m_eff
    if variant == "iocgs":
        return 1 + 2 * m_eff
    return m_eff + 1 + fallbacks
