"""ctypes binding of liblsarnoldi (include/lsarnoldi.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; PyTorch only
provides device memory and the current stream.  Importing this module fails
loudly when the library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_longlong, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblsarnoldi.so")

LSA_OK, LSA_BREAKDOWN, LSA_NOT_CONVERGED = 0, 1, 2
LSA_ERR_ARG, LSA_ERR_CUDA, LSA_ERR_TIMEOUT, LSA_ERR_NUMERIC, LSA_ERR_WORKSPACE = -1, -2, -3, -4, -5

VARIANTS = {"mgs": 0, "cgs2": 1, "hcwy": 2, "hncwy": 3, "hgsmgs": 4, "iocgs": 5}
PRECISIONS = {"fp64": 0, "fp32": 1}
KINDS = {"advdiff2d": 1, "grayscott2d": 2, "adr3d": 3, "grayscott2d_t": 4, "grayscott2d_frechet": 5}


class LsaOp(ctypes.Structure):
    _fields_ = [("kind", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("dx", c_double), ("diff", c_double), ("diff2", c_double),
                ("vel", c_double * 3), ("F", c_double), ("k", c_double),
                ("field0", c_void_p), ("field1", c_void_p), ("aux", c_int)]


class LsaStats(ctypes.Structure):
    _fields_ = [("status", c_int), ("m_eff", c_int), ("breakdown", c_int),
                ("norm_fallbacks", c_int), ("grid_syncs", c_int), ("grid_barriers", c_int),
                ("beta", c_double), ("err_est", c_double), ("h_last", c_double),
                ("ms_arnoldi", ctypes.c_float), ("ms_expm", ctypes.c_float),
                ("ms_combine", ctypes.c_float), ("launches", c_int), ("arnoldi_kernel", c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


# name -> (restype, argtypes): the entry points of include/lsarnoldi.h
SIGNATURES = {
    "lsa_max_m": (c_int, []),
    "lsa_version": (c_int, []),
    "lsa_status_string": (c_char_p, [c_int]),
    "lsa_op_dof": (c_longlong, [POINTER(LsaOp)]),
    "lsa_workspace_bytes": (c_size_t, [POINTER(LsaOp), c_int, c_int, c_int]),
    "lsa_matvec": (c_int, [POINTER(LsaOp), c_void_p, c_void_p, c_int, c_void_p, c_size_t, c_void_p]),
    "lsa_arnoldi": (c_int, [POINTER(LsaOp), c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                            c_void_p, c_size_t, POINTER(LsaStats), c_void_p]),
    "lsa_phiv": (c_int, [POINTER(LsaOp), c_void_p, c_double, c_int, c_int, c_double, c_int, c_int,
                         c_void_p, c_void_p, c_size_t, POINTER(LsaStats), c_void_p]),
    "lsa_phiv_lincomb": (c_int, [POINTER(LsaOp), c_void_p, c_int, c_double, c_int, c_int, c_double,
                                 c_int, c_int, c_void_p, c_void_p, c_size_t, POINTER(LsaStats),
                                 c_void_p]),
    "lsa_phiv_lincomb_adaptive": (c_int, [POINTER(LsaOp), c_void_p, c_int, c_double, c_double, c_int,
                                          c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                          c_size_t, POINTER(LsaStats), POINTER(c_int), POINTER(c_int),
                                          c_void_p]),
    "lsa_lincomb_adaptive_m_workspace_bytes": (c_size_t, [POINTER(LsaOp), c_int]),
    "lsa_phiv_lincomb_adaptive_m": (c_int, [POINTER(LsaOp), c_void_p, c_int, c_double, c_double, c_int,
                                            c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                            c_void_p, c_size_t, POINTER(LsaStats), POINTER(c_int),
                                            POINTER(c_int), POINTER(c_int), c_int, c_void_p]),
    "lsa_phiv_host": (c_int, [POINTER(LsaOp), c_void_p, c_double, c_int, c_int, c_double, c_int, c_int,
                              c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "lsa_probe_fp64_fma": (c_int, [c_int, c_void_p, POINTER(c_double), c_void_p]),
    "lsa_tune_step": (c_int, [POINTER(LsaOp), c_void_p, c_int, c_int, c_int, c_void_p, c_size_t, c_int,
                              POINTER(c_int), POINTER(c_float), POINTER(c_float), c_void_p]),
    "lsa_rhs": (c_int, [POINTER(LsaOp), c_void_p, c_void_p, c_void_p]),
    "lsa_axpby": (c_int, [c_longlong, c_double, c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    "lsa_expm_phi": (c_int, [c_void_p, c_int, c_int, c_double, c_int, c_void_p, c_void_p, c_size_t,
                             c_void_p]),
    "lsa_read_stats": (c_int, [c_void_p, POINTER(LsaStats), c_void_p]),
    "lsa_phiv_noalloc": (c_int, [POINTER(LsaOp), c_void_p, c_double, c_int, c_int, c_double, c_int,
                                 c_int, c_void_p, POINTER(LsaStats), c_void_p]),
    "lsa_selftest_barrier_timeout": (c_int, [c_void_p, c_size_t, c_double, c_void_p]),
    "lsa_batch_workspace_bytes": (c_size_t, [POINTER(LsaOp), POINTER(c_int), c_int, c_int, c_int]),
    "lsa_batch_create": (c_int, [POINTER(LsaOp), POINTER(c_int), c_int, c_double, c_int, c_double,
                                 c_int, c_int, c_void_p, c_size_t, POINTER(c_void_p), c_void_p]),
    "lsa_batch_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                               POINTER(c_longlong), POINTER(c_longlong), POINTER(c_longlong),
                               POINTER(c_longlong)]),
    "lsa_batch_set_tiling": (c_int, [c_void_p, c_int, c_int]),
    "lsa_batch_set_step_form": (c_int, [c_void_p, c_int]),
    "lsa_batch_step_form": (c_int, [c_void_p]),
    "lsa_batch_run": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "lsa_batch_read_stats": (c_int, [c_void_p, POINTER(LsaStats), POINTER(c_int), c_void_p]),
    "lsa_batch_tune": (c_int, [c_void_p, c_void_p, c_void_p, c_int, POINTER(c_int), POINTER(c_int),
                               POINTER(ctypes.c_float), c_void_p]),
    "lsa_batch_destroy": (None, [c_void_p]),
    "lsa_phiv_vjp_workspace_bytes": (c_size_t, [POINTER(LsaOp), c_int]),
    "lsa_phiv_vjp": (c_int, [POINTER(LsaOp), c_void_p, c_double, c_int, c_int, c_void_p, c_void_p,
                             c_void_p, c_void_p, c_void_p, c_size_t, POINTER(LsaStats), c_void_p]),
    "lsa_phiv_batched": (c_int, [POINTER(LsaOp), POINTER(c_int), c_int, c_void_p, c_double, c_int,
                                 c_double, c_int, c_int, c_void_p, c_void_p, c_size_t,
                                 POINTER(LsaStats), c_void_p]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"liblsarnoldi.so not found at {path}; build it with "
            "`python -m paper_2410_14917_gb300.build` (needs nvcc). There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class LsaError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def status_string(status: int) -> str:
    return lib().lsa_status_string(int(status)).decode()
