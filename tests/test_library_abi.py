"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lsarnoldi.h declares.  Host-only calls are exercised; nothing here
needs a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsarnoldi.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(lsa_[a-z0-9_]+)\s*\(", text,
                       flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_14917_gb300 import build as b
    from paper_2410_14917_gb300 import _binding

    b.build()
    return _binding.load_library()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for n in ["lsa_phiv", "lsa_arnoldi", "lsa_matvec", "lsa_expm_phi", "lsa_workspace_bytes",
              "lsa_read_stats", "lsa_selftest_barrier_timeout", "lsa_op_dof"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2410_14917_gb300 import _binding

    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _binding.SIGNATURES, f"binding lacks {name}"


def test_host_only_calls(lib):
    from paper_2410_14917_gb300._binding import LsaOp

    assert lib.lsa_max_m() == 64
    assert lib.lsa_version() >= 100
    assert lib.lsa_status_string(-3) == b"LSA_ERR_TIMEOUT"
    op = LsaOp(1, 64, 64, 1, 1 / 64, 0.01, 0.0, (ctypes.c_double * 3)(1.0, 0.5, 0.0), 0.0, 0.0,
               None, None)
    assert lib.lsa_op_dof(ctypes.byref(op)) == 4096
    bad = LsaOp(1, 64, 64, 2, 1 / 64, 0.01, 0.0, (ctypes.c_double * 3)(1.0, 0.5, 0.0), 0.0, 0.0,
                None, None)
    assert lib.lsa_op_dof(ctypes.byref(bad)) == -1          # 2D operator with nz = 2
    gs = LsaOp(2, 8, 8, 1, 0.1, 1e-3, 1e-3, (ctypes.c_double * 3)(), 0.04, 0.06, None, None)
    assert lib.lsa_op_dof(ctypes.byref(gs)) == -1           # Gray-Scott without its fields
    assert lib.lsa_phiv(None, None, 0.0, 0, 1, 0.0, 0, 0, None, None, 0, None, None) == -1
    assert lib.lsa_phiv_lincomb(None, None, 0, 0.0, 1, 1, 0.0, 0, 0, None, None, 0, None, None) == -1
    assert lib.lsa_rhs(ctypes.byref(op), None, None, None) == -1        # not a Gray-Scott operator
    assert lib.lsa_axpby(-1, 1.0, None, 1.0, None, None, None) == -1
    assert lib.lsa_axpby(0, 1.0, None, 1.0, None, None, None) == 0      # nothing to do


def test_library_targets_sm103a():
    from paper_2410_14917_gb300 import build as b

    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)
