"""The benchmark's roofline arithmetic (host logic; no GPU): the algorithmic
counts of one Arnoldi launch in closed form, and the roofline object each
kernel form reports."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402


def closed_form(N, m, taps, field_elems, bs):
    """Sum over the m steps in closed form: step j moves (j+2) N elements, the
    final projection (m+2) N; flops 6(j-1) + 6 + 2 taps per unknown and step,
    2m + 2 in the final projection."""
    elems = (m * (m + 1) // 2 + 2 * m + m + 2) * N
    flops = (3 * m * (m - 1) + m * (6 + 2 * taps) + 2 * m + 2) * N
    return elems * bs + m * field_elems * bs, flops


@pytest.mark.parametrize("idx,precision,taps", [(1, "fp64", 7), (2, "fp32", 8), (2, "fp64", 8), (0, "fp64", 5)])
def test_algorithmic_counts_closed_form(idx, precision, taps):
    cfg = W.config(idx)
    N, m = W.n_dof(cfg), cfg["m"]
    bs = 8 if precision == "fp64" else 4
    fields = 0 if cfg["kind"] == "advdiff2d" else N
    assert bench.algorithmic_counts(cfg, precision, m) == closed_form(N, m, taps, fields, bs)


def test_headline_counts():
    # Gray-Scott 512^2, m = 64, float64: the figures the default line reports
    byts, flops = bench.algorithmic_counts(W.config(1), "fp64", 64)
    assert (byts, flops) == (9806282752, 7081033728)


@pytest.mark.parametrize("kind,name", [(0, "k_arnoldi (persistent hybrid Arnoldi, one-pass step)"),
                                       (4, "k_arnoldi (persistent hybrid Arnoldi, two-phase step)"),
                                       (5, "k_arnoldi_flat (persistent hybrid Arnoldi, flat two-phase step)")])
def test_fp64_roofline_object(kind, name):
    cfg = W.config(1)
    r = bench.phiv_roofline(cfg, "fp64", "hcwy", 9.5, 64, kind, 1.05, "test peak")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["kernel"] == name
    assert r["achieved"] == pytest.approx(7081033728 / 9.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.05)
    # traffic comes only from a capture of the kernel form that ran
    assert (r["traffic"] is None) == (("grayscott2d_512", "fp64", "hcwy", kind) not in bench.PROFILED_TRAFFIC)


@pytest.mark.parametrize("kind,kernel", [(0, "k_arnoldi"), (1, "k_arnoldi_tma"), (2, "k_arnoldi_stream"),
                                         (4, "k_arnoldi"), (5, "k_arnoldi_flat")])
def test_fp32_roofline_object(kind, kernel):
    cfg = W.config(2)
    r = bench.phiv_roofline(cfg, "fp32", "hcwy", 29.0, 40, kind, 1.05, "test peak")
    hbm, _ = bench.load_peaks()
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == hbm
    assert r["kernel"].startswith(kernel + " ")
    assert r["achieved"] == pytest.approx(r["algorithmic_bytes"] / 29.0e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm)
