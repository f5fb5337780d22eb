"""Roofline arithmetic of bench.py on the host: the algorithmic work per unit and the
achieved / peak / traffic fields computed from sampled kernel times (no GPU)."""
import argparse

import pytest

import bench


def test_algorithmic_flops_per_unique_unknown():
    # per element, divided by the d N^d unique unknowns it owns (N = 7, n = 8 points)
    per = lambda op, d: bench.algorithmic_flops_per_element(op, d, 8) / (d * 7 ** d)
    assert per("rhs", 2) == pytest.approx(8832 / 98)
    assert per("jacT", 2) == pytest.approx(13440 / 98)
    assert per("rhs", 3) == pytest.approx(153.749, abs=1e-3)
    assert per("jacT", 3) == pytest.approx(234.356, abs=1e-3)
    # J and J^T do the same work; J^T / F is 1.5 in the contraction count
    assert bench.algorithmic_flops_per_element("jac", 3, 8) == bench.algorithmic_flops_per_element("jacT", 3, 8)


def _args(workload="2d"):
    return argparse.Namespace(hbm_peak=6795.8, workload=workload, profile_every=64, no_graph=False)


def test_element_kernel_roofline_from_sampled_times():
    w = bench.WORKLOADS["2d"]
    # 10 timed J^T launches of 53 us each dominate; F and the assembly are smaller
    prof = {"rhs": (0.344, 10, 0.0), "jac": (0.0, 0, 0.0), "jacT": (0.53, 10, 0.0), "assemble": (0.2, 20, 1e8)}
    r = bench.roofline_of(prof, _args(), w, None, "fp64")
    flops = bench.algorithmic_flops_per_element("jacT", 2, 8) * 64 ** 2
    assert r["kernel"] == "jact2_kernel<double,8>" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / 53e-6 / 1e12)
    assert r["peak"] == pytest.approx(bench.PEAK_FP64_TFLOPS)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["avg_launch_us"] == pytest.approx(53.0)
    # the HBM roof of the same launch: 24 B per unique unknown (u and v in, J^T v out)
    assert r["hbm"]["algorithmic_bytes"] == 24 * 2 * 448 ** 2
    assert r["hbm"]["frac"] == pytest.approx(24 * 2 * 448 ** 2 / 53e-6 / 1e9 / 6795.8)
    # the recorded DRAM traffic is reported only while the kernel sources hash to its capture
    tr = bench.TRAFFIC["jact2_kernel<double,8>@2d@fp64"]
    expect = tr["bytes"] if tr["src"] == bench.kernel_src_hash("elem") else None
    assert r["traffic"] == expect


def test_assembly_roofline_uses_the_counted_bytes():
    w = bench.WORKLOADS["2d"]
    # 20 timed assembly launches moving 17 MB each in 10 us each
    prof = {"rhs": (0.05, 10, 0.0), "jac": (0.0, 0, 0.0), "jacT": (0.06, 10, 0.0), "assemble": (0.2, 20, 20 * 17e6)}
    r = bench.roofline_of(prof, _args(), w, None, "fp32_bulk")
    assert r["kernel"] == "assemble kernel" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(20 * 17e6 / 0.2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6795.8)
    assert r["traffic"] is None      # no capture recorded for the assembly
