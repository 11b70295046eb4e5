"""CPU checks of bench.py's roofline accounting (no GPU): the derived peaks,
the roofline object built from measured kernel times, and that the committed
DRAM-traffic figures belong to the committed force-kernel sources (else the
bench would report traffic as null)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_derived_peaks():
    # 152 SMs x 2070 MHz x 2 flop per FMA: 128 FP32 lanes, 2 FP64 lanes per SM
    assert bench.PEAK_TFLOPS["mixed"] == pytest.approx(152 * 128 * 2 * 2.07e9 * 1e-12)
    assert bench.PEAK_TFLOPS["fp64"] == pytest.approx(152 * 2 * 2 * 2.07e9 * 1e-12)
    assert bench.FLOPS_PER_INTERACTION == 20


def test_roofline_object():
    n = 10425
    force_ms, verlet_ms = 0.0682, 0.0085
    force_tflops = 20 * n * (n - 1) / (force_ms * 1e-3) * 1e-12
    r = {"force_tflops": force_tflops, "achieved_tflops": 0.9 * force_tflops,
         "kernel_ms": {"force_ms": force_ms, "verlet_ms": verlet_ms, "step_ms": 0.08, "steps": 100}}
    ro = bench.roofline(r, "mixed", 368128)
    assert ro["bound"] == "alu" and ro["unit"] == "TFLOP/s" and ro["traffic"] == 368128
    assert ro["achieved"] == pytest.approx(31.9, rel=2e-3)
    assert ro["frac"] == pytest.approx(ro["achieved"] / ro["peak"])
    assert ro["force_share"] == pytest.approx(force_ms / (force_ms + verlet_ms))
    assert ro["frac_step"] == pytest.approx(0.9 * ro["frac"])
    assert bench.roofline(r, "fp64", None)["peak"] == bench.PEAK_TFLOPS["fp64"]


def test_traffic_figures_match_the_force_kernel_sources():
    h = bench.kernel_hash()
    assert (h, "mixed") in bench.NCU_TRAFFIC and (h, "fp64") in bench.NCU_TRAFFIC, (
        "the force kernel sources changed since the DRAM counters were taken: re-take them with ncu "
        "and update NCU_TRAFFIC")


def test_roofline_against_measured_peaks():
    n = 10425
    r = {"force_tflops": 0.7, "achieved_tflops": 0.65,
         "kernel_ms": {"force_ms": 3.1, "verlet_ms": 0.04, "step_ms": 3.2, "steps": 10}}
    peaks = {"fp32_tflops": 77.4, "fp64_tflops": 1.05}
    ro = bench.roofline(r, "fp64", None, peaks)
    assert ro["peak_measured_tflops"] == 1.05 and ro["frac_of_measured"] == pytest.approx(0.7 / 1.05)
    assert bench.roofline(r, "mixed", None, peaks)["frac_of_measured"] == pytest.approx(0.7 / 77.4)
    assert "frac_of_measured" not in bench.roofline(r, "mixed", None)
