"""bench.py's roofline arithmetic and constants, on CPU: the flop numerator of
every workload is the algorithmic count the oracle composes (written into
bench.py by `python -m oracle.flops`), and the roofline, HBM and ALU-peak
formulas give the figures they state for a hand-built case."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench                      # noqa: E402
from oracle import flops as F     # noqa: E402


@pytest.mark.parametrize("name", sorted(F.BENCH_WORKLOADS))
def test_flop_numerator_is_the_composed_count(name):
    assert name in bench.ALGO_FLOPS
    assert bench.ALGO_FLOPS[name] == pytest.approx(float(F.per_cell_stage(F.BENCH_WORKLOADS[name])), abs=1e-4)


def test_alu_peaks_from_unit_counts():
    # 148 SMs x (2 FP64 | 128 FP32 FMA per clock) x 2 flops x 2032 MHz
    assert bench.alu_peak_tflops("f64", 148, 2032.0) == pytest.approx(1.202944)
    assert bench.alu_peak_tflops("f32", 148, 2032.0) == pytest.approx(76.988416)


def test_roofline_fraction_and_traffic():
    cells, ms = 4096 * 4096, 118.0
    r = bench.roofline("euler2d_char", cells, ms, "f64", 148, 2032.0, "FP64", traffic_per_cell=270.0, probe=1.2)
    achieved = bench.ALGO_FLOPS["euler2d_char"] * cells / (ms * 1e-3) / 1e12
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / 1.202944)
    assert r["frac_of_probe"] == pytest.approx(achieved / 1.2)
    assert r["traffic"] == pytest.approx(270.0 * cells)
    assert r["frac_executed"] == pytest.approx(bench.EXEC_FLOPS[("euler2d_char", "f64")] * cells / (ms * 1e-3)
                                               / 1e12 / 1.202944)
    # the executed count is below the algorithmic one (the kernels share subexpressions)
    for (key, _), ex in bench.EXEC_FLOPS.items():
        assert ex < bench.ALGO_FLOPS[key]


def test_hbm_bytes_per_cell_stage():
    # stage 1 reads F and writes F + D, stages 2-3 read 2F and write F: (8F + D)/3 words
    h = bench.hbm_fraction("euler2d", 8, 1000, 1.0, 6481.1, "of measured")
    assert h["bytes_per_cell_stage"] == pytest.approx((8 * 12 + 8) / 3 * 8)
    assert h["achieved_gbs"] == pytest.approx(h["bytes_per_cell_stage"] * 1000 / 1e-3 / 1e9)
    assert bench.words_per_cell_stage("scalar1d") == pytest.approx((8 * 2 + 1) / 3)
