"""The benchmark's roofline arithmetic on the CPU: algorithmic bytes and
flops per cell-update (2w/bT bytes, 2n-1 flops, Dot2's 10n-7, +1 for a
division), the three roof terms, and the fields of the roofline object that
a reader recomputes from them (achieved rate, fraction, the roof at the
largest built degree)."""
import math

import pytest

import bench
from paper_2001_01473_gb300 import inputs

STAR, BOX = inputs.STAR, inputs.BOX


@pytest.mark.parametrize("ndim,shape,R,dt,post,want", [
    (2, STAR, 1, "f32", None, 9), (2, STAR, 4, "f32", None, 33), (2, BOX, 2, "f64", None, 49),
    (3, STAR, 1, "f32", None, 13), (3, BOX, 1, "f32", None, 53), (3, BOX, 1, "f32", "div", 54),
    (2, STAR, 1, "f32c", None, 43), (2, BOX, 1, "f16", None, 17)])
def test_flops_per_cell(ndim, shape, R, dt, post, want):
    assert bench.flops_per_cell(ndim, shape, R, dt, post) == want


def test_roof_terms_star2d1r():
    t = bench.roof_terms(2, STAR, 1, "f32", 6, None, 6779.0, 40000.0, 80.0)
    assert math.isclose(t["hbm"], 6779e9 * 6 / 8)          # 2 words of 4 bytes per bT steps
    assert math.isclose(t["alu"], 80e12 / 9)
    assert math.isclose(t["smem"], 40000e9 / (2 * 4 / 6))  # the staged row, once per pass
    t64 = bench.roof_terms(2, STAR, 1, "f64", 2, None, 6779.0, 40000.0, 1.0)
    assert math.isclose(t64["hbm"], 6779e9 * 2 / 16)


def test_sweep_roofline_fields(monkeypatch):
    monkeypatch.setattr(bench, "load_measured_peaks", lambda: ({"hbm_gbs": 6779.0}, "measured"))
    inrun = {"fp64_gflops": 1057.0, "smem_gbs": 40083.0}
    cells = 16384.0 * 16384.0
    launch_s = 0.0004943
    r = bench.sweep_roofline(2, STAR, 1, "f32", None, cells, 6, launch_s, inrun, "k", traffic=None)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6779.0
    assert math.isclose(r["algorithmic_bytes_per_launch"], cells * 8)
    assert math.isclose(r["achieved"], cells * 8 / launch_s / 1e9)
    assert math.isclose(r["frac"], r["achieved"] / 6779.0)
    gcells = cells * 6 / launch_s / 1e9
    assert math.isclose(r["temporal_roof_gcells"], 6779.0 * 6 / 8)
    assert math.isclose(r["frac_of_temporal_roof"], gcells / (6779.0 * 6 / 8))
    # the radius-1 FP32 star is built up to bT 10: the roof there is HBM-bound too
    assert r["largest_built_bT"] == max(bench.built_degrees(2, STAR, 1, "f32")) == 10
    assert math.isclose(r["roof_at_largest_bT_gcells"], 6779.0 * 10 / 8)
    # an HBM-bound fraction and the fraction of the temporal roof are the same number
    assert math.isclose(r["frac"], r["frac_of_temporal_roof"])


def test_sweep_roofline_alu_bound_fp64(monkeypatch):
    monkeypatch.setattr(bench, "load_measured_peaks", lambda: ({"hbm_gbs": 6779.0}, "measured"))
    inrun = {"fp64_gflops": 1057.0, "smem_gbs": 40083.0}
    cells = 512.0 ** 3
    r = bench.sweep_roofline(3, STAR, 1, "f64", None, cells, 1, 0.01, inrun, "k")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["peak"], 1.057)
    assert math.isclose(r["achieved"], cells * 13 / 0.01 / 1e12)


def test_batch_roof_one_grid(monkeypatch):
    monkeypatch.setattr(bench, "load_measured_peaks", lambda: ({"hbm_gbs": 8000.0}, "measured"))
    # star R1, 1000 x 2000 cells, T = 23 at degree 4: 5 passes of 4 and the
    # remaining 3 steps at degree 1 (the menu 8 / 4 / 1 below 4): 8 passes
    g = (STAR, 1, None, 1000, 2000, 23)
    r = bench.batch_roof([g], [4, 2, 1, 1])
    assert math.isclose(r["hbm_s"], 8 * 1000 * 2000 * 8.0 / 8000e9)
    alu = 152 * 128 * 2 * 2070e6
    assert math.isclose(r["alu_s"], 1000 * 2000 * 23 * 9 / alu)
    assert math.isclose(r["time_s"], max(r["hbm_s"], r["alu_s"]))


def test_adjoint_roof_one_grid(monkeypatch):
    monkeypatch.setattr(bench, "load_measured_peaks", lambda: ({"hbm_gbs": 8000.0}, "measured"))
    # box R2 (n = 25, nb = 2), T = 5: M = 3 blocks of 2, 2, 1 steps.
    # bytes per cell: 2 forward passes x 8; blocks of 2: recompute 4 + 4, transposed 8 + 8;
    # the block of 1: transposed 8 + 4
    g = (BOX, 2, None, 300, 400, 5)
    r = bench.adjoint_roof([g])
    byt = 2 * 8 + 2 * ((4 + 4) + (8 + 8)) + (8 + 4)
    assert math.isclose(r["hbm_s"], 300 * 400 * byt / 8000e9)
    n = 25
    fl = (2 * n - 1) * 2 * 2 + 2 * (2 * n - 1) * 1 + 5 * (2 * n - 1 + 2 * n)
    assert math.isclose(r["alu_s"], 300 * 400 * fl / (152 * 128 * 2 * 2070e6))


def test_clock_summary():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    rows = [["0", "2070", "2070", "700.5", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["0", "1980", "2070", "1401.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
            ["0", "2070", "2070", "[N/A]", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["0", "2040", "2070", "900.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    c = bench.summarize_clocks(rows)
    assert c["sm_mhz"] == 2040.0          # median of the three samples with a power reading
    assert c["sm_max_mhz"] == 2070.0 and c["power_w_max"] == 1401.0 and c["samples"] == 4
    assert c["reasons"] == ["sw_power_cap"]
    rows[0][5] = "Active"
    assert bench.summarize_clocks(rows)["reasons"] == ["hw_slowdown", "sw_power_cap"]
