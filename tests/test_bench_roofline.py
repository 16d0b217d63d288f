"""The roofline figures bench.py reports, recounted by hand (CPU).

Config 2 (1024 x 1024 cells, central slopes, 2048 x 2048 padded, FP32): the
column pass transforms 1025 columns (the half spectrum of 2048-point rows)
forward once (the slope spectra are formed from sigma's) and inversely twice
(Fx, Fy), at 5 L log2 L flops per complex transform of length L, plus about 60
flops per bin for the slope spectra and the six-term products. It reads the
row pass's 1025 x 1024 complex bins and six real quarter planes of kernel
spectra (1025 x 1025 each) and writes 2 x 1025 x 1024 complex bins.
"""
import math

import pytest

import bench

WL = {"patches": [(0, 1024, 1024, -1.0, -1.0, 2.0 / 1024)], "slope_mode": 1}
INFO = {"cross_mode": 0}


def test_column_pass_flops():
    per_column = 3 * 5 * 2048 * math.log2(2048) + 60 * 2048
    assert bench.algorithmic_flops(WL, INFO, "col_conv") == pytest.approx(1025 * per_column, rel=1e-12)
    assert bench.algorithmic_flops(WL, INFO, "col_conv") == 472_320_000


def test_column_pass_bytes():
    row_bins = 1025 * 1024 * 8          # complex64 bins of sigma's row transforms
    planes = 6 * 1025 * 1025 * 4        # real quarter planes of the three kernel spectra
    out = 2 * 1025 * 1024 * 8           # Fx^, Fy^ after their column transforms
    assert bench.algorithmic_bytes(WL, INFO, "col_conv") == row_bins + planes + out == 50_405_400


def test_row_passes_bytes():
    sigma = 1024 * 1024 * 4
    assert bench.algorithmic_bytes(WL, INFO, "row_fwd") == sigma + 1025 * 1024 * 8
    assert bench.algorithmic_bytes(WL, INFO, "row_inv") == 2 * 1025 * 1024 * 8 + 2 * 1024 * 1024 * 4


def test_caller_slopes_transform_three_fields():
    wl = dict(WL, slope_mode=2)
    per_column = (3 + 2) * 5 * 2048 * math.log2(2048) + 4 * 2 * 3 * 2048
    assert bench.algorithmic_flops(wl, INFO, "col_conv") == pytest.approx(1025 * per_column, rel=1e-12)
    assert bench.algorithmic_bytes(wl, INFO, "row_fwd") == 3 * 1024 * 1024 * 4 + 3 * 1025 * 1024 * 8


def test_measured_traffic_is_the_column_pass_reads():
    # the captured DRAM traffic of the column pass is its reads (row bins and the
    # planes as stored, rows padded to 1028 floats); its output stays in L2
    reads = 1025 * 1024 * 8 + 6 * 1025 * 1028 * 4
    assert bench.TRAFFIC[("spiral1024", "col_conv")] == pytest.approx(reads, rel=0.01)
