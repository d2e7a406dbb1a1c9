"""Host logic of bench.py that prices the CPU baseline: the count of SHT
pairs (one synthesis + one adjoint) in one realization, against a hand
count of the CR-Cycle of Fig. code:mg.

Per visit of a pixel level from a zero start: smoothing (one Y_h pair),
residual (one A_h pair), the recursion, residual after the correction,
smoothing again -- 2 A_h + 2 Y_h pairs; a later visit (n_rec = 2) also forms
the residual first (one more A_h).  The top level has a diagonal smoother:
2 full-band A pairs per cycle.  The FP64 outer residual adds one full-band
pair before every cycle but the first."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_one_pixel_level_two_cycles():
    levels = [(16, 40, 2, None)]  # Nside 16 level, band limit 40, noise on the observation grid
    got = bench.realization_pairs(32, 95, levels, 2)
    assert got[("healpix", 32, 95)] == 2 * 2 + 1  # top residuals + one outer residual
    assert got[("healpix", 32, 40)] == 2 * 2  # A_1 on the observation grid, one visit per cycle
    assert got[("healpix", 16, 40)] == 2 * 2  # Y_1 around the smoother
    assert len(got) == 3


def test_two_levels_second_visited_twice_per_cycle():
    levels = [(16, 40, 2, None), (8, 20, 2, (41, 128))]
    got = bench.realization_pairs(32, 95, levels, 1)
    assert got[("healpix", 32, 95)] == 2
    assert got[("healpix", 32, 40)] == 2
    assert got[("healpix", 16, 40)] == 2
    # level 2 (GL noise grid): visits from zero then from the previous
    # iterate: 2 + 3 A_2 pairs, 2 + 2 Y_2 pairs
    assert got[("gl", 41, 128, 20)] == 5
    assert got[("healpix", 8, 20)] == 4
