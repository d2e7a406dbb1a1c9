"""Host logic of bench.py that turns measurements into the reported line:
the choice of the roofline kernel and its fractions, and the search for the
fewest fixed cycle counts that reach the error target."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.fixture
def no_profile(monkeypatch):
    monkeypatch.setattr(bench, "profile_traffic", lambda stage: (None, None))
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6000.0})


def test_roofline_picks_the_largest_kernel_stage(no_profile):
    # per stage: (ms over all steps, launches over all steps, dense work)
    stages = {"outer_residual": (500.0, 2, 0.0),           # composite: a sum of kernels
              "pixel_smoother.n1024": (900.0, 4, 1.0e9),   # a sub-stage of one kernel stage
              "legendre_adjoint_f64": (200.0, 2, 3.0e11),
              "legendre_synth_f32": (150.0, 40, 4.0e12),
              "ring_fft_apply_f32": (50.0, 40, 2.0e11)}
    r = bench.roofline_of(stages, {"legendre_adjoint_f64": 2.0e11}, 2, {"f64": 1.25, "f32": 80.0})
    assert r["kernel"] == "legendre_adjoint_f64"
    assert r["ms_per_step"] == 100.0 and r["launches_per_step"] == 1.0
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == 1.25
    # executed flops: 2e11 in 200 ms = 1.0 TFLOP/s; dense 1.5
    assert r["achieved"] == pytest.approx(1.0) and r["frac"] == pytest.approx(0.8)
    assert r["frac_executed"] == r["frac"]
    assert r["achieved_dense"] == pytest.approx(1.5) and r["frac_dense"] == pytest.approx(1.2)
    assert r["algorithmic_work_per_launch"] == pytest.approx(1.0e11)
    assert "measured live" in r["peak_source"]


def test_roofline_of_a_memory_stage_uses_the_copy_bandwidth(no_profile):
    stages = {"ring_fft_apply_f32": (100.0, 10, 6.0e11), "top_smoother": (1.0, 1, 0.0)}
    r = bench.roofline_of(stages, {}, 1, {})
    assert r["kernel"] == "ring_fft_apply_f32"
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6000.0
    assert r["achieved"] == pytest.approx(6000.0) and r["frac"] == pytest.approx(1.0)


def test_roofline_without_a_live_peak_falls_back_to_nominal(no_profile):
    r = bench.roofline_of({"legendre_synth_f32": (10.0, 1, 8.0e11)}, {}, 1, {})
    assert r["peak"] == bench.FP32_PEAK_TFLOPS and r["peak_source"].startswith("nominal")


class _Solver:
    """error after c cycles: 10 / 3^c (below 1 uK from 3 cycles on)"""

    def __init__(self):
        self.calls = []

    def solve(self, c):
        self.calls.append(c)

    def worst(self):
        return 10.0 / 3.0 ** self.calls[-1]


@pytest.mark.parametrize("start", [1, 2, 3, 5, 9])
def test_fewest_cycles_from_any_start(start):
    s = _Solver()
    assert bench.fewest_cycles(s.solve, s.worst, start, 12) == 3
    assert s.calls[-1] == 3  # the solution left behind is the chosen count's


def test_fewest_cycles_none_when_the_cap_is_too_small():
    s = _Solver()
    assert bench.fewest_cycles(s.solve, s.worst, 1, 2) is None


def test_cpu_baseline_prices_the_library_noise_grids():
    """The CPU baseline prices each level's inverse-noise term on the grid the
    library uses (Section 3.4's GL downgrade where the GL grid has at most
    3/5 of the observation rings): at Nside 2048 the first level (lmax 3000)
    stays on the observation grid, the second (lmax 2048) and below go to GL."""
    assert bench.gl_noise_grid(2048, 3000) is None
    assert bench.gl_noise_grid(2048, 2048) == (4097, 16384)
    assert bench.gl_noise_grid(2048, 1280) == (2561, 8192)
    assert bench.gl_noise_grid(32, 95) is None  # 191 rings > 3/5 of 127
    for nside, lh in [(2048, 2457), (2048, 2458), (256, 230), (256, 231)]:
        expect = 5 * (2 * lh + 1) <= 3 * (4 * nside - 1)
        assert (bench.gl_noise_grid(nside, lh) is not None) == expect
