"""bench.py's host-side arithmetic on CPU: the roofline records of the FFT and
direct paths from stage times, the accuracy regions, and the reference arm's
extrapolation fields (no GPU; the values are made up)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2208_11422_gb300 import synth  # noqa: E402


def test_fft_roofline_picks_the_slowest_kernel_and_its_fractions():
    g = synth.CONFIGS[2]
    plan = {"F": 64, "bins": 2112, "tiles": 16}
    stage = [8.3, 0.0, 9.0, 0.57, 0.42, 6.5, 6.4, 3.7, 1.7, 1.83, 0.68]
    peaks, src = bench.measured_peaks()
    roof = bench.fft_roofline(g, plan, "bf16x3", stage, peaks, src, 80.0, 2070.0,
                              {"bytes": 32.0e9, "lo_tiles_kept": 1, "lo_tiles": 2})
    assert roof["kernel"] == "forward contraction" and roof["bound"] == "hbm"
    fwd = roof["kernels"]["forward_contraction"]
    assert abs(fwd["algorithmic_bytes"] - (32.0e9 + 8.0 * 2112 * 16 * (11475 + 225))) < 1.0
    assert abs(roof["frac"] - fwd["GBps"] / peaks["hbm_gbs"]) < 1e-12
    assert roof["traffic"] is None                       # no capture of this build's contraction
    assert roof["kernels"]["volume_r2c"]["traffic"] > 0  # the transforms' scaled capture


def test_direct_rooflines_use_the_precision_peak():
    g = synth.CONFIGS[2]
    r16 = bench.direct_tensor_roofline(g, "bf16", [40.0, 0, 38.0])
    r32 = bench.direct_tensor_roofline(g, "tf32", [40.0, 0, 38.0])
    assert abs(r32["peak"] / r16["peak"] - bench.TF32_OVER_BF16) < 1e-12
    assert r32["frac_algorithmic"] > r16["frac_algorithmic"]


def test_accuracy_regions_are_crop_0_of_the_test_crops():
    g = synth.CONFIGS[2]
    (i0, j0), (b0, b1) = bench.accuracy_regions(g)
    rng = np.random.default_rng(300)
    assert (i0, j0) == (int(rng.integers(0, g.H - 255)), int(rng.integers(0, g.W - 255)))
    assert b0 - i0 == b1 - j0 == (bench.ACC_CROP - bench.ACC_BLOCK) // 2
    assert bench.rel_l2([1.0, 2.0], [1.0, 2.0]) == 0.0
