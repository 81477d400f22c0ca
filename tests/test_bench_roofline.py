"""The benchmark's roofline arithmetic on the CPU: the coverage kernel's lane
ops per sample test for a pixel-class mix, the derived ALU peak, and the
whole-job throughput of weak scaling."""
import pytest

import bench


def test_ops_per_test_follow_the_pixel_mix():
    mix = {"convex_pixels": 402330351, "two_triangle_pixels": 564822565, "general_pixels": 0}
    ops = bench.ops_per_test(mix)
    assert ops == pytest.approx((7 * 402330351 + 9 * 564822565) / 967152916)
    assert 7.0 < ops < 9.0
    assert bench.ops_per_test(mix, exact=True) == pytest.approx(8.0)
    assert bench.ops_per_test({}) == bench.OPS_PER_TEST["general_pixels"]


def test_derived_alu_peak():
    # 152 SMs x 128 lane ops per clock at 2070 MHz, 8 ops per test
    assert bench.alu_peak_tests(2070.0, 8.0) == pytest.approx(152 * 128 * 2070e6 / 8.0)
    assert bench.alu_peak_tests(2070.0, 8.168) == pytest.approx(4.93e12, rel=2e-3)


def test_coverage_traffic_per_entry_is_a_plausible_gather():
    # DRAM bytes per bin entry from the capture: below the 40-byte gather of two
    # ribs, a tag and a bin id (neighbouring entries share ribs in L2)
    assert 4.0 < bench.COVERAGE_TRAFFIC_PER_PAIR < 40.0


def test_weak_scaling_throughput():
    assert bench.job_throughput(295431, 4, 17.29) == pytest.approx(4 * 295431 / 17.29e-3)


def test_algorithmic_bytes_follow_the_method():
    # tessellation 40S + 24P + 20R + 4L, binning 16R + 4 pairs + 4 tiles, split
    # over the stage's kernels; coverage counts 16 sample tests per span pixel
    c = {"R": 1000, "L": 70, "S": 30, "P": 10, "pairs": 5000, "tiles": 64, "span_px": 777}
    tess = sum(bench.algorithmic(k, c)[1] for k in ("k_link_setup", "k_emit", "k_arclen_scan"))
    assert tess == 40 * 30 + 24 * 10 + 20 * 1000 + 4 * 70
    binb = sum(bench.algorithmic(k, c)[1] for k in ("k_bin_count", "k_tile_scan", "k_bin_scatter"))
    assert binb == 16 * 1000 + 4 * 5000 + 4 * 64
    assert bench.algorithmic("k_coverage", c) == ("alu", 16 * 777)
    st = bench.stage_report({"k_link_setup": 1.0, "k_emit": 2.0, "k_arclen_scan": 1.0}, c, 1000.0)
    assert st["tessellation"]["algorithmic_bytes"] == tess
    assert st["tessellation"]["achieved_gbs"] == pytest.approx(tess / 4e-3 / 1e9)
    assert "binning" not in st


def test_measured_coverage_peak_follows_the_class_rates():
    mix = {"convex_pixels": 400, "two_triangle_pixels": 600, "general_pixels": 0}
    pk = bench.measured_peak_tests(mix, 2070.0)
    rc = bench.MEASURED_TESTS_PER_SM_CLK["convex_pixels"] * 152 * 2070e6
    rt = bench.MEASURED_TESTS_PER_SM_CLK["two_triangle_pixels"] * 152 * 2070e6
    assert pk == pytest.approx(1.0 / (0.4 / rc + 0.6 / rt))
    assert rt < pk < rc
    assert bench.measured_peak_tests(mix, 2070.0, exact=True) is None
    assert bench.measured_peak_tests({}, 2070.0) is None
