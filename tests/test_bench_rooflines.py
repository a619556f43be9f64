"""The benchmark's roofline arithmetic, on made-up timings (no GPU): each figure follows from its stated
per-unit work, so a slip in a formula shows here rather than in a number on the GPU."""
import pytest

import bench

PEAKS = {"bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0}


def test_flops_per_solve_counts_each_step():
    n, k = 64, 3
    # A G, GENP (sum over steps of 2 (n - s)^2 + (n - s) flops), solves and X = G Y, one sweep
    genp = sum(2 * (n - s - 1) ** 2 + (n - s - 1) for s in range(n))
    assert genp == pytest.approx(2 * n**3 / 3 - n**2 / 2 - n / 6)
    one = bench.flops_per_solve(n, k, 1)
    assert one == pytest.approx((2 * n**3 - n**2) + genp + 4 * n**2 * k + 6 * n**2 * k)
    assert bench.flops_per_solve(n, k, 3) - one == pytest.approx(2 * 6 * n**2 * k)


def test_update_roofline_from_event_timings():
    d = 6
    pairs = d * (d + 1) // 2
    sizes = [(4096, 4096), (2048, 2048)]                      # M = N of two launches
    mma = sum(pairs * 2.0 * m * nn * 128 for m, nn in sizes)
    timing = {"update128": (2, 4.0, mma), "update": (3, 1.0, 3e12)}
    r = bench.update_roofline(timing, steps=1, step_ms=20.0, digits=d, peaks=PEAKS)
    assert r["achieved"] == pytest.approx(mma / 4e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1800.0)
    assert r["frac_of_sustained"] == pytest.approx(r["achieved"] / 1600.0)
    mean_mn = sum(m * nn for m, nn in sizes) / 2
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(16.0 * mean_mn)
    assert r["traffic"] == pytest.approx(bench.UPD128_TRAFFIC_PER_MN * mean_mn)
    assert r["share_of_step"] == pytest.approx(4.0 / 20.0)
    assert r["ms_per_launch"] == pytest.approx(2.0)
    assert r["algorithmic_fp64_tflops"] == pytest.approx(r["achieved"] / pairs)
    assert r["other_updates"]["achieved"] == pytest.approx(3e12 / 1e-3 / 1e12)
    assert bench.update_roofline({"update128": (0, 0.0, 0.0), "update": (0, 0.0, 0.0)}, 1, 1.0, d, PEAKS) is None


def test_apply_roofline_counts_padded_digit_pairs():
    n, d, ms = 1000, 4, 2.0                                  # pads to 1024 x 1024, K to 1024
    r = bench.oz_roofline(n, ms, d, PEAKS)
    assert r["digit_pairs"] == 10
    assert r["achieved"] == pytest.approx(10 * 2.0 * 1024 * 1024 * 1024 / 2e-3 / 1e12)
    assert r["algorithmic_fp64_tflops"] == pytest.approx((2 * n**3 - n**2) / 2e-3 / 1e12)
    assert r["traffic"] == pytest.approx(bench.OZ_AG_TRAFFIC_PER_N3[4] * n**3)
    assert bench.oz_roofline(n, ms, 5, PEAKS)["traffic"] is None  # no capture of the 5-digit kernel


def test_traffic_constants_are_near_the_algorithmic_bytes():
    # the 128-deep update reads and writes E once: 16 B per element, within the digit planes' share
    assert 15.0 <= bench.UPD128_TRAFFIC_PER_MN <= 17.0
