"""Host-side pieces of the benchmark (no GPU): the work models behind the
roofline object, the roofline arithmetic, and the oracle sample of the CPU
baseline on a small matrix."""
import math

import numpy as np
import pytest

import bench
from paper_1604_03703_gb300 import inputs as I


def test_panel_sizes_and_flops():
    n, b = 1024, 128
    Ns = bench.panel_sizes(n, b)
    assert Ns[0] == n - b and all(N >= 2 for N in Ns)
    assert len(Ns) == math.ceil(n / b) - 1
    amount, unit, bound = bench.kernel_model("syr2k_tc", n, b, 4)
    assert unit == "flop" and bound == "tensor"
    assert amount == pytest.approx(sum(2.0 * N * (N + 1) * b for N in Ns))


def test_band_models_follow_the_schedule():
    n = 4096
    tri, unit, bound = bench.kernel_model("band_tri", n, 128, 4)
    assert unit == "byte" and bound == "hbm"
    assert tri == pytest.approx(2 * 4 * 16 * n ** 2)  # last stage 16 -> 1
    chase, _, _ = bench.kernel_model("band_chase", n, 128, 4)
    # 128 -> 32 (k = 4) and 32 -> 16 (k = 2)
    assert chase == pytest.approx(2 * 4 * (4 + 2) * n ** 2)


def test_band_models_follow_a_tuned_schedule():
    """With the schedule the autotuner chose (128 -> 32 -> 8 -> 1), the band
    work models follow it: 128 -> 32 (k = 4) and 32 -> 8 (k = 4) are chases,
    8 -> 1 is the sliding-window stage."""
    n = 16384
    sched = [128, 32, 8, 1]
    chase, _, _ = bench.kernel_model("band_chase", n, 128, 4, sched)
    assert chase == pytest.approx(2 * 4 * (4 + 4) * n ** 2)
    tri, _, _ = bench.kernel_model("band_tri", n, 128, 4, sched)
    assert tri == pytest.approx(2 * 4 * 8 * n ** 2)


def test_measured_traffic_is_tied_to_its_schedule():
    """The DRAM bytes recorded for a kernel belong to the schedule they were
    taken on; the bench drops them for any other schedule."""
    for name, t in bench.MEASURED_TRAFFIC.items():
        assert t["bytes_per_step"] > 0 and t["note"]
        assert t["schedule"][0] == 128 and t["schedule"][-1] == 1
        b = t["schedule"]
        assert all(x % y == 0 for x, y in zip(b[:-1], b[1:]))


def test_roofline_arithmetic():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1500.0}
    r = bench.roofline("band_chase", 3.0e9, "byte", "hbm", 1000.0, peaks, {"sm_mhz": 2000.0}, 4)
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(3.0)
    assert r["frac"] == pytest.approx(3.0 / 6000.0)
    t = bench.roofline("syr2k_tc", 5.0e12, "flop", "tensor", 100.0, peaks, None, 4)
    assert t["peak"] == pytest.approx(500.0) and t["achieved"] == pytest.approx(50.0)


def test_oracle_sample_extrapolates(orc):
    A = I.semicircle(96, 3)
    r = bench.oracle_sample(A, 96, 1e-9, 0.2)
    assert r["seconds_extrapolated"] > 0 and r["value"] > 0
    assert "Householder steps" in r["sample"]


def test_oracle_openmp_build_gives_the_same_bits(orc):
    """The all-cores CPU baseline runs the oracle compiled with OpenMP; its
    results must be the serial oracle's, bit for bit."""
    if orc.load_omp() is None:
        pytest.skip("no OpenMP runtime")
    for n in (5, 130, 517):
        A = I.semicircle(n, 40 + n)
        d1, e1 = orc.tridiagonalize(A)
        M = np.array(A, order="F", copy=True)
        d2, e2 = np.zeros(n), np.zeros(n)
        orc.tridiagonalize_inplace(M, d2, e2, -1, omp=True)
        np.testing.assert_array_equal(d1, d2)
        np.testing.assert_array_equal(e1, e2[: n - 1])
        np.testing.assert_array_equal(orc.bisect_range(d1, e1, 0, n, 1e-14, omp=True), orc.bisect(d1, e1, 1e-14))


def test_oracle_sample_all_cores(orc):
    A = I.semicircle(96, 4)
    r = bench.oracle_sample(A, 96, 1e-9, 0.2, omp=True)
    if r is None:
        pytest.skip("no OpenMP runtime")
    assert r["cores"] == bench.host_cores() and r["value"] > 0
