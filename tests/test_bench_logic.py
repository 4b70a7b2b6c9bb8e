"""Host-side arithmetic of bench.py: the segments that keep a long measurement
inside the range where the diagonals' e^{2 alpha t} growth (Eq. 6) stays
finite in FP32, and the kernel launch count of whole captured graphs."""
import pytest

import bench


@pytest.mark.parametrize("n", [1, 7, 99, 100, 101, 250, 1000])
def test_segments_cover_the_steps_within_the_bound(n):
    segs = bench.segments(n)
    assert sum(segs) == n
    assert all(0 < s <= bench.SEG for s in segs)
    assert len(segs) == -(-n // bench.SEG)


def test_default_run_is_one_segment():
    assert bench.segments(100) == [100]


def test_graph_launch_count():
    # a 100-iteration segment launches 13 graphs of 8 iterations: 104 iterations' kernels
    assert bench.GRAPH_ITERS == 8
    assert bench.launched_iterations(100) == 104
    assert bench.launched_iterations(400) == 4 * 104
    assert bench.launched_iterations(101) == 104 + 8
    assert bench.launched_iterations(1) == 8


def test_set_segments_stay_below_the_earliest_overflow():
    # warm-up (25 schedule trials + one captured chunk of 8) plus a segment: 60 < 66, the
    # earliest overflow in the set
    assert bench.SET_WARM >= 1 + 8 * 3 + bench.GRAPH_ITERS
    assert bench.SET_WARM + bench.SEG_SET <= 60


PEAKS = {"bf16_tflops": 1950.4, "bf16_tflops_sustained": 1744.4, "sm_max_mhz": 2070.0, "hbm_gbs": 6700.2}


def test_burst_peak_only_for_a_short_region_at_the_maximum_clock():
    at_max = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0}
    p, src = bench.tensor_peak(PEAKS, "measured", at_max, 190.0)
    assert p == PEAKS["bf16_tflops"] and "burst" in src
    assert bench.tensor_peak(PEAKS, "measured", {"sm_mhz": 1500.0, "sm_max_mhz": 2070.0}, 190.0)[0] == 1744.4
    assert bench.tensor_peak(PEAKS, "measured", at_max, 4000.0)[0] == 1744.4
    assert bench.tensor_peak(PEAKS, "measured", None, 100.0)[0] == 1744.4


class _FakePanda:
    PANDA_FP32, PANDA_BF16X3, PANDA_BF16X2, PANDA_FP8MIX = 0, 1, 2, 3


def test_issued_flops_per_precision():
    T, G = 1000, 17000
    useful = 2.0 * T * G * G + 2.0 * T * T * G
    u, issued, units = bench.kernel_flops(_FakePanda, 1, "k_tc_phase1", T, G)
    assert u == useful and issued == units == 3 * useful
    assert bench.kernel_flops(_FakePanda, 2, "k_tc_phase1", T, G)[1] == 2 * useful
    u, issued, units = bench.kernel_flops(_FakePanda, 3, "k_tc_phase1", T, G)
    assert issued == 2.0 * T * G * G + 3 * 2.0 * T * T * G and units == T * G * G + 6.0 * T * T * G
    assert bench.kernel_flops(_FakePanda, 1, "k_fin", T, G)[0] == 0.0


def test_roofline_reports_both_phase_kernels_and_the_iteration():
    T, G = 1000, 17000
    kstats = [("k_tc_phase1", 107.0, 100), ("k_reduce_wnorms", 0.5, 100), ("k_tc_phase2", 76.0, 100),
              ("k_fin", 2.3, 100), ("k_tail", 0.4, 100)]
    roof = bench.roofline(_FakePanda, 1, kstats, T, G, "none", PEAKS, "measured",
                          {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0}, 186.0, None, 530.0)
    assert roof["kernel"] == "k_tc_phase1" and roof["peak"] == PEAKS["bf16_tflops"]
    assert abs(roof["frac"] - (2.0 * T * G * G + 2.0 * T * T * G) / 1.07e-3 / 1e12 / 1950.4) < 1e-9
    names = [k["kernel"] for k in roof["kernels"]]
    assert names == ["k_tc_phase1", "k_tc_phase2"]
    it = roof["iteration"]
    assert abs(it["useful_frac"] * 3 - it["issued_frac"]) < 1e-12
