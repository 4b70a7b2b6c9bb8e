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
    # warm-up at most 20, segment at most 40: 60 < 66, the earliest overflow in the set
    assert 20 + bench.SEG_SET <= 60
