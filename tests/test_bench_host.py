"""Host-side helpers of bench.py that choose where the serving loop's score
ciphertexts go in its page-locked arena: the runs of slices that copy at full
rate, and the ring that hands out block ranges inside them."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_fast_segments_skip_slow_and_remember_them():
    seen = set()
    # 10 slices of 100 blocks; slices 0-2 slow now
    segs = bench.fast_segments([2.0, 2.6, 4.9] + [193.0] * 7, seen, 100, 1000, 50)
    assert segs == [(300, 1000)] and seen == {0, 1, 2}
    # fast again later, but once slow they stay out
    assert bench.fast_segments([193.0] * 10, seen, 100, 1000, 50) == [(300, 1000)]
    # a new slow slice in the middle splits the run; the last slice is cut at total
    segs = bench.fast_segments([193.0] * 6 + [20.0] + [193.0] * 3, seen, 100, 950, 50)
    assert segs == [(300, 600), (700, 950)] and 6 in seen


def test_fast_segments_drop_short_runs_and_fall_back():
    seen = set()
    # run [100, 200) is shorter than the largest request (150 blocks)
    assert bench.fast_segments([1.0, 193.0, 1.0, 193.0, 193.0], seen, 100, 500, 150) == [(300, 500)]
    # nothing long enough: the whole buffer
    assert bench.fast_segments([193.0, 1.0, 193.0], set(), 100, 300, 150) == [(0, 300)]


def test_slot_ring_stays_inside_segments_and_wraps():
    # every request fits any segment (the bench keeps only runs at least one
    # largest request long)
    ring = bench.SlotRing([(300, 600), (700, 950)])
    sizes = (200, 200, 100, 200, 100, 250, 250)
    placed = [ring.place(nb) for nb in sizes]
    assert placed == [300, 700, 300, 400, 700, 300, 700]
    for p, nb in zip(placed, sizes):
        assert (300 <= p and p + nb <= 600) or (700 <= p and p + nb <= 950), (p, nb)
