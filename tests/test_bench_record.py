"""The bench's `traffic` figure comes from the committed ncu summary of the
query step (the windowed passes of one chunk).  That record names the sha of
the kernels' sources and the L2 fetch granularity it was captured at; both
must match what bench.py runs, else the figure would describe other kernels."""
from __future__ import annotations

import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_traffic_record_matches_the_current_query_kernel():
    default_gran = bench.parse_defaults()["l2_fetch_granularity"]
    per_launch = bench.recorded_traffic(10**9, 10**9, default_gran)
    assert per_launch is not None, "recapture the query kernel: its sources changed since the record"
    # The DRAM bytes per key must exceed the algorithmic minimum (8 key + 4 result + one pilot byte).
    assert 13e9 < per_launch < 200e9


def test_traffic_record_is_refused_at_another_granularity_or_structure():
    assert bench.recorded_traffic(10**9, 10**9, 32) is None
    assert bench.recorded_traffic(10**8, 10**8, 128) is None   # a smaller structure: other bytes per key
    assert bench.recorded_traffic(10**9, 2**26, 128) == 62.39 * 2**26
