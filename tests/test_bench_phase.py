"""Host logic of bench.py: placing the timed mpcd_step(n) call in the replay
cycle.  The fake context below follows the library's rule for the re-sort
counter (each of a call's n - 1 fused passes increments it; reaching the sort
period re-sorts, which resets it and swaps the solvent buffers), and records a
CUDA graph per (n, buffer parity, counter) key as mpcd_step does; the GPU test
test_resorts_per_call_follow_the_fused_pass_count checks that rule on the
library itself."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class FakeContext:
    def __init__(self, period):
        self.period, self.since, self.par = period, 0, 0
        self.graphs = set()
        self.last_sorts, self.last_replayed = 0, False

    def step(self, n):
        key = (n, self.par, self.since)
        self.last_replayed = key in self.graphs
        self.graphs.add(key)
        sorts = 0
        for _ in range(n - 1):
            self.since += 1
            if self.since >= self.period:
                self.since, self.par = 0, self.par ^ 1
                sorts += 1
        self.last_sorts = sorts


@pytest.mark.parametrize("period", [1, 2, 3, 4, 7, 20, 33])
def test_timed_call_replays_and_holds_its_share_of_resorts(period):
    for n in range(1, 130):
        ctx = FakeContext(period)
        share = bench.place_timed_call(lambda: ctx.step(n), n, period)
        ctx.step(n)   # the timed call
        assert share == (-(-(n - 1) // period) if n >= 2 else 0), (n, period)
        assert ctx.last_sorts == share, (n, period, ctx.last_sorts, share)
        if n >= 2:
            assert ctx.last_replayed, (n, period)


def test_call_right_after_a_resort_holds_none():
    """The placement matters: from the state right after a re-sort, a 20-step
    call with period 20 re-sorts zero times."""
    ctx = FakeContext(20)
    ctx.step(20)
    assert ctx.last_sorts == 0
    ctx.step(20)
    assert ctx.last_sorts == 1
