"""Nested coarse-graining levels coupled pairwise (Sec. 2.3).

Level 0 is the coarsest and covers the whole domain; level k + 1 is embedded in
level k and coupled to it by coupler k (level k its coarse side, level k + 1 its
fine side).  A level in the middle is the fine side of one coupler and the
coarse side of the next, so it takes the sum of both couplers' controller
forces: every coupler runs in add mode on forces cleared at the start of each
coupling interval.  All levels share one time step (no sub-cycling).

Host orchestration only: every step, measurement, controller and insertion
runs in the library's kernels through the C ABI.
"""
from __future__ import annotations

from . import dem


class Hierarchy:
    """Levels (single-instance DEM contexts, coarsest first) and the couplers between neighbours."""

    def __init__(self, levels, specs, steps_per_graph=True):
        if len(specs) != len(levels) - 1:
            raise ValueError("one coupling spec per pair of neighbouring levels")
        intervals = {int(s["interval"]) for s in specs}
        if len(intervals) != 1:
            raise ValueError("all couplers must share one coupling interval")
        self.interval = intervals.pop()
        self.levels = list(levels)
        for lv in self.levels:
            lv.clear_external_force()
        self.couplers = [dem.Coupler(levels[k], levels[k + 1], **dict(s, add_forces=1)) for k, s in enumerate(specs)]
        if steps_per_graph:
            for lv in self.levels:
                lv.set_graph(self.interval)
        self.calls = 0

    def advance(self, intervals=1):
        """Run `intervals` coupling intervals: every level steps `interval` times, then the couplers
        measure, update their controllers, insert and remove, finest pair last."""
        for _ in range(intervals):
            for lv in self.levels:
                lv.step(self.interval)
            for lv in self.levels:
                lv.clear_external_force()
            for cp in self.couplers:
                cp.couple()
            self.calls += 1
        return self

    def counts(self):
        """Live particles per level."""
        return [int(lv.counts()[0][0]) for lv in self.levels]

    def close(self):
        for cp in self.couplers:
            cp.close()
        self.couplers = []
