"""Nested coarse-graining levels coupled pairwise (Sec. 2.3).

Level 0 is the coarsest and covers the whole domain; level k + 1 is embedded in
level k and coupled to it by coupler k (level k its coarse side, level k + 1 its
fine side).  A level in the middle is the fine side of one coupler and the
coarse side of the next, so it takes the sum of both couplers' controller
forces: every coupler runs in add mode on forces cleared at the start of each
coupling interval.

Levels may run different time steps (multi-rate): the time step may grow with the
coarse-graining ratio, since a coarser grain's contacts last longer (Sec. 3,
runtimes).  All couplers exchange at one common period T; a level with time step
dt_l advances T / dt_l steps per period (an integer), and coupler k counts its
interval in steps of its fine level (T / dt_{k+1}).

Host orchestration only: every step, measurement, controller and insertion
runs in the library's kernels through the C ABI.
"""
from __future__ import annotations

from . import dem


def period_steps(dts, intervals):
    """The common coupling period T and the steps each level takes per period: coupler k
    exchanges every intervals[k] steps of its fine level k + 1, so T = intervals[k] dts[k + 1]
    for every k, and level l advances T / dts[l] steps (a whole number)."""
    if len(intervals) != len(dts) - 1:
        raise ValueError("one coupling spec per pair of neighbouring levels")
    periods = [int(n) * dts[k + 1] for k, n in enumerate(intervals)]
    T = periods[0]
    if any(abs(p - T) > 1e-6 * T for p in periods):
        raise ValueError("all couplers must exchange at one period (interval x fine time step)")
    steps = []
    for dt in dts:
        n = int(round(T / dt))
        if n < 1 or abs(n * dt - T) > 1e-6 * T:
            raise ValueError(f"the coupling period {T:g} s is not a whole number of steps of {dt:g} s")
        steps.append(n)
    return T, steps


class Hierarchy:
    """Levels (single-instance DEM contexts, coarsest first) and the couplers between neighbours."""

    def __init__(self, levels, specs, steps_per_graph=True, lanes=0):
        if len(specs) != len(levels) - 1:
            raise ValueError("one coupling spec per pair of neighbouring levels")
        self.levels = list(levels)
        self.period, self.steps = period_steps([lv.dts[0] for lv in self.levels], [s["interval"] for s in specs])
        self.interval = self.steps[-1]          # steps of the finest level per period
        for lv in self.levels:
            lv.clear_external_force()
        self.couplers = [dem.Coupler(levels[k], levels[k + 1], **dict(s, add_forces=1)) for k, s in enumerate(specs)]
        for lv in self.levels:
            lv.set_step_lanes(lanes)             # 0: by size (small levels: fused steps, several lanes)
        if steps_per_graph:
            for lv, n in zip(self.levels, self.steps):
                lv.set_graph(n)
        self.calls = 0

    def advance(self, intervals=1):
        """Run `intervals` coupling periods: every level steps through one period, then the couplers
        measure, update their controllers, insert and remove, finest pair last."""
        for _ in range(intervals):
            for lv, n in zip(self.levels, self.steps):
                lv.step(n)
            for lv in self.levels:
                lv.clear_external_force()
            for cp in self.couplers:
                cp.couple()
            self.calls += 1
        return self

    def fields(self, lo, h, n):
        """Output fields on a uniform grid evaluated at the highest resolution available (Sec. 2.3):
        each cell takes the volume fraction, mass and Favre velocity of the finest level whose
        coupling region holds the cell's centre (level 0 elsewhere).  (n2, n1, n0, 5) CUDA tensor
        and the (n2, n1, n0) index of the level used."""
        import torch
        per = [lv.grid_fields(lo, h, n) for lv in self.levels]
        dev = per[0].device
        ax = [torch.arange(n[a], dtype=torch.float64, device=dev) * h + lo[a] + 0.5 * h for a in range(3)]
        zc, yc, xc = torch.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        which = torch.zeros(zc.shape, dtype=torch.int64, device=dev)
        for k, cp in enumerate(self.couplers):
            sp = cp.spec
            inside = ((xc >= sp.lo[0]) & (xc < sp.hi[0]) & (yc >= sp.lo[1]) & (yc < sp.hi[1]) &
                      (zc >= sp.lo[2]) & (zc < sp.hi[2]))
            which = torch.where(inside, torch.full_like(which, k + 1), which)
        out = torch.zeros_like(per[0])
        for k, f in enumerate(per):
            out = torch.where((which == k)[..., None], f, out)
        return out, which

    def counts(self):
        """Live particles per level."""
        return [int(lv.counts()[0][0]) for lv in self.levels]

    def close(self):
        for cp in self.couplers:
            cp.close()
        self.couplers = []
