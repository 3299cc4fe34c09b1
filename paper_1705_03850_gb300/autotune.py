"""Autotuner for multi-instance (batched) runs.

Chooses the neighbour-list skin (the rebuild interval), the cell width, the
number of steps captured per CUDA graph, the list width, the step kernel's
block size (64, 128 or 256 threads) and its lanes per particle (1, 2, 4 or 8) by timing each
candidate through the C ABI on a representative subset of the instances
(evenly spread over their sizes) for the run's full length, so that the cost of
list rebuilds is part of what is measured: create a context, load the same
state, time the start-up step (including the first list build) and the
remaining steps, and keep the fastest candidate that ran without a device
error.  The block size is searched second, for the best of the other settings
(the other settings change the work; the block size only how it is spread), and
the lanes per particle last, at 128 threads, when every instance is in the sample
(how many lanes pay depends on how many particles the whole context holds).
"""
from __future__ import annotations

import itertools
import time
from dataclasses import dataclass

import numpy as np

from . import dem


@dataclass
class Choice:
    skin_factor: float      # skin = skin_factor * d (d = 2 r_max of each instance)
    cell_factor: float      # cell width >= cell_factor * 2 r_max + skin
    graph_steps: int
    max_neighbors: int
    block: int = 128        # threads per block of the step kernel
    lanes: int = 1          # lanes per particle of the step kernel
    ms_start: float = float("nan")
    ms_per_step: float = float("nan")
    ok: bool = False

    def as_dict(self):
        return dict(skin_factor=self.skin_factor, cell_factor=self.cell_factor, graph_steps=self.graph_steps,
                    max_neighbors=self.max_neighbors, block=self.block, lanes=self.lanes, ms_start=self.ms_start,
                    ms_per_step=self.ms_per_step)


def descs_for(workloads, choice: Choice, floor_v=None):
    out = []
    for wl in workloads:
        rmax = float(np.max(wl.r)) if wl.n else 1e-3
        d = dem.desc_from_workload(wl, r_max=rmax * choice.cell_factor)
        d.skin = choice.skin_factor * 2.0 * rmax
        if floor_v is not None:
            for a in range(3):
                d.floor_v[a] = floor_v[a]
        out.append(d)
    return out


def concat_state(workloads):
    cat = lambda f: np.concatenate([getattr(w, f) for w in workloads]) if workloads else np.zeros((0, 3))
    return cat("x"), cat("v"), cat("w"), cat("r"), cat("m")


def make_context(workloads, choice: Choice, device=None, state=None):
    sim = dem.DEM(descs_for(workloads, choice), max_neighbors=choice.max_neighbors, device=device)
    sim.set_step_block(choice.block)
    sim.set_step_lanes(choice.lanes)
    x, v, w, r, m = state if state is not None else concat_state(workloads)
    sim.write_state(x, v, w, r, m)
    return sim


def subset_indices(workloads, count):
    """Indices of `count` instances evenly spread over the sizes (all of them if fewer)."""
    if len(workloads) <= count:
        return list(range(len(workloads)))
    order = sorted(range(len(workloads)), key=lambda k: workloads[k].n)
    return sorted({order[int(round(i * (len(order) - 1) / (count - 1)))] for i in range(count)})


def subset(workloads, count):
    """`count` instances evenly spread over the sizes (all of them if fewer)."""
    return [workloads[k] for k in subset_indices(workloads, count)]


def tune(workloads, skin_factors=(0.025, 0.05, 0.1), cell_factors=(1.0, 1.25), graph_steps=(50, 100),
         max_neighbors=(32,), blocks=(64, 128, 256), lanes=(1, 2, 4, 8), window=2000, sample=32, device=None,
         state=None, log=None):
    """Time every candidate on `sample` instances for `window` steps; return (best, all).
    The other settings are searched at 128 threads per block and one lane per particle, then
    `blocks` for the best of them, then `lanes` at 128 threads if every instance is sampled.
    `state`, if given, is the concatenated (x, v, w, r, m) of all the workloads (e.g. after settling);
    the sampled instances start from their part of it, otherwise from their own inputs."""
    import torch
    picked = subset_indices(workloads, sample)
    whole = len(picked) == len(workloads)
    if state is not None:
        off = np.concatenate([[0], np.cumsum([w.n for w in workloads])])
        rows = torch.as_tensor(np.concatenate([np.arange(off[k], off[k + 1]) for k in picked]),
                               device=state[0].device)
        state = [torch.as_tensor(a).index_select(0, rows) for a in state]
    workloads = [workloads[k] for k in picked]
    if state is None:
        state = [torch.as_tensor(a, dtype=torch.float64, device=device or "cuda") for a in concat_state(workloads)]
    results = []

    def run(ch):
        sim = None
        try:
            sim = make_context(workloads, ch, device=device, state=state)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.step(1)
            sim.sync()
            ch.ms_start = (time.perf_counter() - t0) * 1e3
            gs = ch.graph_steps
            sim.set_graph(gs)
            n = max(gs, (window // gs) * gs)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(sim.stream)
            sim.step(n)
            ev1.record(sim.stream)
            sim.sync()
            ch.ms_per_step = ev0.elapsed_time(ev1) / n
            ch.ok = True
        except dem.DemError as e:
            ch.ok = False
            if log:
                log(f"candidate {ch.as_dict()} rejected: {e}")
        finally:
            if sim is not None:
                sim.close()
        results.append(ch)
        if log:
            log(f"candidate {ch.as_dict()} ok={ch.ok}")
        return ch

    cost = lambda c: c.ms_start + c.ms_per_step * window
    for sf, cf, gs, lm in itertools.product(skin_factors, cell_factors, graph_steps, max_neighbors):
        run(Choice(sf, cf, gs, lm, 128))
    good = [c for c in results if c.ok]
    if not good:
        raise RuntimeError("no autotuner candidate ran without a device error")
    best = min(good, key=cost)
    for b in blocks:
        if b != best.block:
            run(Choice(best.skin_factor, best.cell_factor, best.graph_steps, best.max_neighbors, b))
    best = min((c for c in results if c.ok), key=cost)
    if whole:
        base = next(c for c in results if c.ok and c.block == 128 and c.lanes == 1 and
                    (c.skin_factor, c.cell_factor, c.graph_steps, c.max_neighbors) ==
                    (best.skin_factor, best.cell_factor, best.graph_steps, best.max_neighbors))
        for ln in lanes:
            if ln != 1:
                run(Choice(base.skin_factor, base.cell_factor, base.graph_steps, base.max_neighbors, 128, ln))
        best = min((c for c in results if c.ok), key=cost)
    return best, results
