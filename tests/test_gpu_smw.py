"""SM-wide step blocks (896 threads, one block per SM, warps claiming the slices of a contiguous
range of the tiles that hold live slots from a shared counter): chosen by default for a single
instance with at least four slices for every resident warp, and the same bits as every other
block size (each particle sums its own row in row order), with and without walls, with spare
capacity, in graphs with in-graph list builds and in direct launches.  The oracle parity of the
path itself is in the full-size test of test_gpu_parity.py, which takes these blocks by default.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_1705_03850_gb300 import dem, workloads

pytestmark = pytest.mark.gpu


def _run(wl, threads, graph=25, steps=150, walls=None, z_remove=-math.inf, capacity=None):
    sim = dem.DEM([dem.desc_from_workload(wl, capacity=capacity)], max_neighbors=32)
    sim.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    if walls is not None:
        sim.set_walls(0, (0.0, 0.0), walls, z_remove)
    sim.set_step_block(threads)
    sim.step(1)
    if graph:
        sim.set_graph(graph)
    sim.step(steps)
    sim.sync()
    st = sim.stats()
    out = (sim.read(dem.POS), sim.read(dem.VEL), sim.read(dem.OMEGA), st["rebuilds"], st["step_threads"])
    assert sim.status() == 0
    sim.close()
    return out


def test_chosen_for_a_large_single_instance_and_the_same_bits_as_other_block_sizes():
    # 600,000 spheres in motion (4,688 tiles: more than four slices for each of the 152 x 28
    # resident warps) with a skin small enough for several list builds inside the graphs
    wl = workloads.dense_block(100, 100, 60, seed=31, vel=0.3)
    wl = dataclasses.replace(wl, skin=0.03 * 2 * float(wl.r.max()))
    auto = _run(wl, 0)
    assert auto[4] == 896
    assert auto[3] >= 3
    for threads in (128, 256, 896):
        other = _run(wl, threads)
        assert other[4] == threads
        for a, b in zip(auto[:4], other[:4]):
            assert np.array_equal(a, b), threads


@pytest.mark.parametrize("spare", [1, 3])
def test_direct_launches_a_small_instance_and_spare_capacity(spare):
    # 9,216 spheres (72 tiles: fewer tiles than SMs, so each block takes one tile), in a context
    # of their size or of three times their size (the blocks share only the tiles holding live
    # slots): the automatic choice stays at 128 threads; explicit SM-wide blocks give the same
    # bits, graph or not
    wl = workloads.dense_block(24, 24, 16, seed=5, vel=0.4)
    wl = dataclasses.replace(wl, skin=0.02 * 2 * float(wl.r.max()))
    cap = spare * wl.n
    ref = _run(wl, 0, capacity=cap)
    assert ref[4] == 128
    for graph in (0, 25):
        got = _run(wl, 896, graph=graph, capacity=cap)
        assert got[4] == 896
        for a, b in zip(ref[:4], got[:4]):
            assert np.array_equal(a, b), graph


def test_with_walls_and_removal():
    # the packed vessel draining through its orifice: wall contacts, removal below the orifice
    wl = workloads.small_vessel(seed=23, n=900, closed=False)
    walls = wl.meta["walls"]
    ref = _run(wl, 128, steps=400, walls=walls, z_remove=0.005)
    got = _run(wl, 896, steps=400, walls=walls, z_remove=0.005)
    for a, b in zip(ref[:4], got[:4]):
        assert np.array_equal(a, b)


def test_refused_for_batched_contexts_and_other_sizes():
    boxes = [workloads.dense_block(5, 6, 4, seed=40), workloads.dense_block(4, 4, 3, seed=41)]
    sim = dem.DEM([dem.desc_from_workload(b) for b in boxes], max_neighbors=32)
    with pytest.raises(dem.DemError):
        sim.set_step_block(896)
    with pytest.raises(dem.DemError):
        sim.set_step_block(512)
    assert sim.stats()["step_threads"] == 128
    sim.close()
