"""Fused steps (one cooperative launch runs the steps between list builds, with a grid barrier
between steps) compute exactly what one launch per step computes: the same bits with walls and
removal, for batched instances, across graph launches with a list build pending, and with the
automatic choice (fused only when every tile's block is resident at once)."""
import math

import numpy as np
import pytest

from paper_1705_03850_gb300 import autotune, dem, workloads

pytestmark = pytest.mark.gpu


def _pair(make, steps, graph, rounds=1, lanes=1):
    out = []
    for mode in (1, 2):
        sim = make()
        sim.set_step_lanes(lanes)
        sim.step(1)
        sim.set_graph_mode(mode)
        sim.set_graph(graph)
        for _ in range(rounds):
            sim.step(steps)
        sim.sync()
        st = sim.stats()
        assert st["graph_fused"] == (mode == 2)
        out.append((sim, st))
    return out


def _same(a, b, fields=(dem.POS, dem.VEL, dem.OMEGA)):
    for f in fields:
        xa, xb = a.read(f), b.read(f)
        assert np.array_equal(np.isnan(xa), np.isnan(xb))
        assert np.array_equal(np.nan_to_num(xa), np.nan_to_num(xb)), f


@pytest.mark.parametrize("lanes", [1, 4])
def test_fused_steps_with_walls_and_removal_equal_one_launch_per_step(lanes):
    wl = workloads.small_vessel(seed=24)
    walls = wl.meta["walls"][1:]                             # orifice open
    z_rem = wl.meta["z_o"] - 0.004

    def make():
        sim = dem.from_workload(wl)
        sim.set_walls(0, (0.0, 0.0), walls, z_rem)
        return sim
    (a, sa), (b, sb) = _pair(make, 4000, 50, lanes=lanes)
    assert sa["step_lanes"] == sb["step_lanes"] == lanes
    assert sa["rebuilds"] == sb["rebuilds"] > 5
    _same(a, b)
    assert a.wall_removed() == b.wall_removed()


@pytest.mark.parametrize("lanes", [1, 2])
def test_fused_steps_of_batched_instances_equal_one_launch_per_step(lanes):
    wls = [workloads.dense_block(*sh, seed=40 + k, vel=0.4) for k, sh in enumerate([(5, 6, 4), (9, 7, 5), (4, 4, 3)])]
    ch = autotune.Choice(skin_factor=0.01, cell_factor=1.0, graph_steps=25, max_neighbors=32)
    (a, sa), (b, sb) = _pair(lambda: autotune.make_context(wls, ch), 50, 25, rounds=4, lanes=lanes)
    assert sa["rebuilds"] == sb["rebuilds"] >= 3 * len(wls)
    _same(a, b)


def test_graph_length_not_dividing_the_steps_and_a_pending_build():
    # 37-step graphs for 200 steps: graph launches, then direct steps for the rest; a list build
    # is often pending across the boundaries
    wl = workloads.dense_block(10, 10, 6, seed=14, vel=0.5)
    (a, sa), (b, sb) = _pair(lambda: dem.from_workload(wl), 200, 37, rounds=3)
    assert sa["rebuilds"] == sb["rebuilds"] > 5
    _same(a, b)


def test_fused_steps_are_chosen_by_size():
    small = dem.from_workload(workloads.dense_block(6, 6, 4, seed=3))
    small.set_graph(20)
    assert small.stats()["graph_fused"] == 1
    small.set_step_lanes(0)                                 # by size: fused steps with 8 lanes
    assert small.stats()["step_lanes"] == 8 and small.stats()["graph_fused"] == 1
    small.set_step_lanes(1).set_step_block(64)              # fused steps need 128-thread blocks
    assert small.stats()["graph_fused"] == 0
    with pytest.raises(dem.DemError):
        small.set_graph_mode(2)
    assert small.stats()["graph_fused"] == 0                # the previous graph is kept
    big = dem.from_workload(workloads.shear_bed(400_000, seed=2))
    big.set_graph(20)
    assert big.stats()["graph_fused"] == 0                  # more tiles than resident blocks
    big.set_graph_mode(2)                                   # fused on request: blocks walk several tiles
    assert big.stats()["graph_fused"] == 1


def test_fused_steps_with_several_tiles_per_block_equal_one_launch_per_step():
    # more tiles than resident blocks: each block of the cooperative launch walks a range of tiles
    wl = workloads.shear_bed(300_000, seed=2)
    (a, sa), (b, sb) = _pair(lambda: dem.from_workload(wl), 100, 50, rounds=2)
    _same(a, b)


def test_spare_capacity_changes_nothing_and_steps_only_live_tiles():
    # a context with ten times the slots it holds walks only the tiles with live particles: the
    # same bits as a context without spare slots, and fused steps chosen by the live tiles
    wl = workloads.dense_block(40, 40, 20, seed=9, vel=0.3)       # 32,000 spheres
    runs = []
    for cap in (None, 10 * wl.n):
        sim = dem.DEM([dem.desc_from_workload(wl, capacity=cap)])
        sim.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
        sim.step(1)
        sim.set_graph(25)
        assert sim.stats()["graph_fused"] == 1
        sim.step(200).sync()
        runs.append((sim.read(dem.POS), sim.read(dem.VEL), sim.stats()["rebuilds"]))
    assert runs[0][2] == runs[1][2] > 1
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_a_barrier_wait_that_runs_out_is_reported_not_hung():
    # one block of a fused launch leaves without arriving at the barrier (a test hook): the
    # other blocks give up after about a second and the host reads DEM_ERR_TIMEOUT
    import time
    wl = workloads.dense_block(20, 20, 12, seed=3, vel=0.2)           # 4,800 spheres: 38 blocks
    sim = dem.from_workload(wl)
    sim.step(1)
    sim.set_graph(25)
    assert sim.stats()["graph_fused"] == 1
    sim.step(50).sync()
    sim.test_stall_barrier()
    t0 = time.perf_counter()
    sim.step(25)
    assert sim.status() == 6                                           # DEM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
