"""Batched instances: one context advancing several independent boxes equals each box alone."""
import dataclasses

import numpy as np
import pytest

from paper_1705_03850_gb300 import autotune, dem, workloads

pytestmark = pytest.mark.gpu


def _boxes():
    mats = [workloads.Material(E=E, nu=0.25, e=e, mu=mu, rho=2500.0)
            for E, e, mu in ((5e6, 0.5, 0.2), (2e7, 0.9, 0.8), (5e7, 0.7, 0.5), (1e7, 0.6, 0.3))]
    shapes = [(5, 6, 4), (9, 7, 5), (4, 4, 3), (12, 10, 6)]
    return [workloads.dense_block(*sh, seed=40 + k, vel=0.4, mat=m) for k, (sh, m) in enumerate(zip(shapes, mats))]


def test_batched_context_equals_each_instance_alone_bitwise():
    wls = _boxes()
    ch = autotune.Choice(skin_factor=0.1, cell_factor=1.0, graph_steps=25, max_neighbors=32)
    both = autotune.make_context(wls, ch)
    both.step(1)
    both.set_graph(25)
    both.step(199)
    both.sync()
    assert both.stats()["rebuilds"] > 2 * len(wls)      # lists were rebuilt per instance while running
    x = both.read(dem.POS)
    w = both.read(dem.OMEGA)
    off = 0
    for wl in wls:
        one = autotune.make_context([wl], ch)
        one.step(1)
        one.set_graph(25)
        one.step(199)
        one.sync()
        assert np.array_equal(one.read(dem.POS), x[off:off + wl.n])
        assert np.array_equal(one.read(dem.OMEGA), w[off:off + wl.n])
        off += wl.n


def test_autotuner_returns_a_working_choice():
    wls = workloads.batch(12, seed=4, scale=0.02)
    best, allc = autotune.tune(wls, skin_factors=(0.05, 0.1), cell_factors=(1.0,), graph_steps=(25,), window=50,
                               sample=6)
    assert best.ok and best.ms_per_step > 0
    assert len(allc) == 4                  # two skins at 128 threads, then 64 and 256 for the better one
    assert best.block in (64, 128, 256)
    assert sorted(c.block for c in allc) == [64, 128, 128, 256]
    assert all(c.lanes == 1 for c in allc)  # a subset of the instances: no lanes stage
    sim = autotune.make_context(wls, best)
    sim.step(1)
    sim.set_graph(best.graph_steps)
    sim.step(50)
    assert sim.status() == 0


def test_batched_instances_each_match_the_oracle():
    # four boxes of 120, 315, 48 and 720 spheres (none a multiple of the 128-slot tile) with their
    # own (E, e, mu), in one context: CUDA graphs of 25 steps, a skin of 1 % of d so that every box
    # rebuilds its lists inside the graphs several times; each box against its own oracle run at
    # the 100-step bar (positions within max(1e-4 d, 64 ulp_fp32(|x|)))
    from _util import min_image, oracle_sim
    wls = _boxes()
    ch = autotune.Choice(skin_factor=0.01, cell_factor=1.0, graph_steps=25, max_neighbors=32)
    sim = autotune.make_context(wls, ch)
    sim.step(1)
    sim.set_graph(25)
    sim.step(99)
    sim.sync()
    assert sim.stats()["rebuilds"] >= 3 * len(wls)
    x = sim.read(dem.POS)
    off = 0
    for wl in wls:
        o = oracle_sim(wl).run(100)
        d = min_image(x[off:off + wl.n] - o.x, wl)
        tol = np.maximum(1e-4 * 2 * wl.r[:, None], 64 * np.spacing(np.abs(o.x).astype(np.float32)).astype(np.float64))
        assert (np.abs(d) <= tol).all(), (wl.n, np.abs(d).max())
        off += wl.n
    # the materials differ enough that a box run with another's (E, e, mu) would fail the bar
    o_wrong = oracle_sim(dataclasses.replace(wls[1], material=wls[2].material)).run(100)
    d = min_image(x[wls[0].n:wls[0].n + wls[1].n] - o_wrong.x, wls[1])
    assert np.abs(d).max() > 1e-4 * 2 * wls[1].r.max()


@pytest.mark.parametrize("threads", [64, 256])
def test_step_block_size_does_not_change_the_run(threads):
    # every particle sums its own row in row order whatever the block size: the same bits
    wls = _boxes()
    ch = autotune.Choice(skin_factor=0.05, cell_factor=1.0, graph_steps=25, max_neighbors=32)
    runs = []
    for c in (ch, dataclasses.replace(ch, block=threads)):
        sim = autotune.make_context(wls, c)
        sim.step(1)
        sim.set_graph(25)
        sim.step(150)
        sim.sync()
        runs.append((sim.read(dem.POS), sim.read(dem.OMEGA), sim.stats()["rebuilds"]))
    assert runs[0][2] > len(wls)
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_autotuner_tries_lanes_when_every_instance_is_sampled():
    wls = workloads.batch(3, seed=5, scale=0.02)
    best, allc = autotune.tune(wls, skin_factors=(0.05,), cell_factors=(1.0,), graph_steps=(25,), window=50,
                               sample=6)
    assert sorted((c.block, c.lanes) for c in allc) == [(64, 1), (128, 1), (128, 2), (128, 4), (128, 8), (256, 1)]
    assert best.ok and all(c.ok for c in allc)
    sim = autotune.make_context(wls, best)
    assert sim.stats()["step_lanes"] == best.lanes and sim.stats()["step_threads"] == best.block


@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_lanes_per_particle_match_the_oracle_and_repeat_bitwise(lanes):
    # the multi-lane step kernel (each lane a share of the row, partial sums combined in a fixed
    # order): graph and direct runs give the same bits, and every box meets the 100-step bar
    # against its own oracle run, with the lists rebuilt inside the graphs
    from _util import min_image, oracle_sim
    wls = _boxes()
    ch = autotune.Choice(skin_factor=0.01, cell_factor=1.0, graph_steps=25, max_neighbors=32, lanes=lanes)
    runs = []
    for graph in (25, 0):
        sim = autotune.make_context(wls, ch)
        sim.step(1)
        sim.set_graph(graph)
        sim.step(99)
        sim.sync()
        st = sim.stats()
        assert st["step_lanes"] == lanes and st["rebuilds"] >= 3 * len(wls)
        runs.append((sim.read(dem.POS), sim.read(dem.OMEGA)))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    x = runs[0][0]
    off = 0
    for wl in wls:
        o = oracle_sim(wl).run(100)
        d = min_image(x[off:off + wl.n] - o.x, wl)
        tol = np.maximum(1e-4 * 2 * wl.r[:, None], 64 * np.spacing(np.abs(o.x).astype(np.float32)).astype(np.float64))
        assert (np.abs(d) <= tol).all(), (wl.n, np.abs(d).max())
        off += wl.n


def test_lanes_are_chosen_by_size():
    # 0 = by size: several lanes for a context far smaller than the GPU's resident threads, one
    # lane for a large one; other block sizes keep one lane
    small = dem.from_workload(workloads.dense_block(6, 6, 4, seed=3))
    small.set_step_lanes(0)
    assert small.stats()["step_lanes"] == 8
    big = dem.from_workload(workloads.shear_bed(200_000, seed=2))
    big.set_step_lanes(0)
    assert big.stats()["step_lanes"] == 1
    mid = dem.from_workload(workloads.shear_bed(40_000, seed=2))  # 314 tiles: fused steps, two lanes
    mid.set_step_lanes(0)
    assert mid.stats()["step_lanes"] == 2
    small.set_step_lanes(1).set_step_block(64)
    small.set_step_lanes(0)
    assert small.stats()["step_lanes"] == 1
    with pytest.raises(dem.DemError):
        small.set_step_lanes(4)              # more than one lane needs the 128-thread block
    with pytest.raises(dem.DemError):
        small.set_step_lanes(3)
