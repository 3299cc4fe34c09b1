"""Batched instances: one context advancing several independent boxes equals each box alone."""
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
    assert len(allc) == 2
    sim = autotune.make_context(wls, best)
    sim.step(1)
    sim.set_graph(best.graph_steps)
    sim.step(50)
    assert sim.status() == 0
