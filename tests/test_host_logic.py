"""Host-side logic that needs no GPU: the multi-rate period arithmetic of the level
hierarchy and the autotuner's instance sampling and per-candidate descriptors."""
import numpy as np
import pytest

from paper_1705_03850_gb300 import autotune, levels, workloads


def test_single_rate_levels_step_the_interval():
    T, steps = levels.period_steps([1e-6, 1e-6, 1e-6], [15, 15])
    assert T == pytest.approx(15e-6) and steps == [15, 15, 15]


def test_multi_rate_levels_take_whole_steps_of_one_period():
    # time steps scaled with the grain (8, 4, 2 mm: 4, 2, 1 us), coupling every 16 finest steps
    T, steps = levels.period_steps([4e-6, 2e-6, 1e-6], [8, 16])
    assert T == pytest.approx(16e-6) and steps == [4, 8, 16]
    # five nested levels, alpha 16 .. 1
    T, steps = levels.period_steps([16e-6, 8e-6, 4e-6, 2e-6, 1e-6], [2, 4, 8, 16])
    assert steps == [1, 2, 4, 8, 16]


def test_inconsistent_periods_are_refused():
    with pytest.raises(ValueError):
        levels.period_steps([4e-6, 2e-6, 1e-6], [15, 15])      # 30 us and 15 us
    with pytest.raises(ValueError):
        levels.period_steps([4e-6, 1e-6], [15])                # 15 us is not whole 4 us steps
    with pytest.raises(ValueError):
        levels.period_steps([1e-6, 1e-6], [15, 15])            # one spec per neighbouring pair


def test_workload_specs_give_consistent_periods():
    lv, specs = workloads.chute(length=0.3, width=0.06, height=0.1, bed=0.04,
                                regions=((0.1, 0.12), (0.14, 0.04)), multirate=True, interval=16)
    T, steps = levels.period_steps([w.dt for w in lv], [s["interval"] for s in specs])
    assert steps == [4, 8, 16]
    for w, n in zip(lv, steps):
        assert n * w.dt == pytest.approx(T, rel=1e-6)


def test_autotune_samples_spread_over_the_sizes():
    wls = workloads.batch(256, seed=4, scale=0.01)
    idx = autotune.subset_indices(wls, 32)
    assert len(idx) == 32 and idx == sorted(set(idx))
    n = np.array([wls[k].n for k in idx])
    all_n = np.array([w.n for w in wls])
    assert n.min() == all_n.min() and n.max() == all_n.max()      # both ends of the size range
    assert autotune.subset_indices(wls[:5], 32) == list(range(5))


def test_autotune_descriptors_follow_the_candidate():
    wls = workloads.batch(4, seed=4, scale=0.01)
    c = autotune.Choice(skin_factor=0.05, cell_factor=1.25, graph_steps=50, max_neighbors=32)
    for w, d in zip(wls, autotune.descs_for(wls, c)):
        rmax = float(np.max(w.r))
        assert d.skin == pytest.approx(0.05 * 2 * rmax)
        assert d.r_max == pytest.approx(1.25 * rmax)
        assert d.n == w.n
    x, v, wv, r, m = autotune.concat_state(wls)
    assert x.shape == (sum(w.n for w in wls), 3) and r.shape == (x.shape[0],)
