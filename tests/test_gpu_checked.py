"""The bounds-checked build (the step kernel's gathered particle indices and the list build's
cell codes and candidate ranges tested against the capacity in the kernels) runs the same bits
as the plain build and finds no index out of range: a dense block in motion with lists rebuilt
inside CUDA graphs, three batched boxes, and three coupled chute levels with insertion and
removal.  Also: a position outside the fixed-point range is reported, not wrapped.
"""
import dataclasses
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1705_03850_gb300 import dem, levels, workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = dict(length=0.3, width=0.06, height=0.1, bed=0.04, regions=((0.1, 0.12), (0.14, 0.04)))


def _runs():
    """Positions and status after each run; called in this process (plain build) and in a child
    with CGDEM_CHECKED=1 (checked build)."""
    out = {}
    wl = workloads.dense_block(24, 24, 16, seed=5, vel=0.4)             # 9,216 spheres in motion
    wl = dataclasses.replace(wl, skin=0.02 * 2 * float(wl.r.max()))     # lists rebuilt every ~50 steps
    sim = dem.from_workload(wl)
    sim.step(1)
    sim.set_graph(25)
    sim.step(299)
    sim.sync()
    out["bed_x"] = sim.read(dem.POS)
    out["bed_rebuilds"] = np.array(sim.stats()["rebuilds"])
    out["bed_status"] = np.array(sim.status())

    boxes = [workloads.dense_block(*sh, seed=40 + k, vel=0.4) for k, sh in enumerate([(5, 6, 4), (9, 7, 5), (4, 4, 3)])]
    sim = dem.DEM([dem.desc_from_workload(b) for b in boxes], max_neighbors=32)
    sim.write_state(np.concatenate([b.x for b in boxes]), np.concatenate([b.v for b in boxes]),
                    np.concatenate([b.w for b in boxes]), np.concatenate([b.r for b in boxes]),
                    np.concatenate([b.m for b in boxes]))
    sim.step(200).sync()
    out["box_x"] = sim.read(dem.POS)
    out["box_status"] = np.array(sim.status())

    lv, specs = workloads.chute(**SMALL, u0=10.0, interval=15)
    ctx = []
    for k, w in enumerate(lv):
        cap = None if k == 0 else w.n + 20000
        d = dem.DEM([dem.desc_from_workload(w, capacity=cap)], max_neighbors=24)
        v = np.zeros_like(w.v)
        v[:, 0] = 10.0
        d.write_state(w.x, v, w.w, w.r, w.m)
        ctx.append(d)
    h = levels.Hierarchy(ctx, specs, steps_per_graph=True)
    h.advance(12)
    for k, lvl in enumerate(h.levels):
        out[f"lv{k}_x"] = np.nan_to_num(lvl.read(dem.POS), nan=-1e30)
        out[f"lv{k}_status"] = np.array(lvl.status())
    out["counts"] = np.array(h.counts(), dtype=np.int64)
    return out


def test_checked_build_runs_the_same_bits_and_finds_no_index_out_of_range(tmp_path):
    if not os.path.exists(os.path.join(ROOT, "paper_1705_03850_gb300", "_build", "libcgdem_checked.so")):
        pytest.fail("bounds-checked library not built (build_all)")
    dst = tmp_path / "checked.npz"
    code = ("import sys, numpy as np; sys.path[:0] = [%r, %r]; import test_gpu_checked as t; "
            "np.savez(%r, **t._runs())" % (ROOT, os.path.join(ROOT, "tests"), str(dst)))
    env = dict(os.environ, CGDEM_CHECKED="1")
    subprocess.run([sys.executable, "-c", code], check=True, env=env, timeout=600)
    checked = dict(np.load(dst))
    plain = _runs()
    assert set(checked) == set(plain)
    for k in plain:
        if k.endswith("status"):
            assert int(checked[k]) == 0 and int(plain[k]) == 0, (k, int(checked[k]), int(plain[k]))
    assert int(plain["bed_rebuilds"]) > 2
    for k in plain:
        assert np.array_equal(checked[k], plain[k]), k


def test_position_beyond_the_fixed_point_range_is_reported():
    # a finite position far outside the box cannot be held in the 32-bit integer coordinates:
    # the write flags it (DEM_ERR_ESCAPED) instead of wrapping it into the box
    wl = workloads.dense_block(6, 6, 4, seed=22)
    x = wl.x.copy()
    x[7, 2] = 1.0e9
    sim = dem.DEM([dem.desc_from_workload(wl)])
    sim.write_state(x, wl.v, wl.w, wl.r, wl.m)
    sim.step(1)
    assert sim.status() == 5  # DEM_ERR_ESCAPED
