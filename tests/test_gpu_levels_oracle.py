"""Coupled levels on the GPU against the FP64 oracle driven in the same schedule (Sec. 2.3 with
time steps scaled by the grain, Sec. 3 runtimes).

Two levels (4 and 2 mm, time steps 2 and 1 us: two fine steps per coarse step) and three nested
levels (8, 4 and 2 mm; 4, 2 and 1 us) of a short chute, the finest bed started compressed (every
neighbour pair in contact), plug flow fast enough that lattice planes of the coarser level cross
the feed face: the library's hierarchy (CUDA graphs of one period per level, couplers in add
mode) against oracle.Sim and oracle.Coupler in the schedule of tests/_coupled_oracle.py.

Compared: IDs handed out and removed per level (exact); per call and surface cell the
inserted counts and carried mass (exact: no insertion decision within the borderline band of
4 q occurs, which the oracle reports); positions of every particle, matched by ID, within the
100-step bar max(1e-4 d, 64 ulp_fp32(|x|)); and at the first call the held controller forces
within the bound that float rounding of the Eq. 7 stresses allows (1e-5 of each cell's stress
scale times K_p + K_i T_c, times pi r^2) and of the cell velocities (1e-6 relative).
"""
import dataclasses

import numpy as np
import pytest

from paper_1705_03850_gb300 import dem, levels, workloads
from _coupled_oracle import OracleLevels
from _util import min_image, oracle_params

pytestmark = pytest.mark.gpu

TWO = dict(length=0.1, width=0.03, height=0.06, bed=0.025, regions=((0.03, 0.04),), diameters=(4e-3, 2e-3))
THREE = dict(length=0.16, width=0.03, height=0.06, bed=0.025, regions=((0.04, 0.08), (0.06, 0.03)),
             diameters=(8e-3, 4e-3, 2e-3))


def _run(cfg, u0, periods):
    lv, specs = workloads.chute(**cfg, u0=u0, multirate=True, interval=16, gap=-3e-6)
    start = []
    for wl in lv:
        v = np.zeros_like(wl.v)
        v[:, 0] = workloads.f32(u0)
        start.append(dataclasses.replace(wl, v=v))
    ctx = []
    for k, wl in enumerate(start):
        d = dem.DEM([dem.desc_from_workload(wl, capacity=None if k == 0 else wl.n + 20000)], max_neighbors=24)
        d.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
        ctx.append(d)
    h = levels.Hierarchy(ctx, specs, steps_per_graph=True)
    o = OracleLevels([oracle_params(wl) for wl in start], start, specs)
    assert h.steps == o.steps
    first = None
    for call in range(periods):
        h.advance(1)
        o.advance(1)
        for k, cp in enumerate(h.couplers):
            out = o.outs[-1][k]
            assert np.all(out["border"] < 0), f"borderline insertion decision at call {call}"
            mu = specs[k]["mass_unit"]
            assert np.array_equal(cp.read(dem.CPL_SURFACE_INSERTED).astype(np.int64), out["nins"].astype(np.int64))
            assert np.array_equal(np.round(cp.read(dem.CPL_SURFACE_CARRY) / mu).astype(np.int64), out["carry"])
            assert np.array_equal(np.round(cp.read(dem.CPL_SURFACE_MASS) / mu).astype(np.int64),
                                  out["cross"].astype(np.int64))
        if call == 0:
            first = [lvl.read(dem.FEXT) for lvl in h.levels], [f.copy() for f in o.fext], \
                [(cp_.read(dem.CPL_LAYER_STRESS)) for cp_ in h.couplers]
    return lv, specs, h, o, first


def _compare(lv, specs, h, o, first):
    inserted = 0
    for k, (wl, lvl) in enumerate(zip(lv, h.levels)):
        live, ids = lvl.counts()
        assert ids[0] == o.next_id[k]
        x = lvl.read(dem.POS)            # removed IDs (dropped, or marked at the last call) read as NaN
        xo = o.positions_by_id(k, ids[0])
        assert np.array_equal(np.isnan(x[:, 0]), np.isnan(xo[:, 0]))
        assert (~np.isnan(x[:, 0])).sum() == o.sims[k].n
        ok = ~np.isnan(x[:, 0])
        r = lvl.read(dem.RADIUS)[ok]
        d = min_image(x[ok] - xo[ok], wl)
        tol = np.maximum(1e-4 * 2 * r[:, None], 64 * np.spacing(np.abs(xo[ok]).astype(np.float32)).astype(np.float64))
        assert (np.abs(d) <= tol).all(), (k, np.abs(d).max())
        inserted += ids[0] - wl.n
    assert inserted > 0                                   # the fine levels did receive particles
    # held forces at the first call (same inputs up to one period of float rounding)
    g_f, o_f, stress = first
    for k in range(len(lv)):
        scale = 0.0
        if k > 0:                                         # fine side of coupler k - 1: stress controller
            sp = specs[k - 1]
            Tc = sp["interval"] * sp["dt"]
            sig = np.abs(stress[k - 1][:, :, :3]).max()
            scale = 1e-5 * 2 * sig * (sp["kp"] + sp["ki"] * Tc) * np.pi * lv[k].r.max() ** 2
        if k < len(lv) - 1:                               # coarse side of coupler k: velocity correction
            sp = specs[k]
            Tc = sp["interval"] * sp["dt"]
            vmax = np.abs(lv[k].v).max() + 1.0
            scale += sp["kv"] * lv[k].m.max() * 5 * 1e-6 * vmax / Tc
        n = len(o_f[k])
        assert np.all(np.abs(g_f[k][:n] - o_f[k]) <= scale + 1e-6 * np.abs(o_f[k])), k


def test_two_levels_at_two_to_one_time_steps_match_the_oracle():
    _compare(*_run(TWO, u0=20.0, periods=8))


def test_three_nested_levels_multirate_match_the_oracle():
    _compare(*_run(THREE, u0=20.0, periods=6))
