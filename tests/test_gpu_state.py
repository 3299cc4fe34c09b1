"""State I/O and stored overlaps on the GPU against the FP64 oracle (through the C ABI).

* Resume: a run stopped, read out (state, contacts, floor overlaps), written into a new context
  and continued equals the oracle restarted the same way from its own state and history
  (100-step bar: positions within max(1e-4 d, 64 ulp_fp32(|x|))).
* Stored overlaps carried across frequent list rebuilds equal the oracle's contact history, pair
  by pair.
* Arbitrary FP64 input: positions and radii are rounded to the position quantum q as documented
  (exactly), and forces at that input match the oracle fed the unrounded values (per-particle
  bar 1e-5 of sum_j |F_ij|: moving a centre by q/2 changes a force far less).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1705_03850_gb300 import dem, workloads
from _util import gpu_pairs, min_image, oracle_pairs, oracle_sim

pytestmark = pytest.mark.gpu


def _ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


def _rollout_bar(x, xo, wl):
    d = min_image(x - xo, wl)
    tol = np.maximum(1e-4 * 2 * wl.r[:, None], 64 * _ulp32(xo))
    assert (np.abs(d) <= tol).all(), np.abs(d).max()
    return np.abs(d).max()


def test_resume_through_the_c_abi_matches_the_oracle_restarted_the_same_way():
    wl = workloads.dense_block(10, 9, 6, seed=31, vel=0.3)
    k, m = 40, 60
    a = dem.from_workload(wl)
    a.step(k).sync()
    state = [a.read(f) for f in (dem.POS, dem.VEL, dem.OMEGA, dem.RADIUS, dem.MASS)]
    partner, xi = a.read_contacts(width=24)
    wxi = a.read(dem.WALL_XI)
    assert (np.abs(wxi).max(axis=1) > 0).sum() > 20          # floor contacts with stored overlaps
    b = dem.DEM([dem.desc_from_workload(wl)])
    b.write_state(*state)
    b.write_contacts(partner, xi)
    b.write(dem.WALL_XI, wxi)
    # the new context holds the written contacts and overlaps (read out by an evaluation at the
    # written state: sticking contacts give back what was written, slipping ones are truncated
    # again at the written integer-step velocities, so only the pattern is compared here)
    p2, xi2 = b.read_contacts(width=24)
    assert np.array_equal(p2, partner)
    assert np.array_equal(xi2 != 0, xi != 0)
    assert np.array_equal(b.read(dem.WALL_XI) != 0, wxi != 0)
    b.step(m).sync()
    # the oracle: its own run to step k, restarted from (x, v, w) and its contact history
    o = oracle_sim(wl).run(k)
    ha, hb, hx, _ = o.history()
    assert (hb < 0).sum() > 20
    o2 = oracle.Sim(o.P, o.x, o.v, o.w, o.r, o.m)
    o2.set_history(ha, hb, hx)
    o2.run(m)
    _rollout_bar(b.read(dem.POS), o2.x, wl)
    # and the restart is a small perturbation of the uninterrupted run
    a.step(m).sync()
    _rollout_bar(b.read(dem.POS), a.read(dem.POS), wl)


def test_stored_overlaps_carried_across_list_rebuilds_match_the_oracle():
    # a small skin makes the lists rebuild every step or two; every carried overlap must land on
    # the right pair (a lost or misplaced one is off by its whole size)
    wl = dataclasses.replace(workloads.dense_block(10, 10, 6, seed=32, vel=0.6), skin=workloads.qgrid(4e-6))
    steps = 20
    sim = dem.from_workload(wl)
    sim.step(steps).sync()
    assert sim.stats()["rebuilds"] >= 6
    partner, gxi = sim.read_contacts(width=24)
    o = oracle_sim(wl).run(steps)
    x = sim.read(dem.POS)
    _rollout_bar(x, o.x, wl)
    dx = np.abs(min_image(x - o.x, wl)).max(axis=1)
    ha, hb, hx, _ = o.history()
    ref = {(int(p), int(q)): x for p, q, x in zip(ha, hb, hx) if q >= 0}
    assert gpu_pairs(partner) == set(ref)
    scale = max(np.abs(hx).max(), 1e-30)
    nz = 0
    for i, row in enumerate(partner):
        for t, p in enumerate(row):
            if p < 0:
                break
            o_xi = ref[(min(i, p), max(i, p))]
            # float32 accumulation of v_t dt (1e-4), and a slipping contact's overlap follows the
            # normal force (it is mu f_n / k_t, proportional to the overlap delta): relative error
            # up to the pair's centre differences over delta
            dd = min_image(o.x[i] - o.x[p], wl)
            delta = o.r[i] + o.r[p] - np.linalg.norm(dd)
            rel = 1e-4 + 2 * np.sqrt(3) * (dx[i] + dx[p]) / delta
            assert np.abs(gxi[i, t] - o_xi).max() <= rel * np.abs(o_xi).max() + 1e-6 * scale, (i, p, rel)
            nz += np.abs(o_xi).max() > 1e-3 * scale
    assert nz > wl.n


def test_unrounded_fp64_input_is_rounded_as_documented_and_matches_the_oracle():
    wl = workloads.dense_block(11, 9, 6, seed=33)
    rng = np.random.default_rng(33)
    x = wl.x + rng.uniform(-0.5, 0.5, wl.x.shape) * workloads.GRID       # off every power-of-two grid
    v = wl.v * (1.0 + rng.uniform(-1e-3, 1e-3, wl.v.shape))               # not float32 values
    w = wl.w * (1.0 + rng.uniform(-1e-3, 1e-3, wl.w.shape))
    r = wl.r * (1.0 + rng.uniform(-1e-4, 1e-4, wl.n))
    m = wl.material.rho * 4.0 / 3.0 * np.pi * r ** 3
    assert not np.array_equal(workloads.qgrid(x), x)
    sim = dem.DEM([dem.desc_from_workload(wl)])
    sim.write_state(x, v, w, r, m)
    inf = sim.info()
    q, lo = inf["q"], np.array(inf["lo"])
    # positions and radii: the nearest multiple of q from the box origin (round half to even)
    assert np.array_equal(sim.read(dem.POS), lo + np.rint((x - lo) / q) * q)
    assert np.array_equal(sim.read(dem.RADIUS), np.rint(r / q) * q)
    assert np.array_equal(sim.read(dem.MASS), m.astype(np.float32).astype(np.float64))
    # forces at that state against the oracle fed the unrounded input: the float bar 1e-5 of
    # sum_j |F_ij| plus what rounding the centres and radii (by at most sqrt(3) q / 2 and q / 2)
    # does to a Hertz normal force at the start-up evaluation (no stored overlaps):
    # dF = 2 E* sqrt(R delta) d(delta) with d(delta) <= (sqrt(3) + 1) q per contact
    F = sim.read(dem.FORCE)
    P = oracle_sim(wl).P
    Fo, To, hist, fabs = oracle.Sim(P, x, v, w, r, m).evaluate()
    mt = wl.material
    Estar = mt.E / (2 * (1 - mt.nu ** 2))
    slack = np.zeros(wl.n)
    for i, j in oracle.pairs(P, x, r, 0.0):
        dd = min_image(x[i] - x[j], wl)
        delta = r[i] + r[j] - np.linalg.norm(dd)
        dF = 2 * Estar * np.sqrt(r[i] * r[j] / (r[i] + r[j]) * delta) * (np.sqrt(3) + 1) * q
        slack[i] += dF
        slack[j] += dF
    slack += 2 * Estar * np.sqrt(r * np.maximum(r - x[:, 2], 0)) * (np.sqrt(3) + 1) * q * (x[:, 2] < r)
    err = np.abs(F - Fo).max(axis=1)
    assert np.all(err <= 1e-5 * fabs + slack), (err / (1e-5 * fabs + slack)).max()
    partner, _ = sim.read_contacts(width=24)
    g, o = gpu_pairs(partner), oracle_pairs(hist)
    # a pair whose overlap is within the rounding of the centres (sqrt(3) q) may differ
    for i, j in g ^ o:
        dd = min_image(x[i] - x[j], wl)
        assert abs(r[i] + r[j] - np.linalg.norm(dd)) < 2 * np.sqrt(3) * q, (i, j)
    assert len(o) > 2 * wl.n
