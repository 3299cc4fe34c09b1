"""Axisymmetric walls (the silo's cone and cylinder, the orifice disk) and removal below the
orifice, on the GPU against the FP64 oracle (Eqs. 3-6 at a particle-wall contact).

Bars: forces at identical state within 1e-5 of sum_j |F_ij| + |m g| per particle (as for
particle pairs); 300-step positions within max(1e-4 d, 64 ulp_fp32(|x|)); graph-captured and
direct stepping bit-identical; removal bookkeeping exact.
"""
import math

import numpy as np
import pytest

from paper_1705_03850_gb300 import dem, workloads
from _util import oracle_sim

pytestmark = pytest.mark.gpu

FORCE_REL = 1e-5


def _sim(wl, walls, z_remove=-math.inf, graph=0, lanes=1):
    sim = dem.from_workload(wl)
    sim.set_step_lanes(lanes)
    sim.set_walls(0, (0.0, 0.0), walls, z_remove)
    if graph:
        sim.set_graph(graph)
    return sim


def _ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("seed,closed", [(21, True), (22, False)])
def test_wall_forces_at_identical_state(seed, closed):
    # spheres scattered over the vessel's bounding cylinder: contacts with the cone, the
    # cylinder, the rims at the orifice and at the cone-cylinder kink, the orifice disk, and
    # from outside the wall
    wl = workloads.small_vessel(seed=seed, n=900, packed=False, closed=closed)
    walls = wl.meta["walls"]                                 # with the orifice disk when closed
    sim = _sim(wl, walls)
    F = sim.read(dem.FORCE)
    T = sim.read(dem.TORQUE)
    Fo, To, hist, fabs = oracle_sim(wl, walls).evaluate()
    nw = int((hist[1] <= -2).sum())
    assert nw > 50
    segs = set((-2 - hist[1][hist[1] <= -2]).tolist())
    assert segs == set(range(len(walls) - 1))            # every segment is touched
    err = np.abs(F - Fo).max(axis=1) / (fabs + 1e-30)
    assert err.max() <= FORCE_REL, (err.max(), err.argmax())
    terr = np.abs(T - To).max(axis=1) / (fabs * wl.r + 1e-30)
    assert terr.max() <= FORCE_REL
    st = sim.stats()
    assert st["wall_contacts"] == nw


@pytest.mark.parametrize("lanes", [1, 4])
def test_filling_of_a_small_vessel_matches_oracle(lanes):
    # a lattice thrown down (1 m/s) into the closed vessel: exact positions over the first 300
    # steps (the first impacts on the cone), then mean height and kinetic energy at 600 steps,
    # once the impacts on the cone and on the orifice disk have spread through the packing;
    # with one thread per particle and with four lanes per particle (the multi-lane step kernel
    # with walls)
    wl = workloads.small_vessel(seed=23)
    wl.v[:, 2] = workloads.f32(wl.v[:, 2] - 1.0)
    walls = wl.meta["walls"]
    sim = _sim(wl, walls, lanes=lanes)
    assert sim.stats()["step_lanes"] == lanes
    o = oracle_sim(wl, walls)
    sim.step(300).sync()
    o.run(300)
    x = sim.read(dem.POS)
    tol = np.maximum(1e-4 * 2 * wl.r[:, None], 64 * _ulp32(o.x))
    assert (np.abs(x - o.x) <= tol).all(), np.abs(x - o.x).max()
    sim.step(300).sync()
    o.run(300)
    x, v = sim.read(dem.POS), sim.read(dem.VEL)
    assert x[:, 2].mean() == pytest.approx(o.x[:, 2].mean(), rel=1e-4)
    ke, ke_o = (wl.m[:, None] * v ** 2).sum(), (wl.m[:, None] * o.v ** 2).sum()
    assert ke == pytest.approx(ke_o, rel=1e-2)
    _, _, hist, _ = o.evaluate(dt_hist=wl.dt)
    assert int((hist[1] <= -2).sum()) > 10                  # wall contacts did form,
    assert set((-2 - hist[1][hist[1] <= -2]).tolist()) == {0, 1}   # on the disk and on the cone


@pytest.mark.parametrize("case", ["cone", "kink", "rim"])
def test_single_sphere_against_the_wall_matches_oracle(case):
    # one sphere running round the cone, sitting in the cone-cylinder corner (two contacts,
    # then one), sliding off the orifice's edge: a wall contact and its tangential overlap
    # carried over 2,000 steps
    wl = workloads.vessel_sphere(case)
    walls = wl.meta["walls"]
    sim = _sim(wl, walls)
    o = oracle_sim(wl, walls)
    for n in (500, 1500):
        sim.step(n).sync()
        o.run(n)
        x, v = sim.read(dem.POS), sim.read(dem.VEL)
        assert np.abs(x - o.x).max() <= 5e-7, np.abs(x - o.x).max()
        assert np.abs(v - o.v).max() <= 1e-3 * np.abs(o.v).max() + 1e-5
    _, _, hist, _ = o.evaluate(dt_hist=wl.dt)
    assert (hist[1] <= -2).any()                            # still in contact with the wall


@pytest.mark.parametrize("lanes", [1, 8])
def test_graph_and_direct_stepping_agree_with_walls_and_removal(lanes):
    wl = workloads.small_vessel(seed=24)
    walls = wl.meta["walls"][1:]                             # orifice open
    z_rem = wl.meta["z_o"] - 0.004
    a = _sim(wl, walls, z_rem, graph=25, lanes=lanes)
    b = _sim(wl, walls, z_rem, lanes=lanes)
    a.step(4000).sync()
    b.step(4000).sync()
    xa, xb = a.read(dem.POS), b.read(dem.POS)
    assert np.array_equal(np.isnan(xa), np.isnan(xb))
    assert np.array_equal(np.nan_to_num(xa), np.nan_to_num(xb))
    assert a.wall_removed() == b.wall_removed()


def test_removal_below_the_orifice():
    # the vessel drains through the open orifice; particles falling below z_remove are gone,
    # and count and mass removed add up exactly
    wl = workloads.small_vessel(seed=25)
    walls = wl.meta["walls"][1:]
    z_rem = wl.meta["z_o"] - 0.002
    sim = _sim(wl, walls, z_rem, graph=50)
    sim.step(30000).sync()
    x = sim.read(dem.POS)
    gone = np.isnan(x[:, 0])
    count, mass = sim.wall_removed()
    assert count == int(gone.sum()) > 0
    assert mass == pytest.approx(float(wl.m[gone].sum()), rel=1e-6)
    assert (x[~gone, 2] >= z_rem).all()
    live, ids = sim.counts()            # parked particles count as live until a list build drops them
    assert wl.n - count <= live[0] <= wl.n and ids[0] == wl.n
    rho = np.hypot(x[~gone, 0], x[~gone, 1])
    assert (rho < 0.012 + 1e-3).all()                        # held by the cylinder


def test_walls_refused_by_rollouts_and_checked():
    wl = workloads.small_vessel(seed=26, n=100)
    sim = dem.from_workload(wl)
    with pytest.raises(dem.DemError):
        sim.set_walls(0, (0.0, 0.0), [(0.01, 0.01)])         # one point
    with pytest.raises(dem.DemError):
        sim.set_walls(0, (0.0, 0.0), [(0.01, 0.01), (0.01, 0.01)])   # zero-length segment
    sim.set_walls(0, (0.0, 0.0), wl.meta["walls"])
    with pytest.raises(dem.DemError):
        sim.rollout_forward(10, 5)


def test_coarse_grain_silo_discharge_rate_reproduces_table_2():
    # Sec. 3, Table 2: the coarse-grain silo (alpha = 2, 23,438 spheres of 5.6 mm) discharges at
    # 0.315 +- 0.028 kg/s through the 4 cm orifice, measured 1 cm below it at 100 Hz; the
    # synthetic fill (a settled lattice instead of the paper's pouring) must give a mean within
    # two of the paper's standard deviations, and its own scatter of the same order
    from paper_1705_03850_gb300 import silo
    r = silo.run(2, settle_s=0.3, discharge_s=0.6, skip_s=0.1)
    assert r["particles"] == 23_438
    assert abs(r["rate_mean_kg_s"] - 0.315) <= 2 * 0.028, r["rate_mean_kg_s"]
    assert 0.25 * 0.028 <= r["rate_std_kg_s"] <= 4 * 0.028, r["rate_std_kg_s"]
    assert r["removed_mass_kg"] > 0.1                  # 0.5 s of steady flow at ~0.3 kg/s left the silo
