"""Three nested coarse-graining levels of an inclined chute, coupled pairwise (Sec. 2.3), on the GPU.

Checks what holds at any size: graph-captured and direct stepping agree bit for
bit through coupling, insertion and removal; the mass bookkeeping of every surface
cell closes over many calls (entered = inserted + carried, with the inserted masses
as the particles keep them in float32); no particle of a fine level is left beyond
a drain face after a call.
"""

import numpy as np
import pytest

from paper_1705_03850_gb300 import dem, levels, workloads

pytestmark = pytest.mark.gpu

SMALL = dict(length=0.3, width=0.06, height=0.1, bed=0.04, regions=((0.1, 0.12), (0.14, 0.04)))


def _hierarchy(graph, u0=0.5, multirate=False, streams=False):
    lv, specs = workloads.chute(**SMALL, u0=u0, multirate=multirate, interval=16 if multirate else 15)
    ctx = []
    for k, wl in enumerate(lv):
        cap = None if k == 0 else wl.n + 20000
        kw = {}
        if streams:
            import torch
            kw["stream"] = torch.cuda.Stream()
        d = dem.DEM([dem.desc_from_workload(wl, capacity=cap)], max_neighbors=24, **kw)
        v = np.zeros_like(wl.v)
        v[:, 0] = u0
        d.write_state(wl.x, v, wl.w, wl.r, wl.m)
        ctx.append(d)
    return lv, specs, levels.Hierarchy(ctx, specs, steps_per_graph=graph)


def test_graph_and_direct_stepping_agree_through_coupling():
    _, _, a = _hierarchy(True)
    _, _, b = _hierarchy(False)
    a.advance(8)
    b.advance(8)
    assert a.counts() == b.counts()
    for la, lb in zip(a.levels, b.levels):
        xa, xb = la.read(dem.POS), lb.read(dem.POS)
        assert np.array_equal(np.isnan(xa), np.isnan(xb))
        assert np.array_equal(np.nan_to_num(xa), np.nan_to_num(xb))


def test_one_stream_per_level_equals_one_stream_for_all():
    # levels on their own streams step concurrently within a period; the coupling call orders
    # them (the fine side after the coarse side's steps, the coarse side's next steps after the
    # coupling kernels), so the run is the one on a single stream, bit for bit, through
    # insertion and removal
    lv, _, a = _hierarchy(True, u0=10.0)
    _, _, b = _hierarchy(True, u0=10.0, streams=True)
    a.advance(30)
    b.advance(30)
    assert a.counts() == b.counts()
    assert a.counts()[2] != lv[2].n                                        # particles came and went
    for la, lb in zip(a.levels, b.levels):
        for f in (dem.POS, dem.VEL):
            xa, xb = la.read(f), lb.read(f)
            assert np.array_equal(np.isnan(xa), np.isnan(xb))
            assert np.array_equal(np.nan_to_num(xa), np.nan_to_num(xb))


def _rows_of_new_particles_complete(level, wl, first_new_id):
    # every pair of a particle inserted at the last call with any live particle closer than
    # r_i + r_j + skin (brute force over the positions read back) is in both neighbour rows
    from scipy.spatial import cKDTree
    x = level.read(dem.POS)
    rad = level.read(dem.RADIUS)
    live = ~np.isnan(x[:, 0])
    ids = np.flatnonzero(live)
    lo, hi = np.array(wl.lo), np.array(wl.hi)
    box = np.where(wl.periodic, hi - lo, 10.0 * (hi - lo) + 1.0)
    xl = np.mod(x[live] - lo, box)
    rl = rad[live]
    pairs = cKDTree(xl, boxsize=box).query_pairs(2.0 * rl.max() + wl.skin, output_type="ndarray")
    d = xl[pairs[:, 0]] - xl[pairs[:, 1]]
    d -= np.where(wl.periodic, box * np.round(d / box), 0.0)
    near = np.sqrt((d ** 2).sum(1)) < rl[pairs[:, 0]] + rl[pairs[:, 1]] + wl.skin - 1e-9
    new = (ids[pairs[:, 0]] >= first_new_id) | (ids[pairs[:, 1]] >= first_new_id)
    rows = level.read_neighbors(width=24)
    checked = 0
    for a_, b_ in pairs[near & new]:
        ia, ib = ids[a_], ids[b_]
        assert ib in rows[ia] and ia in rows[ib], (ia, ib)
        checked += 1
    return checked


def test_inserted_particles_get_complete_rows_without_a_list_build():
    # insertion builds the new particles' rows and appends them to their partners' rows instead
    # of rebuilding every list: right after calls that inserted particles, every pair of a new
    # particle within r_i + r_j + skin of another is in both rows
    lv, specs, h = _hierarchy(True, u0=10.0)
    fine = h.levels[2]
    checked, pairs = 0, 0
    for _ in range(200):
        before = int(fine.counts()[1][0])
        h.advance(1)
        if fine.counts()[1][0] > before:
            pairs += _rows_of_new_particles_complete(fine, lv[2], before)
            checked += 1
            if checked == 3:
                break
    assert checked == 3 and pairs > 20


@pytest.mark.parametrize("multirate", [False, True])
def test_mass_bookkeeping_closes_and_drained_particles_are_gone(multirate):
    lv, specs, h = _hierarchy(True, u0=10.0, multirate=multirate)
    entered = [0, 0]
    inserted = [0, 0]
    slack = [0, 0]
    carry = [None, None]
    for call in range(40):                               # 6 mm of plug flow: lattice planes cross the faces
        nid0 = [lvl.counts()[1][0] for lvl in h.levels]
        h.advance(1)
        for k, cp in enumerate(h.couplers):
            mu = specs[k]["mass_unit"]
            cross = np.round(cp.read(dem.CPL_SURFACE_MASS) / mu).astype(np.int64)
            nins = cp.read(dem.CPL_SURFACE_INSERTED).astype(np.int64)
            carry[k] = np.round(cp.read(dem.CPL_SURFACE_CARRY) / mu).astype(np.int64)
            fine = h.levels[k + 1]
            nid1 = fine.counts()[1][0]
            assert nid1 - nid0[k + 1] == nins.sum()
            # each inserted particle counts the mass of its drawn radius in whole units; the
            # particle keeps that mass as float32 (its radius, on the position grid, differs by
            # < q / 2): the stored masses give the units within float32 rounding and 1/2 unit each
            mass = fine.read(dem.MASS)[nid0[k + 1]:nid1]
            per_cell = np.zeros(len(cross))
            np.add.at(per_cell, np.repeat(np.arange(len(nins)), nins), mass / mu)
            slack_c = np.zeros(len(cross))
            np.add.at(slack_c, np.repeat(np.arange(len(nins)), nins), 1e-7 * mass / mu + 0.5)
            entered[k] = entered[k] + cross
            inserted[k] = inserted[k] + per_cell
            slack[k] = slack[k] + slack_c
            # nothing of the fine level is left beyond the drain face (x hi) of its region
            x = fine.read(dem.POS)
            live = ~np.isnan(x[:, 0])
            assert np.all(x[live, 0] < specs[k]["hi"][0])
    for k in range(2):
        assert np.all(np.abs(entered[k] - (inserted[k] + carry[k])) <= slack[k])
        assert entered[k].sum() > 0                      # coarse material did enter the region
    assert sum(int(i.sum()) for i in inserted) > 0       # and fine particles were inserted
    for lvl in h.levels:
        x = lvl.read(dem.POS)
        assert np.isfinite(x[~np.isnan(x[:, 0])]).all()


def test_multirate_levels_advance_one_common_period():
    # time steps scaled with the grain (8 mm: 4 dt, 4 mm: 2 dt, 2 mm: dt): per coupling period the
    # levels take 4, 8 and 16 steps and advance the same physical time, and graph-captured and
    # direct runs agree bit for bit
    _, _, a = _hierarchy(True, u0=10.0, multirate=True)
    _, _, b = _hierarchy(False, u0=10.0, multirate=True)
    assert a.steps == [4, 8, 16]
    a.advance(24)
    b.advance(24)
    t = [lv.stats()["steps"] * lv.dts[0] for lv in a.levels]
    assert max(t) - min(t) <= 1e-6 * max(t)
    assert a.counts() == b.counts()
    for la, lb in zip(a.levels, b.levels):
        xa, xb = la.read(dem.POS), lb.read(dem.POS)
        assert np.array_equal(np.isnan(xa), np.isnan(xb))
        assert np.array_equal(np.nan_to_num(xa), np.nan_to_num(xb))


def test_five_nested_levels_multirate():
    # the recursive nesting of the runtime discussion (alpha = 16, 8, 4, 2, 1; filled volume
    # quartered per level) at a small size: every level advances the same physical time per
    # period, graph-captured and direct runs agree bit for bit, positions stay finite
    SMALL5 = dict(length=5.12, width=0.06, height=0.06, bed=0.04, start=0.5, u0=10.0)

    def build(graph):
        lv, specs = workloads.nested_levels(**SMALL5)
        ctx = []
        for k, wl in enumerate(lv):
            d = dem.DEM([dem.desc_from_workload(wl, capacity=None if k == 0 else wl.n + 20000)], max_neighbors=24)
            v = np.zeros_like(wl.v)
            v[:, 0] = 10.0
            d.write_state(wl.x, v, wl.w, wl.r, wl.m)
            ctx.append(d)
        return levels.Hierarchy(ctx, specs, steps_per_graph=graph)

    a, b = build(True), build(False)
    assert a.steps == [1, 2, 4, 8, 16]
    a.advance(20)
    b.advance(20)
    t = [lv.stats()["steps"] * lv.dts[0] for lv in a.levels]
    assert max(t) - min(t) <= 1e-6 * max(t)
    assert a.counts() == b.counts()
    for la, lb in zip(a.levels, b.levels):
        xa, xb = la.read(dem.POS), lb.read(dem.POS)
        assert np.array_equal(np.isnan(xa), np.isnan(xb))
        assert np.array_equal(np.nan_to_num(xa), np.nan_to_num(xb))
        assert np.isfinite(xa[~np.isnan(xa[:, 0])]).all()


def test_output_fields_at_the_highest_resolution_available():
    # per-level grid fields equal the plain definition (oracle) at the read-back state, and the
    # composed fields take the finest level inside each region, the coarse level outside
    import oracle
    _, specs, h = _hierarchy(True, u0=2.0)
    h.advance(3)
    lo, hcell, n = (0.0, 0.0, 0.0), 0.01, (30, 6, 5)
    for lv in h.levels:
        g = lv.grid_fields(lo, hcell, n).cpu().numpy()
        x, v, r, m = lv.read(dem.POS), lv.read(dem.VEL), lv.read(dem.RADIUS), lv.read(dem.MASS)
        live = ~np.isnan(x[:, 0])
        ref = oracle.grid_fields(x[live], v[live], r[live], m[live], lo, hcell, n)
        assert np.allclose(g[..., :2], ref[..., :2], rtol=1e-12, atol=0)
        assert np.allclose(g[..., 2:], ref[..., 2:], rtol=1e-9, atol=1e-12)
    f, which = h.fields(lo, hcell, n)
    f, which = f.cpu().numpy(), which.cpu().numpy()
    per = [lv.grid_fields(lo, hcell, n).cpu().numpy() for lv in h.levels]
    xc = lo[0] + (np.arange(n[0]) + 0.5) * hcell
    inner = (xc >= specs[1]["lo"][0]) & (xc < specs[1]["hi"][0])
    assert inner.any() and (~inner).any()
    assert np.array_equal(f[:, :, inner], per[2][:, :, inner])
    outer = (xc < specs[0]["lo"][0]) | (xc >= specs[0]["hi"][0])
    assert np.array_equal(f[:, :, outer], per[0][:, :, outer])
    assert set(np.unique(which).tolist()) == {0, 1, 2}
