"""Coupling of a coarse and a fine level (Sec. 2.3) on the GPU against the FP64 oracle, same inputs.

Integer bookkeeping (entered mass, histograms, carries, insertion sets) must be
bit-exact; stresses, velocities and controller forces agree within float
rounding of the contact forces (1e-5 relative to each cell's scale)."""
import numpy as np
import pytest

import oracle
from paper_1705_03850_gb300 import dem, workloads
from _util import oracle_params

pytestmark = pytest.mark.gpu


def _state(wl):
    return dict(x=wl.x, v=wl.v, w=wl.w, r=wl.r, m=wl.m, id=np.arange(wl.n))


# a vertical cylinder wall about the column's axis, radius 10 mm: it cuts through the
# transition cells and the feed face's surface cells of both levels
WALL_AXIS = (0.012, 0.012)
WALL = [(0.010, -0.01), (0.010, 0.07)]
# a cone closed below by a disk: radius 4 mm at z = 0 to 16 mm at z = 24 mm, then a cylinder
CONE = [(0.0, 0.0), (0.004, 0.0), (0.016, 0.024), (0.016, 0.06)]


def _setup(pre_force=None, walls=None, **extra):
    A, B, fine_wl, spec = workloads.coupling_case()
    spec = dict(spec, **extra)
    rmax_c, rmax_f = float(A.r.max()), float(fine_wl.r.max())
    coarse = dem.DEM([dem.desc_from_workload(A, r_max=rmax_c)])
    coarse.write_state(A.x, A.v, A.w, A.r, A.m)
    fine = dem.DEM([dem.desc_from_workload(fine_wl, r_max=rmax_f, capacity=fine_wl.n + 4000)])
    fine.write_state(fine_wl.x, fine_wl.v, fine_wl.w, fine_wl.r, fine_wl.m)
    if walls is not None:
        coarse.set_walls(0, WALL_AXIS, walls)
        fine.set_walls(0, WALL_AXIS, walls)
    cp = dem.Coupler(coarse, fine, **spec)
    coarse.write_state(B.x, B.v, B.w, B.r, B.m)
    if pre_force is not None:
        coarse.write(dem.FEXT, pre_force(coarse.n, 0.1))
        fine.write(dem.FEXT, pre_force(fine.n, 2e-5))
    cp.couple()
    qf = oracle.quantum(fine_wl.lo, fine_wl.hi)
    orc = oracle.Coupler(spec, oracle_params(B, walls, WALL_AXIS), oracle_params(fine_wl, walls, WALL_AXIS), fine_wl.lo, qf,
                         int(np.ceil(rmax_f / qf)), fine_wl.material.rho, idcap=A.n)
    orc.record(A.x, np.arange(A.n))
    out = orc.call(_state(B), _state(fine_wl), 0.0, 0.0)
    return A, B, fine_wl, spec, coarse, fine, cp, out, qf


@pytest.mark.parametrize("walls", [None, WALL, CONE])
def test_coupling_bookkeeping_and_insertion_are_bit_exact(walls):
    A, B, fine_wl, spec, coarse, fine, cp, out, qf = _setup(walls=walls)
    mu = spec["mass_unit"]
    assert out["cross"].sum() > 0 and out["nins"].sum() > 0      # material entered and was inserted
    assert np.array_equal(np.round(cp.read(dem.CPL_SURFACE_MASS) / mu).astype(np.int64), out["cross"].astype(np.int64))
    assert np.array_equal(cp.read(dem.CPL_SURFACE_HIST).astype(np.int64), out["hist"].astype(np.int64))
    assert np.array_equal(np.round(cp.read(dem.CPL_SURFACE_CARRY) / mu).astype(np.int64), out["carry"])
    nins = cp.read(dem.CPL_SURFACE_INSERTED).astype(np.int64)
    assert np.array_equal(nins, out["nins"].astype(np.int64))
    # the inserted particles, in cell order, appended after the fine level's own
    live, ids = fine.counts()
    assert ids[0] == fine_wl.n + nins.sum()
    x = fine.read(dem.POS)[fine_wl.n:]
    r = fine.read(dem.RADIUS)[fine_wl.n:]
    ref = np.concatenate([out["ins_u"][c, :out["nins"][c]] for c in range(len(nins))])
    assert np.array_equal(x, np.asarray(fine_wl.lo) + ref[:, :3] * qf)
    assert np.array_equal(r, ref[:, 3] * qf)
    # no inserted particle overlaps another or a fine particle (brute force)
    allx = fine.read(dem.POS)
    allr = fine.read(dem.RADIUS)
    pairs = oracle.pairs(oracle_params(fine_wl), allx, allr, 0.0, method="brute")
    assert not np.any(pairs[:, 1] >= fine_wl.n)
    # mass conservation: inserted + carry = entered (exact, integer units)
    mass_in = np.array([sum(round(m / mu) for m in out["ins_m"][c, :out["nins"][c]]) for c in range(len(nins))])
    assert np.array_equal(mass_in + out["carry"], out["cross"].astype(np.int64))
    if walls is WALL:             # inserted spheres lie inside the wall, clear of it
        rho = np.hypot(x[:, 0] - WALL_AXIS[0], x[:, 1] - WALL_AXIS[1])
        assert np.all(rho + r <= WALL[0][0])
    if walls is CONE:             # inside the cone (normal at atan(1/2) from the horizontal), clear of it
        rho = np.hypot(x[:, 0] - WALL_AXIS[0], x[:, 1] - WALL_AXIS[1])
        assert np.all((0.004 + 0.5 * x[:, 2] - rho) / np.hypot(1.0, 0.5) >= r)


@pytest.mark.parametrize("walls,extra", [(None, {}), (WALL, {}), (None, {"velocity_below": 0.01})])
def test_coupling_measurements_and_controllers_match_oracle(walls, extra):
    # the third case: mass-flow correction cells centred below 10 mm take the velocity target
    A, B, fine_wl, spec, coarse, fine, cp, out, qf = _setup(walls=walls, **extra)
    S = cp.S
    st = cp.read(dem.CPL_LAYER_STRESS)                 # (S, 2, 6)
    ref = np.transpose(out["lay"][:, :, :6], (1, 0, 2))
    scale = np.abs(ref).max(axis=2, keepdims=True) + 1e-12
    assert np.all(np.abs(st - ref) <= 1e-5 * scale)
    phi = cp.read(dem.CPL_LAYER_PHI)
    assert np.allclose(phi, out["lay"][:, :, 6].T, rtol=1e-12, atol=0)
    vel = cp.read(dem.CPL_LAYER_VEL)
    assert np.allclose(vel, np.transpose(out["lay"][:, :, 7:10], (1, 0, 2)), rtol=1e-6, atol=1e-9)
    ctrl = cp.read(dem.CPL_LAYER_CTRL)
    assert np.all(np.abs(ctrl - out["ctrl"]) <= 1e-5 * (np.abs(out["ctrl"]).max(axis=0) + 1e-12))
    fav = cp.read(dem.CPL_SURFACE_VEL)
    ref_v = out["fav"][:, 1:4] / np.maximum(out["fav"][:, :1], 1e-300)
    assert np.allclose(fav, ref_v, rtol=1e-6, atol=1e-9)
    # controller forces held on the particles
    fc = coarse.read(dem.FEXT)
    assert np.abs(fc - out["fext_c"]).max() <= 1e-5 * np.abs(out["fext_c"]).max() + 1e-12
    ff = fine.read(dem.FEXT)[:fine_wl.n]
    assert np.abs(ff - out["fext_f"]).max() <= 1e-4 * np.abs(out["fext_f"]).max() + 1e-12
    assert np.abs(out["fext_f"]).max() > 0 and np.abs(out["fext_c"]).max() > 0


def test_added_controller_forces_sum_with_the_held_ones():
    # a level shared by two couplers takes the sum of their forces (add_forces = 1)
    # (held forces of the size of each level's controller forces, float32 values)
    held = lambda n, s: (np.random.default_rng(n).normal(size=(n, 3)) * s).astype(np.float32).astype(np.float64)
    A, B, fine_wl, spec, coarse, fine, cp, out, qf = _setup(pre_force=held, add_forces=1)
    fc = coarse.read(dem.FEXT)
    ref_c = held(coarse.n, 0.1) + out["fext_c"]
    assert np.abs(fc - ref_c).max() <= 1e-5 * np.abs(ref_c).max()
    assert np.abs(fc - out["fext_c"]).max() > 1e-2          # the held part is there
    ff = fine.read(dem.FEXT)[:fine_wl.n]
    ref_f = held(fine_wl.n, 2e-5) + out["fext_f"]         # (fine.n now counts the inserted particles)
    assert np.abs(ff - ref_f).max() <= 1e-4 * np.abs(ref_f).max()
    assert np.abs(ff - out["fext_f"]).max() > 2e-6
    # the inserted particles start with no held force; clearing zeroes every one
    assert np.abs(fine.read(dem.FEXT)[fine_wl.n:]).max() == 0.0
    coarse.clear_external_force()
    assert np.abs(coarse.read(dem.FEXT)).max() == 0.0


def test_held_external_force_acts_like_gravity():
    # a held force m g in a gravity-free box moves the particles as gravity g does
    import dataclasses
    wl = workloads.dense_block(4, 4, 3, seed=5, vel=0.0, spin=0.0, floor_v=(0.0, 0.0, 0.0))
    g = np.array([0.0, 0.0, -9.81])
    a = dem.DEM([dem.desc_from_workload(wl)])
    a.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    wl0 = dataclasses.replace(wl, g=(0.0, 0.0, 0.0))
    b = dem.DEM([dem.desc_from_workload(wl0)])
    b.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    b.write(dem.FEXT, wl.m[:, None] * g[None, :])
    assert np.allclose(b.read(dem.FEXT), wl.m[:, None] * g[None, :], rtol=1e-7, atol=0)
    a.step(200)
    b.step(200)
    va, vb = a.read(dem.VEL), b.read(dem.VEL)
    assert np.abs(va - vb).max() <= 1e-4 * np.abs(va).max()
    assert np.abs(a.read(dem.POS) - b.read(dem.POS)).max() <= 1e-9


def test_coupled_levels_keep_stepping():
    A, B, fine_wl, spec, coarse, fine, cp, out, qf = _setup()
    for _ in range(3):
        coarse.step(spec["interval"])
        fine.step(spec["interval"])
        cp.couple()
    coarse.sync()
    fine.sync()
    live, ids = fine.counts()
    assert live[0] == ids[0] >= fine_wl.n
    assert np.isfinite(fine.read(dem.POS)).all()
