"""Coupling of a coarse and a fine level (Sec. 2.3) on the GPU against the FP64 oracle, same inputs.

Integer bookkeeping (entered mass, histograms, carries) must be bit-exact.  Insertion: the
oracle draws radii and centres in continuous space and tests overlaps in metres; the GPU
draws the same values and rounds them to its position grid (quantum q) before testing, so
the two agree on every candidate whose clearance is outside (-4 q, 4 q) -- rounding moves
a clearance by at most (sqrt(3) + 1) q.  Cells with such a borderline decision (and the
cells of later faces, whose candidates test against them) are compared only up to it;
elsewhere the inserted sets are equal, centres and radii within q / 2.  Stresses,
velocities and controller forces agree within float rounding of the contact forces (1e-5
relative to each cell's scale)."""
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


BAND_Q = 4.0      # borderline band of an insertion decision, in fine quanta


def compared_cells(out, faces):
    """Surface cells whose insertion sequence is compared in full: no borderline decision in the
    cell, nor in any cell of an earlier face.  faces: list of (first cell, cell count)."""
    ok = np.ones(len(out["nins"]), dtype=bool)
    earlier = False
    for off, n in faces:
        cells = slice(off, off + n)
        if earlier:
            ok[cells] = False
        ok[cells] &= out["border"][cells] < 0
        earlier = earlier or bool((out["border"][cells] >= 0).any())
    return ok


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
    orc = oracle.Coupler(spec, oracle_params(B, walls, WALL_AXIS), oracle_params(fine_wl, walls, WALL_AXIS), rmax_f,
                         fine_wl.material.rho, idcap=A.n, band=BAND_Q * qf)
    orc.record(A.x, np.arange(A.n))
    out = orc.call(_state(B), _state(fine_wl), 0.0, 0.0)
    return A, B, fine_wl, spec, coarse, fine, cp, out, qf


@pytest.mark.parametrize("walls", [None, WALL, CONE])
def test_coupling_bookkeeping_and_insertion_match_the_oracle(walls):
    A, B, fine_wl, spec, coarse, fine, cp, out, qf = _setup(walls=walls)
    mu = spec["mass_unit"]
    assert out["cross"].sum() > 0 and out["nins"].sum() > 0      # material entered and was inserted
    assert np.array_equal(np.round(cp.read(dem.CPL_SURFACE_MASS) / mu).astype(np.int64), out["cross"].astype(np.int64))
    assert np.array_equal(cp.read(dem.CPL_SURFACE_HIST).astype(np.int64), out["hist"].astype(np.int64))
    nins = cp.read(dem.CPL_SURFACE_INSERTED).astype(np.int64)
    carry = np.round(cp.read(dem.CPL_SURFACE_CARRY) / mu).astype(np.int64)
    # only the top face feeds the column: one face of 2 x 2 cells
    faces = [(0, len(nins))]
    ok = compared_cells(out, faces)
    assert ok.mean() >= 0.75, out["border"]
    assert np.array_equal(nins[ok], out["nins"][ok].astype(np.int64))
    assert np.array_equal(carry[ok], out["carry"][ok])
    # the inserted particles, in cell order, appended after the fine level's own
    live, ids = fine.counts()
    assert ids[0] == fine_wl.n + nins.sum()
    x = fine.read(dem.POS)[fine_wl.n:]
    r = fine.read(dem.RADIUS)[fine_wl.n:]
    start = np.concatenate([[0], np.cumsum(nins)])
    tol = 0.5 * qf * (1 + 1e-9)
    for c in np.nonzero(ok)[0]:
        ref = out["ins_x"][c, :out["nins"][c]]
        gx, gr = x[start[c]:start[c + 1]], r[start[c]:start[c + 1]]
        assert np.all(np.abs(gx - ref[:, :3]) <= tol), (c, np.abs(gx - ref[:, :3]).max() / qf)
        assert np.all(np.abs(gr - ref[:, 3]) <= tol)
    # the positions are not merely on a coarser grid: the inserted centres take the grid
    # points nearest to the oracle's continuous ones (the radii, drawn continuously, differ from
    # one another by more than q)
    assert len(np.unique(np.round(r / qf))) > 0.9 * len(r)
    # no inserted particle overlaps another or a fine particle (brute force)
    allx = fine.read(dem.POS)
    allr = fine.read(dem.RADIUS)
    pairs = oracle.pairs(oracle_params(fine_wl), allx, allr, 0.0, method="brute")
    assert not np.any(pairs[:, 1] >= fine_wl.n)
    # mass conservation: inserted + carry = entered (exact, integer units; the GPU's carry equals it above)
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
    # fine controller force u pi r^2 w(s): u = (K_p + K_i T_c) e at the first call, and the
    # error e = sigma_coarse - sigma_fine is a difference of two stresses each within 1e-5 of
    # its cell's scale, so |du| <= 1e-5 (|sigma_c| + |sigma_f|) (K_p + K_i T_c): the bound
    # below, plus float rounding of the product (the clip only lowers the sensitivity)
    ff = fine.read(dem.FEXT)[:fine_wl.n]
    Tc = spec["interval"] * spec["dt"]
    sig = np.abs(out["lay"][:, :, 2])                  # (level, cell): sigma_zz of the top face's layer
    du = 1e-5 * (sig[0] + sig[1]).max() * (spec["kp"] + spec["ki"] * Tc)
    tol = du * np.pi * fine_wl.r[:, None] ** 2 + 1e-6 * np.abs(out["fext_f"]) + 1e-15
    assert np.all(np.abs(ff - out["fext_f"]) <= tol), np.max(np.abs(ff - out["fext_f"]) / tol)
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
    Tc = spec["interval"] * spec["dt"]
    sig = np.abs(out["lay"][:, :, 2])
    du = 1e-5 * (sig[0] + sig[1]).max() * (spec["kp"] + spec["ki"] * Tc)   # as in the test above
    tol = du * np.pi * fine_wl.r[:, None] ** 2 + 1e-6 * np.abs(ref_f) + 1e-15
    assert np.all(np.abs(ff - ref_f) <= tol)
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
