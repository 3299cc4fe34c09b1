"""Pins of the coupling oracle (Sec. 2.3) against closed forms and invariants (CPU only)."""
import math

import numpy as np
import pytest

import oracle

RHO = 2500.0
E, NU = 1e7, 0.25


def _P(lo, hi, periodic=(True, True, False), floor=False, g=(0, 0, 0)):
    return oracle.make_params(E=E, nu=NU, e=0.6, mu=0.4, dt=1e-6, g=g, lo=lo, hi=hi, periodic=periodic, floor=floor)


def _spec(**kw):
    s = dict(lo=(0.0, 0.0, 0.0), hi=(0.024, 0.024, 0.02), feed_faces=1 << 5, drain_faces=0, surface_cell=0.012,
             layer=0.012, corr_cell=0.008, interval=15, bins=16, alpha=2.0, kp=1.0, ki=0.0, kv=0.5, mode=0,
             max_attempts=100, seed=7, mass_unit=1e-15, max_insert=256, dt=1e-6)
    s.update(kw)
    return s


def _state(x, v=None, r=None, rho=RHO):
    x = np.atleast_2d(np.asarray(x, dtype=float))
    n = len(x)
    v = np.zeros((n, 3)) if v is None else np.atleast_2d(np.asarray(v, dtype=float))
    r = np.full(n, 1e-3) if r is None else np.asarray(r, dtype=float)
    m = rho * 4.0 / 3.0 * math.pi * r ** 3
    return dict(x=x, v=v, w=np.zeros((n, 3)), r=r, m=m, id=np.arange(n))


def _coupler(spec, Pc, Pf, rmax_f=1e-3, idcap=64):
    qf = oracle.quantum(Pf[9:12], Pf[12:15])
    return oracle.Coupler(spec, Pc, Pf, rmax_f, RHO, idcap), qf


def test_eq7_stress_of_one_compressed_pair_and_two_moving_particles():
    # One contact inside a transition cell: both ends lie in the cell, each adds
    # 1/2 r_ij f_ij, so sigma_zz = F d / V.  Kinetic part: two equal masses
    # moving at +-u along z add 2 m u^2 / V.
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    Pc, Pf = _P(lo, hi), _P(lo, hi)
    spec = _spec()
    cp, qf = _coupler(spec, Pc, Pf)
    d = 2e-3 - 4e-6
    fine = _state([[0.006, 0.006, 0.015], [0.006, 0.006, 0.015 + d]], v=[[0, 0, 0], [0, 0, 0]])
    out = cp.call(_state([[0.006, 0.006, 0.05]]), fine, 0.0, 0.0)
    c = oracle.pair_coeffs(Pf, 1e-3, 1e-3, fine["m"][0], fine["m"][1], 4e-6)
    F = c["kn"] * 4e-6
    V = 0.012 * 0.012 * 0.012
    cell = 0                      # x, y < 12 mm
    assert out["lay"][1, cell, 2] == pytest.approx(F * d / V, rel=1e-12)
    assert abs(out["lay"][1, cell, 0]) < 1e-12 * F * d / V      # no xx part for a vertical contact
    u = 0.3
    moving = _state([[0.003, 0.003, 0.012], [0.009, 0.009, 0.012]], v=[[0, 0, u], [0, 0, -u]])
    out = cp.call(_state([[0.006, 0.006, 0.05]]), moving, 0.0, 0.0)
    m = moving["m"][0]
    # same cell, <v> = 0, v' = +-u
    assert out["lay"][1, 0, 2] == pytest.approx(2 * m * u * u / V, rel=1e-12)
    assert out["lay"][1, 0, 0] == 0.0


def test_entry_through_the_feed_face_only_and_histogram_bin():
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    Pc, Pf = _P(lo, hi), _P(lo, hi)
    cp, qf = _coupler(_spec(), Pc, Pf, idcap=4)
    r = np.array([2e-3, 2e-3, 2e-3])
    before = _state([[0.006, 0.006, 0.0215], [0.018, 0.018, 0.03], [0.006, 0.018, 0.025]], r=r)
    cp.record(before["x"], before["id"])
    after = _state([[0.006, 0.006, 0.0195], [0.018, 0.018, 0.029], [0.006, 0.018, 0.0199]], r=r)
    out = cp.call(after, _state([[0.012, 0.012, 0.003]]), 0.0, 0.0)
    m = after["m"][0]
    # particles 0 and 2 entered through the top face (cells 0 and 2 of the 2 x 2 grid); particle 1 did not
    expect = np.zeros(4, dtype=np.int64)
    expect[0] = round(m / 1e-15)
    expect[2] = round(m / 1e-15)
    assert np.array_equal(out["cross"].astype(np.int64), expect)
    # diameter histogram of r / alpha = 1 mm over [0, r_max fine]: the top bin
    assert out["hist"][0].sum() == 1 and out["hist"][0][-1] == 1


def test_insertion_conserves_mass_and_makes_no_overlaps():
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    Pc, Pf = _P(lo, hi), _P(lo, hi)
    cp, qf = _coupler(_spec(), Pc, Pf, idcap=200)
    rng = np.random.default_rng(3)
    xs = np.column_stack([rng.uniform(0, 0.024, 72), rng.uniform(0, 0.024, 72), np.full(72, 0.021)])
    cg = _state(xs, r=np.full(72, 2e-3))
    cp.record(cg["x"], cg["id"])
    cg2 = dict(cg)
    cg2["x"] = xs - np.array([0, 0, 0.002])
    fine = _state([[0.012, 0.012, 0.003]])
    out = cp.call(cg2, fine, 0.0, 0.0)
    ins = np.concatenate([out["ins_x"][c, :out["nins"][c]] for c in range(4)])
    assert len(ins) > 20
    mass_in = np.array([sum(round(m / 1e-15) for m in out["ins_m"][c, :out["nins"][c]]) for c in range(4)])
    assert np.array_equal(mass_in + out["carry"], out["cross"].astype(np.int64))
    x = np.vstack([fine["x"], ins[:, :3]])
    r = np.concatenate([fine["r"], ins[:, 3]])
    assert len(oracle.pairs(Pf, x, r, 0.0, method="brute")) == 0
    # inside the region, within r of nothing outside: below the top face by at least r
    assert np.all(x[1:, 2] + r[1:] <= 0.02 + 1e-12)


def test_controllers_special_cases():
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    Pc, Pf = _P(lo, hi), _P(lo, hi)
    # identical coarse and fine material in the correction cells: v* = v_cg -> no force on coarse particles
    v = [[0.1, 0.0, -0.2]]
    for mode in (0, 1):
        cp, qf = _coupler(_spec(mode=mode), Pc, Pf)
        out = cp.call(_state([[0.004, 0.004, 0.004]], v=v, r=[1e-3]), _state([[0.004, 0.004, 0.004]], v=v),
                      0.0, 0.0)
        assert np.abs(out["fext_c"]).max() == 0.0
    # a velocity mismatch gives F = kv m (v_f - v_cg) / T_c (mode 0)
    cp, qf = _coupler(_spec(mode=0), Pc, Pf)
    c = _state([[0.004, 0.004, 0.004]], v=[[0.0, 0.0, 0.0]], r=[1e-3])
    out = cp.call(c, _state([[0.004, 0.004, 0.004]], v=[[0.0, 0.0, -0.3]]), 0.0, 0.0)
    assert out["fext_c"][0, 2] == pytest.approx(0.5 * c["m"][0] * (-0.3) / 15e-6, rel=1e-12)
    # mass-flow mode multiplies the fine velocity by phi_f / phi_cg (here 8 particles vs 1: capped at 4)
    cp, qf = _coupler(_spec(mode=1), Pc, Pf)
    fine = _state([[0.002 + 0.002 * i, 0.002 + 0.002 * j, 0.002 + 0.002 * k] for i in range(2) for j in range(2)
                   for k in range(2)], v=[[0.0, 0.0, -0.1]] * 8)
    out = cp.call(_state([[0.004, 0.004, 0.004]], r=[1e-3]), fine, 0.0, 0.0)
    assert out["fext_c"][0, 2] == pytest.approx(0.5 * c["m"][0] * (-0.1 * 4.0) / 15e-6, rel=1e-12)
    # ... except in correction cells centred below velocity_below (the region's 20 mm are two
    # cells of 10 mm: the one holding both particles is centred at 5 mm): there the target is
    # the fine velocity itself, as in mode 0
    for vb, f in ((0.006, 1.0), (0.004, 4.0)):
        cp, qf = _coupler(_spec(mode=1, velocity_below=vb), Pc, Pf)
        out = cp.call(_state([[0.004, 0.004, 0.004]], r=[1e-3]), fine, 0.0, 0.0)
        assert out["fext_c"][0, 2] == pytest.approx(0.5 * c["m"][0] * (-0.1 * f) / 15e-6, rel=1e-12)
    # PI with ki = 0: the force on a fine particle is linear in the stress mismatch
    spec = _spec(kp=2.0)
    cp, qf = _coupler(spec, Pc, Pf)
    d = 2e-3 - 4e-6
    cg = _state([[0.006, 0.006, 0.0185], [0.006, 0.006, 0.0185 - d]], r=[1e-3, 1e-3])
    probe = _state([[0.018, 0.006, 0.0195]], v=[[0, 0, -1e-3]])
    out = cp.call(cg, probe, 0.0, 0.0)
    ctrl = out["ctrl"]
    e = ctrl[0, 0]
    assert ctrl[0, 2] == pytest.approx(2.0 * e, rel=1e-14)


def _Pw(lo, hi, walls):
    return oracle.make_params(E=E, nu=NU, e=0.6, mu=0.4, dt=1e-6, lo=lo, hi=hi, periodic=(False, False, False),
                              walls=walls)


def test_eq7_stress_includes_an_axisymmetric_wall_contact():
    # one fine particle at rest pressed by delta into a vertical cylinder wall (axis at the
    # region's centre, radius 11 mm) inside a transition cell: the wall adds r_c f with r_c
    # the branch vector from the contact point to the centre, |r_c| = r - delta, along the
    # wall normal -x: sigma_xx = (r - delta) F / V with the Hertz force F = 4/3 E* sqrt(r delta) delta
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    R, r, delta = 0.011, 1e-3, 3e-6
    walls = dict(axis=(0.012, 0.012), points=[(R, 0.0), (R, 0.06)])
    Pc, Pf = _P(lo, hi), _Pw(lo, hi, walls)
    cp, qf = _coupler(_spec(), Pc, Pf)
    fine = _state([[0.012 + R - (r - delta), 0.012, 0.015]])
    out = cp.call(_state([[0.006, 0.006, 0.05]]), fine, 0.0, 0.0)
    Estar = E / (2.0 * (1.0 - NU * NU))
    F = 4.0 / 3.0 * Estar * math.sqrt(r * delta) * delta
    V = 0.012 ** 3
    cell = 3                        # x, y >= 12 mm: cell (1, 1) of the 2 x 2 grid
    assert out["lay"][1, cell, 0] == pytest.approx((r - delta) * F / V, rel=1e-9)
    assert abs(out["lay"][1, cell, 1]) < 1e-9 * F * r / V and abs(out["lay"][1, cell, 2]) < 1e-9 * F * r / V
    # the same particle with the wall removed: no contact part
    out0 = _coupler(_spec(), Pc, _P(lo, hi, periodic=(False, False, False)))[0].call(
        _state([[0.006, 0.006, 0.05]]), fine, 0.0, 0.0)
    assert np.abs(out0["lay"][1, :, :6]).max() == 0.0


def test_insertion_keeps_clear_of_the_fine_levels_walls():
    # the feed face's cells reach beyond a cylinder wall of radius 10 mm about the region's
    # centre; without the wall some inserted spheres straddle it or lie outside it, with it
    # every one lies inside, clear of it
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    R = 0.010
    walls = dict(axis=(0.012, 0.012), points=[(R, 0.0), (R, 0.06)])
    rng = np.random.default_rng(5)
    xs = np.column_stack([rng.uniform(0, 0.024, 72), rng.uniform(0, 0.024, 72), np.full(72, 0.021)])
    cg = _state(xs, r=np.full(72, 2e-3))
    cg2 = dict(cg)
    cg2["x"] = xs - np.array([0, 0, 0.002])
    fine = _state([[0.012, 0.012, 0.003]])
    res = {}
    for name, Pf in (("open", _P(lo, hi, periodic=(False, False, False))), ("walled", _Pw(lo, hi, walls))):
        cp, qf = _coupler(_spec(), _P(lo, hi), Pf, idcap=200)
        cp.record(cg["x"], cg["id"])
        out = cp.call(cg2, fine, 0.0, 0.0)
        ins = np.concatenate([out["ins_x"][c, :out["nins"][c]] for c in range(4)])
        x, r = ins[:, :3], ins[:, 3]
        rho = np.hypot(x[:, 0] - 0.012, x[:, 1] - 0.012)
        res[name] = (len(ins), rho + r > R)
        mass_in = np.array([sum(round(m / 1e-15) for m in out["ins_m"][c, :out["nins"][c]]) for c in range(4)])
        assert np.array_equal(mass_in + out["carry"], out["cross"].astype(np.int64))
    assert res["open"][1].any()
    assert res["walled"][0] > 10 and not res["walled"][1].any()


def test_insertion_inside_a_closed_cone():
    # a cone narrowing downwards (radius 4 mm at z = 0 to 16 mm at z = 24 mm), closed below by a
    # disk (a horizontal segment, which the inside test skips): the top face's cells reach
    # beyond the cone; every inserted sphere lies inside it, clear of it, above the disk
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    axis = (0.012, 0.012)
    pts = [(0.0, 0.0), (0.004, 0.0), (0.016, 0.024), (0.016, 0.06)]
    Pf = _Pw(lo, hi, dict(axis=axis, points=pts))
    rng = np.random.default_rng(9)
    xs = np.column_stack([rng.uniform(0, 0.024, 72), rng.uniform(0, 0.024, 72), np.full(72, 0.021)])
    cg = _state(xs, r=np.full(72, 2e-3))
    cg2 = dict(cg)
    cg2["x"] = xs - np.array([0, 0, 0.002])
    cp, qf = _coupler(_spec(), _P(lo, hi), Pf, idcap=200)
    cp.record(cg["x"], cg["id"])
    out = cp.call(cg2, _state([[0.012, 0.012, 0.003]]), 0.0, 0.0)
    ins = np.concatenate([out["ins_x"][c, :out["nins"][c]] for c in range(4)])
    assert len(ins) > 10
    x, r = ins[:, :3], ins[:, 3]
    rho = np.hypot(x[:, 0] - axis[0], x[:, 1] - axis[1])
    wall = 0.004 + 0.5 * x[:, 2]                      # the cone's radius at each centre's height
    c = 1.0 / math.hypot(1.0, 0.5)                    # the cone's normal against the horizontal
    assert np.all((wall - rho) * c >= r)             # inside, at least r from the cone
    assert np.all(x[:, 2] >= r)


def _hertz(r, delta):
    # two equal spheres pressed together by delta: F = 4/3 E* sqrt(R delta) delta with
    # 1/E* = 2 (1 - nu^2) / E and R = r / 2 (Hertz)
    return 4.0 / 3.0 * E / (2.0 * (1.0 - NU * NU)) * math.sqrt(0.5 * r * delta) * delta


def _pressed_pair(delta, vx, r=1e-3):
    # a coarse pair inside transition cell 0 (x, y < 12 mm, 1.5 and 3.5 mm below the top feed
    # face), moving together along x: no kinetic stress, no dashpot, no tangential force, so the
    # cell's sigma_zz = F d / V and its largest speed is |vx|
    d = 2 * r - delta
    return _state([[0.006, 0.006, 0.0185], [0.006, 0.006, 0.0185 - d]], v=[[vx, 0, 0], [vx, 0, 0]],
                  r=[r, r]), _hertz(r, delta) * d / 0.012 ** 3


def test_stress_pi_controller_integrates_the_error_over_calls():
    # Sec. 2.3 stress controller with K_i != 0 over three calls: I = sum_k e_k T_c and
    # u = K_p e + K_i I, the error being coarse minus fine face-normal stress (Eq. 7)
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    Tc = 15 * 1e-6
    kp, ki = 0.7, 1.0 / (10 * Tc)
    cp, qf = _coupler(_spec(kp=kp, ki=ki), _P(lo, hi), _P(lo, hi))
    probe = _state([[0.018, 0.018, 0.0195]])            # fine: one particle at rest, no stress
    errs = []
    for delta in (4e-6, 7e-6, 2e-6):
        cg, sig = _pressed_pair(delta, vx=5.0)
        out = cp.call(cg, probe, 0.0, 0.0)
        errs.append(sig)
        e, integ, u = out["ctrl"][0]
        assert e == pytest.approx(sig, rel=1e-10)
        assert integ == pytest.approx(sum(errs) * Tc, rel=1e-10)
        assert u == pytest.approx(kp * sig + ki * sum(errs) * Tc, rel=1e-10)
        # cells without coarse or fine stress: zero error, and the integral stays zero
        assert np.abs(out["ctrl"][1:]).max() == 0.0


def test_stress_controller_force_on_fine_particles_fades_linearly():
    # the controller's stress u acts on each fine particle of the layer as u pi r^2 along the
    # face's inward normal (-z for the top face), faded linearly to zero at s = 1.5 d_fine
    # below the face and zero deeper; far below the coarse cell's largest speed, nothing clips
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    rf = 0.5e-3
    kp = 1.3
    cp, qf = _coupler(_spec(kp=kp), _P(lo, hi), _P(lo, hi), rmax_f=rf)
    s = np.array([0.2e-3, 0.7e-3, 1.2e-3, 1.49e-3, 1.6e-3, 4.0e-3])
    xf = np.column_stack([0.0015 + 0.0018 * np.arange(len(s)), np.full(len(s), 0.003), 0.02 - s])
    fine = _state(xf, r=np.full(len(s), rf))
    cg, sig = _pressed_pair(4e-6, vx=5.0)
    out = cp.call(cg, fine, 0.0, 0.0)
    u = out["ctrl"][0, 2]
    assert u == pytest.approx(kp * sig, rel=1e-10)
    w = np.maximum(0.0, 1.0 - s / (1.5 * 2 * rf))
    expect = -u * math.pi * rf * rf * w
    assert np.allclose(out["fext_f"][:, 2], expect, rtol=1e-12, atol=0)
    assert np.abs(out["fext_f"][:, :2]).max() == 0.0
    assert out["fext_f"][4:, 2].tolist() == [0.0, 0.0]


def test_stress_controller_force_is_clipped_at_the_coarse_cells_largest_speed():
    # the force is scaled down along itself so that the fine particle's speed after one step,
    # |v + dt F / m|, equals the coarse cell's largest speed where it would exceed it; a particle
    # already faster than that gets no force, one that the force slows down keeps all of it
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    rf, dt = 0.5e-3, 1e-6
    mf = RHO * 4.0 / 3.0 * math.pi * rf ** 3
    vm = 0.006
    cases = (((0.005, 0.0, -0.003), "clipped"), ((0.0, 0.0, 0.02), "free"), ((0.0, 0.0, -0.0061), "zero"),
             ((0.004, 0.0, 0.0), "clipped"))
    for vf, what in cases:
        cp, qf = _coupler(_spec(kp=1e3), _P(lo, hi), _P(lo, hi), rmax_f=rf)
        fine = _state([[0.003, 0.003, 0.0198]], v=[vf], r=[rf])
        cg, sig = _pressed_pair(40e-6, vx=vm)
        out = cp.call(cg, fine, 0.0, 0.0)
        assert out["lay"][0, 0, 10] == pytest.approx(vm, rel=1e-15)        # the coarse cell's largest speed
        free = -1e3 * sig * math.pi * rf * rf * (1.0 - 0.2e-3 / (3 * rf))
        assert dt * abs(free) / mf > 3 * vm                                # the unclipped kick is large
        F = out["fext_f"][0]
        assert F[0] == 0.0 and F[1] == 0.0
        v1 = np.array(vf) + dt * F / mf
        if what == "free":
            assert F[2] == pytest.approx(free, rel=1e-12)
            assert np.linalg.norm(v1) < vm
        elif what == "zero":
            assert F[2] == 0.0
        else:
            assert 0.0 < F[2] / free < 1.0
            assert np.linalg.norm(v1) == pytest.approx(vm, rel=1e-12)


def test_inserted_radii_are_uniform_within_the_drawn_bin():
    # SSI draws a histogram bin, then a radius uniformly inside it, in continuous space (Sec.
    # 2.3 inserts spheres of the coarse particles' fine-scale size distribution): coarse grains
    # of r = 1.7 mm at alpha = 2 give r / alpha = 0.85 mm, bin 13 of 16 over [0, 1 mm); every
    # inserted radius lies in [13, 14) / 16 mm, and their distribution is uniform there
    from scipy import stats
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    cp, qf = _coupler(_spec(max_insert=512), _P(lo, hi), _P(lo, hi), idcap=400)
    rng = np.random.default_rng(11)
    xs = np.column_stack([rng.uniform(0, 0.024, 300), rng.uniform(0, 0.024, 300), np.full(300, 0.021)])
    cg = _state(xs, r=np.full(300, 1.7e-3))
    cp.record(cg["x"], cg["id"])
    cg2 = dict(cg)
    cg2["x"] = xs - np.array([0, 0, 0.002])
    out = cp.call(cg2, _state([[0.012, 0.012, 0.003]]), 0.0, 0.0)
    assert out["hist"][:, 13].sum() == 300 and out["hist"].sum() == 300
    r = np.concatenate([out["ins_x"][c, :out["nins"][c], 3] for c in range(4)])
    assert len(r) > 80                   # the slabs fill up before the quota is met
    w = 1e-3 / 16
    assert np.all((r >= 13 * w) & (r < 14 * w))
    assert stats.kstest((r - 13 * w) / w, "uniform").pvalue > 1e-3
    # not on the fine level's position grid
    assert np.mean(np.abs(r / qf - np.round(r / qf)) < 1e-6) < 0.01
    # the borderline report: none without a band, every cell that drew a candidate with a band
    # wider than the region
    assert np.all(out["border"] == -1)
    cp2, _ = _coupler(_spec(max_insert=512), _P(lo, hi), _P(lo, hi), idcap=400)
    cp2.band = 1.0
    cp2.record(cg["x"], cg["id"])
    out2 = cp2.call(cg2, _state([[0.012, 0.012, 0.003]]), 0.0, 0.0)
    assert np.all(out2["border"] == 0)


def test_eq7_stress_takes_the_stored_tangential_overlap():
    # a compressed vertical pair at rest holding a stored overlap xi along x (in the frame of the
    # lower ID, i.e. of the upper sphere's partner below it): the contact force on the lower-ID
    # sphere is k_n delta n - k_t xi, so the cell's sigma_xz = 1/2 d (-k_t xi) / V besides
    # sigma_zz = k_n delta d / V; without the history sigma_xz is zero
    lo, hi = (0, 0, 0), (0.024, 0.024, 0.06)
    Pc, Pf = _P(lo, hi), _P(lo, hi)
    delta, xi = 4e-6, 2e-7
    d = 2e-3 - delta
    fine = _state([[0.006, 0.006, 0.015 + d], [0.006, 0.006, 0.015]])   # ID 0 above ID 1: n = +z
    c = oracle.pair_coeffs(Pf, 1e-3, 1e-3, fine["m"][0], fine["m"][1], delta)
    V = 0.012 ** 3
    cg = _state([[0.006, 0.006, 0.05]])
    out0 = _coupler(_spec(), Pc, Pf)[0].call(cg, fine, 0.0, 0.0)
    assert out0["lay"][1, 0, 4] == 0.0
    fine["hist"] = (np.array([0]), np.array([1]), np.array([[xi, 0.0, 0.0]]))
    out = _coupler(_spec(), Pc, Pf)[0].call(cg, fine, 0.0, 0.0)
    assert out["lay"][1, 0, 2] == pytest.approx(c["kn"] * delta * d / V, rel=1e-12)
    assert out["lay"][1, 0, 4] == pytest.approx(-0.5 * d * c["kt"] * xi / V, rel=1e-12)
