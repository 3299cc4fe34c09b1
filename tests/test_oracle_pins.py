"""Pins of the FP64 oracle against closed forms, invariants and textbook results.

None of these re-types the oracle's own formulas: each checks a consequence
that a dropped term, a wrong sign or index, or a transposed operand would
break (values the paper prints, algebraic identities of Eq. 6, the Hertz
impact solution, a scipy solution of the 1-D contact ODE, the 5/7 rolling
law, conservation laws, brute force vs cell list).
"""
import math

import numpy as np
import pytest

import oracle

RHO = 2500.0
E = 1.0e7
NU = 0.25


def sphere_mass(r, rho=RHO):
    return rho * 4.0 / 3.0 * math.pi * r ** 3


# --------------------------------------------------------------- Eq. 6 pins

def test_beta_special_values():
    # e = 1 is an elastic contact: no damping (Eq. 6).
    assert oracle.beta(1.0) == 0.0
    # ln(0.9) = -0.1053605; beta = ln e / sqrt(ln^2 e + pi^2), evaluated by hand.
    assert oracle.beta(0.9) == pytest.approx(-0.0335184, abs=2e-7)
    assert oracle.beta(0.5) == pytest.approx(-0.2154538, abs=2e-7)
    # e -> 0 is the critically damped limit beta -> -1.
    assert oracle.beta(1e-300) == pytest.approx(-1.0, abs=2e-3)
    # beta is negative and increasing in e on (0, 1).
    es = np.linspace(0.05, 0.99, 30)
    bs = [oracle.beta(e) for e in es]
    assert all(b < 0 for b in bs) and np.all(np.diff(bs) > 0)


def test_effective_moduli_closed_form():
    # Same material on both sides: E_eff = E / (2 (1 - nu^2)),
    # G_eff = E / (4 (2 - nu)(1 + nu)); 5.333e6 Pa and 1.1429e6 Pa at E = 1e7, nu = 0.25.
    P = oracle.make_params(E=E, nu=NU, e=0.9, mu=0.5, dt=1e-6)
    c = oracle.pair_coeffs(P, 1e-3, 1.2e-3, 1e-5, 2e-5, 1e-6)
    assert c["Eeff"] == pytest.approx(5.333333e6, rel=1e-6)
    assert c["Geff"] == pytest.approx(1.142857e6, rel=1e-6)
    assert c["Reff"] == pytest.approx(1e-3 * 1.2e-3 / 2.2e-3, rel=1e-14)
    assert c["meff"] == pytest.approx(1e-5 * 2e-5 / 3e-5, rel=1e-14)
    w = oracle.pair_coeffs(P, 1e-3, 0.0, 1e-5, 0.0, 1e-6, wall=True)
    assert w["Reff"] == 1e-3 and w["meff"] == 1e-5


def test_damping_matches_the_2sqrt56_form():
    # The widely used form gamma = -2 sqrt(5/6) beta sqrt(S m_eff) with
    # S_n = 2 E_eff sqrt(R delta) and S_t = 8 G_eff sqrt(R delta) is the same
    # law as Eq. 6 (4 * 5/6 * 2 = 20/3 = 5 * 4/3); checking it guards against a
    # garbled factor in either gamma.
    P = oracle.make_params(E=2.5e7, nu=0.25, e=0.5, mu=0.2, dt=1e-6)
    ri, rj, mi, mj, d = 1.4e-3, 2.8e-3, 1.1e-5, 9e-5, 3e-6
    c = oracle.pair_coeffs(P, ri, rj, mi, mj, d)
    b = oracle.beta(0.5)
    Sn = 2.0 * c["Eeff"] * math.sqrt(c["Reff"] * d)
    St = 8.0 * c["Geff"] * math.sqrt(c["Reff"] * d)
    assert c["gn"] == pytest.approx(-2.0 * math.sqrt(5.0 / 6.0) * b * math.sqrt(Sn * c["meff"]), rel=1e-13)
    assert c["gt"] == pytest.approx(-2.0 * math.sqrt(5.0 / 6.0) * b * math.sqrt(St * c["meff"]), rel=1e-13)
    # and the damping is non-negative (dissipative) for e <= 1
    assert c["gn"] > 0 and c["gt"] > 0


@pytest.mark.parametrize("alpha", [2.0, 4.0, 32.0])
def test_coarse_grain_scaling(alpha):
    # Sec. 2.2: with rho, e, E, mu fixed and r -> alpha r, the stiffnesses
    # scale with alpha and the damping coefficients with alpha^2 (for the same
    # contact geometry scaled by alpha: delta -> alpha delta, m -> alpha^3 m).
    P = oracle.make_params(E=2.5e7, nu=0.25, e=0.5, mu=0.2, dt=1e-6)
    ri, rj, d = 1.4e-3, 1.1e-3, 2e-6
    base = oracle.pair_coeffs(P, ri, rj, sphere_mass(ri, 1000), sphere_mass(rj, 1000), d)
    cg = oracle.pair_coeffs(P, alpha * ri, alpha * rj, sphere_mass(alpha * ri, 1000),
                            sphere_mass(alpha * rj, 1000), alpha * d)
    for k in ("kn", "kt"):
        assert cg[k] / base[k] == pytest.approx(alpha, rel=1e-13)
    for k in ("gn", "gt"):
        assert cg[k] / base[k] == pytest.approx(alpha ** 2, rel=1e-13)


# ------------------------------------------------------------- contact set

def _random_cloud(n, L, Lz, rmin, rmax, seed):
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(0, L, n), rng.uniform(0, L, n), rng.uniform(-0.1 * Lz, 1.2 * Lz, n)])
    r = rng.uniform(rmin, rmax, n)
    return x, r


@pytest.mark.parametrize("periodic", [(True, True, False), (False, False, False), (True, False, False)])
@pytest.mark.parametrize("extra", [0.0, 2e-4])
def test_brute_force_equals_cell_list(periodic, extra):
    L, Lz = 0.02, 0.03
    x, r = _random_cloud(1500, L, Lz, 0.8e-3, 1.2e-3, seed=11)
    P = oracle.make_params(E=E, nu=NU, e=0.9, mu=0.5, dt=1e-6, lo=(0, 0, 0), hi=(L, L, Lz),
                           periodic=periodic)
    a = oracle.pairs(P, x, r, extra, method="brute")
    b = oracle.pairs(P, x, r, extra, method="cells")
    assert len(a) > 100
    assert np.array_equal(a, b)


def test_min_image_pairs_across_the_periodic_boundary():
    # Two spheres straddling x = 0 / x = L overlap through the periodic image.
    L = 0.01
    x = np.array([[0.0004, 0.005, 0.005], [L - 0.0012, 0.005, 0.005]])
    r = np.array([1e-3, 1e-3])
    per = oracle.make_params(E=E, nu=NU, e=0.9, mu=0.5, dt=1e-6, hi=(L, L, L), periodic=(True, True, False))
    non = oracle.make_params(E=E, nu=NU, e=0.9, mu=0.5, dt=1e-6, hi=(L, L, L))
    assert oracle.pairs(per, x, r, method="brute").tolist() == [[0, 1]]
    assert oracle.pairs(non, x, r, method="brute").tolist() == []


# ------------------------------------------------------ dynamics and laws

def _dense_overlapping(n_side, spacing, r, seed, L=None, vel=0.05, omega=20.0):
    rng = np.random.default_rng(seed)
    g = np.arange(n_side) * spacing + spacing / 2
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x = np.column_stack([X.ravel(), Y.ravel(), Z.ravel()]) + rng.uniform(-0.05, 0.05, (n_side ** 3, 3)) * spacing
    n = len(x)
    rad = rng.uniform(0.9 * r, 1.1 * r, n)
    v = rng.normal(0, vel, (n, 3))
    w = rng.normal(0, omega, (n, 3))
    return x, v, w, rad


def test_momentum_conserved_without_walls_and_gravity():
    # Newton's third law per pair: total linear momentum stays constant
    # in a periodic box with no external force.
    L = 6 * 2.0e-3
    x, v, w, r = _dense_overlapping(6, 2.0e-3, 1.02e-3, seed=3)
    P = oracle.make_params(E=E, nu=NU, e=0.7, mu=0.5, dt=2e-6, hi=(L, L, L), periodic=(True, True, True))
    m = sphere_mass(r)
    sim = oracle.Sim(P, x, v, w, r, m)
    p0 = (m[:, None] * sim.v).sum(0)
    scale = (m[:, None] * np.abs(sim.v)).sum()
    sim.run(300)
    p1 = (m[:, None] * sim.v).sum(0)
    assert np.abs(p1 - p0).max() <= 1e-12 * scale
    # contacts actually happened
    assert sim.nh[0] > 50


def test_pair_forces_sum_to_gravity():
    # Each pair force enters i and j with opposite signs, so the sum of all
    # forces equals the total weight (no floor).
    L = 6 * 2.0e-3
    x, v, w, r = _dense_overlapping(6, 2.0e-3, 1.03e-3, seed=4)
    P = oracle.make_params(E=E, nu=NU, e=0.5, mu=0.3, dt=2e-6, g=(0.3, -1.0, -9.81), hi=(L, L, L),
                           periodic=(True, True, True))
    m = sphere_mass(r)
    F, T, hist, fabs = oracle.Sim(P, x, v, w, r, m).evaluate()
    weight = m.sum() * np.array([0.3, -1.0, -9.81])
    assert np.abs(F.sum(0) - weight).max() <= 1e-13 * fabs.sum()
    assert len(hist[0]) > 100


def _energy(sim):
    I = 0.4 * sim.m * sim.r ** 2
    return 0.5 * (sim.m * (sim.v ** 2).sum(1)).sum() + 0.5 * (I * (sim.w ** 2).sum(1)).sum()


def test_energy_conserved_to_second_order_when_elastic_and_frictionless():
    # e = 1, mu = 0: the contact law is conservative (Hertz potential), and
    # velocity Verlet conserves energy to O(dt^2).
    L = 5 * 2.0e-3
    x, v, w, r = _dense_overlapping(5, 2.0e-3, 0.99e-3, seed=5, vel=0.3, omega=0.0)
    P0 = dict(E=E, nu=NU, e=1.0, mu=0.0, hi=(L, L, L), periodic=(True, True, True))
    m = sphere_mass(r)
    T_end = 4e-4
    Eeff = E / (2 * (1 - NU ** 2))

    def potential(sim):
        # elastic energy stored in the overlaps: (8/15) E_eff sqrt(R) delta^(5/2)
        _, _, hist, _ = sim.evaluate()
        pe = 0.0
        for a, b in zip(hist[0], hist[1]):
            d = sim.x[a] - sim.x[b]
            d -= L * np.round(d / L)
            delta = r[a] + r[b] - np.linalg.norm(d)
            R = r[a] * r[b] / (r[a] + r[b])
            pe += 8.0 / 15.0 * Eeff * math.sqrt(R) * delta ** 2.5
        return pe

    errs = []
    for dt in (2e-6, 1e-6):
        sim = oracle.Sim(oracle.make_params(dt=dt, **P0), x, v, w, r, m)
        e0 = _energy(sim) + potential(sim)
        sim.run(int(round(T_end / dt)))
        errs.append(abs(_energy(sim) + potential(sim) - e0) / e0)
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


# ------------------------------------------------------------ two spheres

def _head_on(v0, e, dt, r=1e-3):
    """Two equal spheres meeting head-on; returns (restitution, contact time, max overlap)."""
    P = oracle.make_params(E=E, nu=NU, e=e, mu=0.5, dt=dt, lo=(-0.01, -0.01, -0.01), hi=(0.01, 0.01, 0.01))
    x = np.array([[-r - 0.25 * v0 * dt * 3, 0, 0], [r + 0.25 * v0 * dt * 3, 0, 0]])
    v = np.array([[0.5 * v0, 0, 0], [-0.5 * v0, 0, 0]])
    m = np.full(2, sphere_mass(r))
    sim = oracle.Sim(P, x, v, np.zeros((2, 3)), np.full(2, r), m, use_cells=False)
    steps_in, dmax, started, t = 0, 0.0, False, 0
    gaps = []
    while True:
        sim.run(1)
        t += 1
        gap = np.linalg.norm(sim.x[1] - sim.x[0]) - 2 * r
        gaps.append(gap)
        if gap < 0:
            started = True
            steps_in += 1
            dmax = max(dmax, -gap)
        elif started:
            break
        assert t < 10_000_000
    # contact duration from the linear interpolation of the gap's two zero crossings
    g = np.array(gaps)
    neg = np.nonzero(g < 0)[0]
    i0, i1 = neg[0], neg[-1]
    t_in = (i0 - 1) + g[i0 - 1] / (g[i0 - 1] - g[i0])
    t_out = i1 + g[i1] / (g[i1] - g[i1 + 1])
    vrel = sim.v[1, 0] - sim.v[0, 0]
    return vrel / v0, (t_out - t_in) * dt, dmax


def test_hertz_elastic_impact_closed_form():
    # e = 1 (beta = 0) reduces Eqs. 3 and 6 to Hertz's elastic impact:
    # delta_max = (15 m* v0^2 / (16 E* sqrt(R*)))^(2/5),
    # t_c = 2 (2/5) B(2/5, 1/2) delta_max / v0 = 2.943275 delta_max / v0.
    from scipy.special import beta as B
    r = 1e-3
    v0 = 0.5
    ms = sphere_mass(r) / 2
    Rs = r / 2
    Es = E / (2 * (1 - NU ** 2))
    dmax = (15 * ms * v0 ** 2 / (16 * Es * math.sqrt(Rs))) ** 0.4
    tc = 2 * 0.4 * B(0.4, 0.5) * dmax / v0
    assert 2 * 0.4 * B(0.4, 0.5) == pytest.approx(2.943275, abs=2e-6)
    e_meas, tc_meas, dmax_meas = _head_on(v0, 1.0, dt=2e-7)
    assert e_meas == pytest.approx(1.0, abs=1e-4)
    assert tc_meas == pytest.approx(tc, rel=5e-3)
    assert dmax_meas == pytest.approx(dmax, rel=5e-3)


def _e_model(e):
    """Restitution of the 1-D non-linear damped Hertz ODE, by scipy (independent of the oracle).

    m* x'' = -(k_n(x) x + gamma_n(x) x'),  k_n = 4/3 E* sqrt(R* x),
    gamma_n = -beta sqrt(5 m* k_n); it is scale free, so any (m*, R*, E*, v0) gives the same e.
    """
    from scipy.integrate import solve_ivp
    b = math.log(e) / math.sqrt(math.log(e) ** 2 + math.pi ** 2)
    ms, Rs, Es, v0 = 1.0, 1.0, 1.0, 1.0

    def rhs(t, y):
        x, xd = y
        xp = max(x, 0.0)
        kn = 4.0 / 3.0 * Es * math.sqrt(Rs * xp)
        gn = -b * math.sqrt(5.0 * ms * kn)
        return [xd, -(kn * xp + gn * xd) / ms]

    def out(t, y):
        return y[0]
    out.terminal = True
    out.direction = -1
    sol = solve_ivp(rhs, (0, 100.0), [1e-12, v0], events=out, rtol=1e-12, atol=1e-15, max_step=1e-3)
    return -sol.y_events[0][0][1] / v0


@pytest.mark.slow
@pytest.mark.parametrize("e", [0.9, 0.5])
def test_restitution_matches_the_1d_ode_and_is_velocity_independent(e):
    # For the damped Hertz law of Eq. 6 the restitution depends on beta only;
    # it is not exactly the input e (beta(e) is exact for the linear
    # spring-dashpot), so it is compared with the 1-D ODE solved by scipy.
    em = _e_model(e)
    meas = [_head_on(v0, e, dt=1e-6)[0] for v0 in (0.1, 0.5, 1.0)]
    for m in meas:
        assert m == pytest.approx(em, abs=1e-3)
    assert max(meas) - min(meas) < 1e-3


# ------------------------------------------------------- tangential law

@pytest.mark.slow
def test_sliding_sphere_ends_rolling_at_five_sevenths():
    # A sphere launched sliding on a frictional floor decelerates under
    # kinetic friction mu g until the contact point sticks, then rolls with
    # v = 5/7 v0 and omega_y = v / r (solid sphere, I = 2/5 m r^2).  This pins
    # the tangential force of Eqs. 4-5, the lever arm and sign of the torque,
    # and the rotational half of the integrator.
    r, v0, mu, g = 1e-3, 0.2, 0.3, 9.81
    m = sphere_mass(r)
    P = oracle.make_params(E=E, nu=NU, e=0.5, mu=mu, dt=1e-6, g=(0, 0, -g), lo=(-1, -1, 0), hi=(1, 1, 1),
                           floor=True)
    # start at the static overlap under gravity, delta = (3 m g / (4 E_eff sqrt(r)))^(2/3)
    Eeff = E / (2 * (1 - NU ** 2))
    d0 = (3 * m * g / (4 * Eeff * math.sqrt(r))) ** (2 / 3)
    sim = oracle.Sim(P, [[0, 0, r - d0]], [[v0, 0, 0]], [[0, 0, 0]], [r], [m], use_cells=False)
    t_roll = 2 * v0 / (7 * mu * g)
    sim.run(int(t_roll / 1e-6 * 0.5))
    # mid-slide: speed has dropped by mu g t, spin grown by 5 mu g t / (2 r)
    t = int(t_roll / 1e-6 * 0.5) * 1e-6
    assert sim.v[0, 0] == pytest.approx(v0 - mu * g * t, rel=2e-3)
    assert sim.w[0, 1] == pytest.approx(2.5 * mu * g * t / r, rel=2e-3)
    sim.run(int(t_roll / 1e-6 * 1.0))
    assert sim.v[0, 0] == pytest.approx(5 / 7 * v0, rel=2e-3)
    assert sim.w[0, 1] == pytest.approx(sim.v[0, 0] / r, rel=2e-3)


def test_coulomb_truncation_is_exact_at_slip():
    # In slip the tangential force sits exactly on the Coulomb limit (Eq. 5)
    # and the stored overlap reproduces it through Eq. 4.
    r = 1e-3
    m = sphere_mass(r)
    P = oracle.make_params(E=E, nu=NU, e=0.7, mu=0.25, dt=1e-6, lo=(-0.01,) * 3, hi=(0.01,) * 3)
    x = [[0, 0, 0], [0, 0, 2 * r - 5e-6]]
    v = [[0.3, 0.0, 0.01], [-0.2, 0.1, -0.01]]
    w = [[10.0, -5.0, 3.0], [0.0, 7.0, 0.0]]
    sim = oracle.Sim(P, x, v, w, [r, r], [m, m], use_cells=False)
    sim.set_history([0], [1], [[2e-7, -1e-7, 0.0]])
    F, T, (a, b, xi, slip), _ = sim.evaluate(dt_hist=1e-6)
    assert slip.tolist() == [1]
    nvec = np.array([0.0, 0.0, -1.0])        # from particle 1 to particle 0
    fn = F[0] @ nvec
    ft = F[0] - fn * nvec
    assert np.linalg.norm(ft) == pytest.approx(0.25 * abs(fn), rel=1e-12)
    # torques: T = (-r n) x f_t on both bodies (equal radii: equal torques)
    assert np.allclose(T[0], np.cross(-r * nvec, ft), rtol=1e-12, atol=0)
    assert np.allclose(T[1], T[0], rtol=1e-12, atol=0)
    c = oracle.pair_coeffs(P, r, r, m, m, 5e-6)
    vr = np.array(v[0]) - np.array(v[1])
    vc = vr - np.cross(r * np.array(w[0]) + r * np.array(w[1]), nvec)
    vt = vc - (vc @ nvec) * nvec
    assert np.allclose(-c["kt"] * xi[0] - c["gt"] * vt, ft, rtol=1e-10, atol=1e-15)
    assert abs(xi[0] @ nvec) < 1e-20


def test_history_rotation_keeps_the_length_of_the_stored_overlap():
    # Eq. 4 with the overlap carried while the contact normal turns: the stored xi, tangent to
    # the old normal n0, is brought into the plane of the new normal n at its previous length
    # (reading of Sec. 2.1; the paper does not say how a stored overlap follows the normal).
    # The start-up evaluation (dt_hist = 0) isolates that step: no advance by v_t dt, and with
    # both bodies at rest f_t = -k_t xi exactly.  Dropping the rescale shortens xi by
    # |xi0 - (xi0.n) n| / |xi0| = cos(theta) < 1; dropping the projection leaves xi.n != 0.
    r = 1e-3
    m = sphere_mass(r)
    P = oracle.make_params(E=E, nu=NU, e=0.8, mu=0.9, dt=1e-6, lo=(-0.01,) * 3, hi=(0.01,) * 3)
    delta = 6e-6
    for theta in (0.05, 0.3, 0.9):
        n = np.array([math.sin(theta), 0.0, math.cos(theta)])     # from particle 1 to particle 0
        x = np.array([[0.0, 0.0, 0.0], -(2 * r - delta) * n])
        xi0 = np.array([3e-7, 1.2e-7, 0.0])                        # tangent to n0 = +z
        sim = oracle.Sim(P, x, np.zeros((2, 3)), np.zeros((2, 3)), [r, r], [m, m], use_cells=False)
        sim.set_history([0], [1], [xi0])
        F, T, (a, b, xi, slip), _ = sim.evaluate(dt_hist=0.0)
        assert slip.tolist() == [0]
        x1 = xi[0]
        assert np.linalg.norm(x1) == pytest.approx(np.linalg.norm(xi0), rel=1e-14)
        assert abs(x1 @ n) <= 1e-15 * np.linalg.norm(xi0)
        proj = xi0 - (xi0 @ n) * n
        assert np.allclose(x1, proj * np.linalg.norm(xi0) / np.linalg.norm(proj), rtol=1e-14, atol=0)
        # the force: Hertz along n plus -k_t xi (no dashpots at rest)
        c = oracle.pair_coeffs(P, r, r, m, m, delta)
        assert np.allclose(F[0], c["kn"] * delta * n - c["kt"] * x1, rtol=1e-12, atol=1e-18)
        assert np.array_equal(F[1], -F[0])


def test_resume_from_a_checkpoint_is_bit_exact():
    # The oracle's state is (x, v, w), the forces of the last evaluation and the contact
    # history: a run stopped after k steps, copied out and continued in a new simulation
    # gives the same bits as the uninterrupted run (Sec. 8(c) O11 check on a sheared,
    # rotating dense block with floor contacts, slips and contacts that open and close).
    L = 5 * 2.0e-3
    x, v, w, r = _dense_overlapping(5, 2.0e-3, 1.03e-3, seed=4, vel=0.2, omega=50.0)
    P = oracle.make_params(E=E, nu=NU, e=0.6, mu=0.3, dt=2e-6, g=(0, 0, -9.81), hi=(L, L, L),
                           periodic=(True, True, False), floor=True, floor_v=(0.5, 0, 0))
    m = sphere_mass(r)
    full = oracle.Sim(P, x, v, w, r, m).run(120)
    part = oracle.Sim(P, x, v, w, r, m).run(45)
    ck = part.checkpoint()
    assert len(ck["ha"]) > len(r)
    resumed = oracle.Sim.restore(P, ck).run(75)
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(getattr(resumed, k), getattr(full, k)), k
    for u, t in zip(resumed.history(), full.history()):
        assert np.array_equal(u, t)
    # and the checkpoint is a copy: running on does not change it
    part.run(5)
    assert not np.array_equal(part.x, ck["x"])


def test_results_do_not_depend_on_storage_order():
    L = 5 * 2.0e-3
    x, v, w, r = _dense_overlapping(5, 2.0e-3, 1.03e-3, seed=8)
    P = oracle.make_params(E=E, nu=NU, e=0.6, mu=0.4, dt=2e-6, g=(0, 0, -9.81), hi=(L, L, L),
                           periodic=(True, True, False), floor=True, floor_v=(0.5, 0, 0))
    m = sphere_mass(r)
    a = oracle.Sim(P, x, v, w, r, m).run(50)
    perm = np.random.default_rng(0).permutation(len(r))
    b = oracle.Sim(P, x[perm], v[perm], w[perm], r[perm], m[perm], ids=perm).run(50)
    assert np.allclose(b.x, a.x[perm], rtol=0, atol=1e-15)
    assert np.allclose(b.v, a.v[perm], rtol=1e-9, atol=1e-12)
    ha, hb, hxa, _ = a.history()
    hb_, hbb, hxb, _ = b.history()
    assert np.array_equal(ha, hb_) and np.array_equal(hb, hbb)
    assert np.allclose(hxa, hxb, rtol=1e-8, atol=1e-18)



# ------------------------------------------------------ output grid fields

def test_grid_fields_definition():
    # one sphere: its volume over the cell volume, its mass and velocity, in the cell holding its
    # centre; two spheres in one cell: Favre velocity = momentum over mass; sums conserve mass
    x = np.array([[0.0105, 0.0023, 0.0047], [0.0101, 0.0021, 0.0049], [0.03, 0.001, 0.001]])
    v = np.array([[1.0, 0.0, -2.0], [3.0, 0.5, 0.0], [9.0, 9.0, 9.0]])
    r = np.array([1e-3, 2e-3, 1e-3])
    m = np.array([2.0, 6.0, 1.0])
    f = oracle.grid_fields(x, v, r, m, (0.0, 0.0, 0.0), 0.005, (4, 2, 2))
    c = f[0, 0, 2]
    assert c[0] == pytest.approx(4.0 / 3.0 * math.pi * (1e-9 + 8e-9) / 0.005 ** 3, rel=1e-14)
    assert c[1] == 8.0
    assert np.allclose(c[2:5], (2.0 * v[0] + 6.0 * v[1]) / 8.0, rtol=1e-15)
    assert f[..., 1].sum() == 8.0                       # the third sphere lies outside the grid
    assert np.count_nonzero(f[..., 1]) == 1


# ------------------------------------------------------- axisymmetric walls

def _wall_params(points, floor=False, g=(0.0, 0.0, 0.0), mu_wall=0.3):
    return oracle.make_params(E=1e7, nu=0.25, e=0.6, mu=0.4, mu_wall=mu_wall, dt=1e-6, g=g, lo=(-0.2, -0.2, -0.1),
                              hi=(0.2, 0.2, 0.5), periodic=(False, False, False), floor=floor,
                              walls=None if points is None else dict(axis=(0.01, -0.02), points=points))


def _one(P, x, v=(0, 0, 0), w=(0, 0, 0), r=1e-3):
    m = 2500.0 * 4.0 / 3.0 * math.pi * r ** 3
    s = oracle.Sim(P, np.array([x], dtype=float), np.array([v], dtype=float), np.array([w], dtype=float),
                   np.array([r]), np.array([m]))
    return s, m


def test_wall_contacts_of_a_cylinder_a_cone_and_its_rim():
    r, d0 = 1e-3, 3e-6
    pts = [(0.02, 0.0), (0.135, 0.2), (0.135, 0.4)]
    P = _wall_params(pts)
    kn = lambda delta: oracle.pair_coeffs(P, r, 0.0, 2500.0 * 4 / 3 * math.pi * r ** 3, 0.0, delta, wall=True)["kn"]
    ax = np.array([0.01, -0.02, 0.0])
    # cylinder: centre at radius 0.135 - r + d0 in direction e (unit, in the x-y plane), z = 0.3
    e = np.array([0.6, 0.8, 0.0])
    s, _ = _one(P, ax + (0.135 - r + d0) * e + np.array([0, 0, 0.3]))
    F, T, hist, _ = s.evaluate()
    assert np.allclose(F[0], -kn(d0) * d0 * e, rtol=1e-9, atol=1e-18)       # (delta from a difference of radii)
    assert np.abs(T).max() == 0.0 and list(hist[1]) == [-3]          # segment 1
    # cone (segment 0) at mid height: inward normal (-dz, dr) / |.| in the (rho, z) half-plane
    dr, dz = 0.115, 0.2
    L = math.hypot(dr, dz)
    nr, nz = -dz / L, dr / L
    rho, z = 0.02 + 0.5 * dr + (r - d0) * nr, 0.1 + (r - d0) * nz
    s, _ = _one(P, ax + rho * e + np.array([0, 0, z]))
    F, T, hist, _ = s.evaluate()
    assert np.allclose(F[0], kn(d0) * d0 * np.array([nr * e[0], nr * e[1], nz]), rtol=1e-9, atol=1e-18)
    assert list(hist[1]) == [-2]
    # the free rim at the orifice: a centre below it, the normal from the rim point to the centre
    u = np.array([0.3, -0.95393920141694566])           # unit, pointing down and inward in (rho, z)
    rho, z = 0.02 + (r - d0) * u[0], (r - d0) * u[1]
    s, _ = _one(P, ax + rho * e + np.array([0, 0, z]))
    F, T, hist, _ = s.evaluate()
    assert np.allclose(F[0], kn(d0) * d0 * np.array([u[0] * e[0], u[0] * e[1], u[1]]), rtol=1e-9, atol=1e-18)


def test_a_flat_wall_profile_acts_as_the_floor():
    # a horizontal profile segment under the sphere is the floor plane: the same trajectory for a
    # sphere that lands, slides and spins (normal, tangential history, friction and torque)
    x, v, w = (0.05, 0.03, 0.99e-3), (0.2, 0.05, -0.1), (30.0, -50.0, 10.0)
    a, _ = _one(_wall_params(None, floor=True, g=(0, 0, -9.81)), x, v, w)
    b, _ = _one(_wall_params([(0.0, 0.0), (0.3, 0.0)], g=(0, 0, -9.81)), x, v, w)
    a.run(3000)
    b.run(3000)
    assert np.allclose(a.x, b.x, rtol=0, atol=1e-15)
    assert np.allclose(a.v, b.v, rtol=1e-12, atol=1e-15)
    assert np.allclose(a.w, b.w, rtol=1e-12, atol=1e-12)


def test_openmp_build_gives_the_same_bits():
    # the all-cores build of the oracle (the timed CPU baseline) runs the per-pair contact law
    # in parallel and sums serially: the same bits as the serial build
    L = 6 * 2.0e-3
    x, v, w, r = _dense_overlapping(6, 2.0e-3, 1.03e-3, seed=21, vel=0.2, omega=40.0)
    P = oracle.make_params(E=E, nu=NU, e=0.7, mu=0.3, dt=2e-6, g=(0, 0, -9.81), hi=(L, L, L),
                           periodic=(True, True, False), floor=True, floor_v=(0.5, 0, 0))
    m = sphere_mass(r)
    a = oracle.Sim(P, x, v, w, r, m).run(60)
    b = oracle.Sim(P, x, v, w, r, m, openmp=True).run(60)
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    for u, t in zip(a.history(), b.history()):
        assert np.array_equal(u, t)


def test_held_external_force_acts_like_gravity():
    # the coupling controllers' force is held on a particle and added to its other forces: a held
    # m g without gravity moves a block exactly as gravity g does (the same sums, in another order)
    L = 5 * 2.0e-3
    x, v, w, r = _dense_overlapping(5, 2.0e-3, 1.03e-3, seed=6)
    m = sphere_mass(r)
    g = np.array([0.0, 0.0, -9.81])
    kw = dict(E=E, nu=NU, e=0.6, mu=0.3, dt=2e-6, hi=(L, L, L), periodic=(True, True, False), floor=True)
    a = oracle.Sim(oracle.make_params(g=tuple(g), **kw), x, v, w, r, m).run(50)
    b = oracle.Sim(oracle.make_params(**kw), x, v, w, r, m)
    b.fext = m[:, None] * g[None, :]
    b.run(50)
    assert np.allclose(b.x, a.x, rtol=0, atol=1e-15)
    assert np.allclose(b.v, a.v, rtol=1e-10, atol=1e-13)
    assert not np.allclose(oracle.Sim(oracle.make_params(**kw), x, v, w, r, m).run(50).x, a.x, rtol=0, atol=1e-12)
