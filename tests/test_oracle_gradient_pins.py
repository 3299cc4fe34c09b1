"""Pins of the oracle's complex-step derivatives (the FP64 reference gradient).

Each compares d(state)/d(E, e, mu) from the complex step with something else:
closed forms of the sliding sphere, the derivative of the 1-D restitution ODE
(scipy) with respect to e, the scale invariance of the Hertz restitution in E,
and FP64 central differences of the oracle's real rollout.
"""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import RHO, E, NU, sphere_mass, _dense_overlapping, _e_model


def test_sliding_sphere_mu_derivative_closed_form():
    # while sliding: v = v0 - mu g t, omega_y = 5 mu g t / (2 r)
    # => dv/dmu = -g t, domega_y/dmu = 5 g t / (2 r)
    r, v0, mu, g = 1e-3, 0.2, 0.3, 9.81
    m = sphere_mass(r)
    P = oracle.make_params(E=E, nu=NU, e=0.5, mu=mu, dt=1e-6, g=(0, 0, -g), lo=(-1, -1, 0), hi=(1, 1, 1),
                           floor=True)
    Eeff = E / (2 * (1 - NU ** 2))
    d0 = (3 * m * g / (4 * Eeff * math.sqrt(r))) ** (2 / 3)
    steps = 8000
    out = oracle.rollout_derivative(P, [[0, 0, r - d0]], [[v0, 0, 0]], [[0, 0, 0]], [r], [m], steps, "mu",
                                    use_cells=False)
    t = steps * 1e-6
    assert out["dv"][0, 0] == pytest.approx(-g * t, rel=3e-3)
    assert out["dw"][0, 1] == pytest.approx(2.5 * g * t / r, rel=3e-3)
    # E does not enter the Coulomb-limited sliding law
    outE = oracle.rollout_derivative(P, [[0, 0, r - d0]], [[v0, 0, 0]], [[0, 0, 0]], [r], [m], steps, "E",
                                     use_cells=False)
    assert abs(outE["dv"][0, 0] * E) < 1e-3 * v0


def _collide(e, param, v0=0.5, r=1e-3, dt=1e-6, steps=600):
    P = oracle.make_params(E=E, nu=NU, e=e, mu=0.5, dt=dt, lo=(-0.01,) * 3, hi=(0.01,) * 3)
    x = np.array([[-r - 2e-7, 0, 0], [r + 2e-7, 0, 0]])
    v = np.array([[0.5 * v0, 0, 0], [-0.5 * v0, 0, 0]])
    m = np.full(2, sphere_mass(r))
    # long enough for the whole contact (t_c ~ 2.4e-4 s) and separation
    return oracle.rollout_derivative(P, x, v, np.zeros((2, 3)), np.full(2, r), m, steps, param, use_cells=False)


@pytest.mark.slow
def test_restitution_derivative_approaches_the_1d_ode():
    # After the collision the relative speed is e_model(e) v0, and the scipy ODE
    # gives its slope with respect to e.  The complex step is the derivative of
    # the discrete map with the number of contact steps held fixed, which
    # misses the shift of the exit time; so it approaches the ODE slope as dt
    # shrinks (2.2 % at dt = 1e-6, 1.7 % at 2e-7) while matching the
    # discrete map's own central difference to 1e-6.
    e, v0 = 0.7, 0.5
    de = 1e-4
    slope = v0 * (_e_model(e + de) - _e_model(e - de)) / (2 * de)
    errs = []
    for dt in (1e-6, 2e-7):
        out = _collide(e, "e", dt=dt, steps=int(round(6e-4 / dt)))
        dvrel = out["dv"][1, 0] - out["dv"][0, 0]
        plus = _collide(e + 1e-5, "e", dt=dt, steps=int(round(6e-4 / dt)))
        minus = _collide(e - 1e-5, "e", dt=dt, steps=int(round(6e-4 / dt)))
        vrel = lambda o: o["v"][1, 0] - o["v"][0, 0]
        fd = (vrel(plus) - vrel(minus)) / 2e-5
        assert dvrel == pytest.approx(fd, rel=1e-6)
        errs.append(abs(dvrel - slope) / slope)
    assert errs[0] < 0.03
    assert errs[1] < errs[0]


def test_restitution_does_not_depend_on_stiffness():
    # The damped Hertz law is scale free: the rebound speed does not depend on
    # E.  With the contact pattern held fixed the discrete derivative misses
    # the shift of the exit time (t_c ~ E^-2/5), so it vanishes only as dt -> 0:
    # E dv/dE / v0 = -0.051, -0.036, -0.015 at dt = 1e-6, 2e-7, 5e-8.
    vals = []
    for dt in (1e-6, 2e-7, 5e-8):
        out = _collide(0.7, "E", dt=dt, steps=int(round(6e-4 / dt)))
        vals.append(abs((out["dv"][1, 0] - out["dv"][0, 0]) * E / 0.5))
    assert vals[0] < 0.06 and vals[2] < vals[1] < vals[0]


@pytest.mark.parametrize("param", ["E", "e", "mu"])
def test_complex_step_matches_central_differences(param):
    L = 4 * 2.0e-3
    x, v, w, r = _dense_overlapping(4, 2.0e-3, 1.01e-3, seed=9, vel=0.05, omega=20.0)
    P = oracle.make_params(E=2e7, nu=NU, e=0.6, mu=0.4, dt=2e-6, g=(0, 0, -9.81), hi=(L, L, 3 * L),
                           periodic=(True, True, False), floor=True, floor_v=(0.3, 0, 0))
    m = sphere_mass(r)
    steps = 60
    cs = oracle.rollout_derivative(P, x, v, w, r, m, steps, param)
    idx = oracle.PARAM_INDEX[param]
    slot = [0, 2, 3][idx]
    h = 1e-6 * P[slot]

    def run(delta):
        Q = P.copy()
        Q[slot] += delta
        if param == "mu":
            Q[4] += delta   # the floor friction follows mu
        s = oracle.Sim(Q, x, v, w, r, m).run(steps)
        return s.x.copy(), s.v.copy()

    (xp, vp), (xm, vm) = run(h), run(-h)
    fd_v = (vp - vm) / (2 * h)
    fd_x = (xp - xm) / (2 * h)
    scale_v = np.abs(cs["dv"]).max()
    assert scale_v > 0
    assert np.abs(cs["dv"] - fd_v).max() <= 1e-5 * scale_v
    assert np.abs(cs["dx"] - fd_x).max() <= 1e-5 * np.abs(cs["dx"]).max()
