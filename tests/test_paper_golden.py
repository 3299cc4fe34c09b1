"""Pins against numbers the paper prints (tests/golden/paper_values.txt, each with its
citation): the coarse-grain scaling of the silo example (Sec. 2.2, Sec. 3), its material
(Table 1) run through the oracle, and the particle-count arithmetic of Sec. 3."""
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _gold():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, value = line.split()[:2]
        out[name] = float(value)
    return out


G = _gold()


def _silo_params():
    return oracle.make_params(E=G["silo_E"], nu=G["silo_nu"], e=G["silo_e"], mu=G["silo_mu_pp"],
                              dt=G["silo_dt"], g=(0, 0, 0), lo=(0, 0, 0), hi=(0.1, 0.1, 0.1),
                              periodic=(True, True, True), floor=False)


def test_coarse_grain_counts_and_sizes_of_the_silo():
    # a coarse grain of ratio alpha stands for alpha^3 original particles and is alpha times larger
    a = G["cg_alpha"]
    assert round(G["ref_particles"] / a ** 3) == G["cg_particles"]
    assert G["silo_d"] * a == pytest.approx(G["cg_d"], rel=1e-12)


def test_silo_material_contact_coefficients_scale_with_the_grain():
    # Sec. 2.2 with the Table 1 material: the same contact geometry scaled by alpha (radii and
    # overlap times alpha, masses times alpha^3) has stiffnesses times alpha and dampings times alpha^2
    P = _silo_params()
    a = G["cg_alpha"]
    r = G["silo_d"] / 2
    m = G["silo_rho"] * 4.0 / 3.0 * math.pi * r ** 3
    c1 = oracle.pair_coeffs(P, r, r, m, m, 1e-6)
    c2 = oracle.pair_coeffs(P, a * r, a * r, a ** 3 * m, a ** 3 * m, a * 1e-6)
    assert c2["kn"] == pytest.approx(a * c1["kn"], rel=1e-13)
    assert c2["kt"] == pytest.approx(a * c1["kt"], rel=1e-13)
    assert c2["gn"] == pytest.approx(a * a * c1["gn"], rel=1e-13)
    assert c2["gt"] == pytest.approx(a * a * c1["gt"], rel=1e-13)


def test_silo_material_head_on_impact_rebounds_at_the_model_restitution():
    # two Table 1 spheres (2.8 mm, 1000 kg/m^3, E = 2.5e7 Pa, e = 0.5) meet head-on; the oracle's
    # rebound speed ratio equals the restitution of the damped-Hertz model it integrates,
    # obtained here from the 1-D equation of the normal overlap (scipy, independent of the oracle)
    from scipy.integrate import solve_ivp
    P = _silo_params()
    r = G["silo_d"] / 2
    m = G["silo_rho"] * 4.0 / 3.0 * math.pi * r ** 3
    v0 = 0.5
    c = oracle.pair_coeffs(P, r, r, m, m, 1e-6)
    meff = m / 2
    # k_n = K sqrt(delta), gamma_n = Gm delta^(1/4) from the coefficients at delta = 1e-6
    K = c["kn"] / math.sqrt(1e-6)
    Gm = c["gn"] / 1e-6 ** 0.25

    def rhs(t, y):
        d, dd = y
        f = K * max(d, 0.0) ** 1.5 + Gm * max(d, 0.0) ** 0.25 * dd
        return [dd, -f / meff]

    end = lambda t, y: y[0]
    end.terminal, end.direction = True, -1
    sol = solve_ivp(rhs, (0.0, 1e-2), [0.0, 2 * v0], events=end, rtol=1e-10, atol=1e-16, max_step=1e-7,
                    first_step=1e-9)
    e_model = -sol.y_events[0][0][1] / (2 * v0)
    x = np.array([[0.05 - r - 1e-5, 0.05, 0.05], [0.05 + r + 1e-5, 0.05, 0.05]])
    v = np.array([[v0, 0, 0], [-v0, 0, 0]])
    sim = oracle.Sim(P, x, v, np.zeros((2, 3)), np.full(2, r), np.full(2, m))
    sim.run(int(2.5e-4 / G["silo_dt"]))
    e_sim = (sim.v[1, 0] - sim.v[0, 0]) / (2 * v0)
    assert 0.3 < e_model < 0.7
    assert e_sim == pytest.approx(e_model, abs=2e-3)


def test_particle_count_arithmetic_of_the_runtime_discussion():
    # the full system is the reference size reduced by 32: 32^3 times the particles
    assert G["ref_particles"] * G["proj_scale"] ** 3 == pytest.approx(G["proj_particles"], rel=1e-3)
    # five levels, alpha_l = 2^(l-1), volume quartered per level
    L = int(G["proj_levels"])
    total = sum(G["proj_particles"] * (2.0 ** (l - 1)) ** -3 * 4.0 ** (l - L) for l in range(1, L + 1))
    assert total == pytest.approx(G["proj_total"], rel=1e-3)
    # the two-level silo: reference particles over coarse plus fine ones
    ratio = G["ref_particles"] / (G["cg_particles"] + G["ml_fine_particles"])
    assert ratio == pytest.approx(G["ml_ratio"], abs=5e-3)
    # the two-level discharge rate deviates from the reference by the stated amount
    assert (G["rate_ref"] - G["rate_ml"]) / G["rate_ref"] == pytest.approx(G["rate_ml_dev"], rel=1e-9)


def test_silo_setup_follows_the_paper():
    # the silo workloads and runner use the printed geometry, material, measurement and
    # Table 2 rates (the values the runner reports beside its own)
    from paper_1705_03850_gb300 import silo, workloads
    m = workloads.SILO_MATERIAL
    assert (m.E, m.nu, m.e, m.mu, m.mu_wall, m.rho) == (G["silo_E"], G["silo_nu"], G["silo_e"], G["silo_mu_pp"],
                                                        G["silo_mu_pw"], G["silo_rho"])
    z_o = 0.05
    pts = workloads.silo_walls(z_o, closed=False)
    assert pts[0][0] == pytest.approx(G["silo_orifice_diam"] / 2, abs=1e-7)
    assert pts[-1][0] == pytest.approx(G["silo_cyl_diam"] / 2, abs=1e-7)
    assert pts[-1][1] - pts[0][1] == pytest.approx(G["silo_height"], abs=1e-7)
    assert pts[1][1] - pts[0][1] == pytest.approx(G["silo_height"] / 2, abs=1e-7)   # the lower half is the cone
    assert silo.PAPER_RATE == {1: (G["rate_ref"], G["rate_ref_std"]), 2: (G["rate_cg"], G["rate_cg_std"])}
    assert silo.PAPER_RATE_TWO_LEVEL == {"fine": (G["rate_ml"], G["rate_ml_std"]),
                                         "coarse": (G["rate_ml_cg"], G["rate_ml_cg_std"])}
    import inspect
    sig = inspect.signature(silo.run)
    assert sig.parameters["sample_s"].default == pytest.approx(1.0 / G["rate_sampling_hz"])
    assert silo.PLANE_BELOW == G["rate_plane_below"]
    coarse, fine, spec = workloads.silo_two_level()
    assert spec["interval"] == G["controller_steps"]
    w = (spec["hi"][0] - spec["lo"][0]) / int(np.floor((spec["hi"][0] - spec["lo"][0]) / spec["surface_cell"]))
    assert w == pytest.approx(G["grid_cell"], rel=1e-6)
