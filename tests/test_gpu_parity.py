"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Bars (stated with each test): contact sets bit-exact; per-particle forces
within 1e-5 of sum_j |F_ij| + |m g| on identical input state; 100-step
positions within max(1e-4 d, 64 ulp_fp32(|x|)).
"""
import numpy as np
import pytest

import oracle
from paper_1705_03850_gb300 import dem, workloads
from _util import gpu_pairs, min_image, oracle_pairs, oracle_params, oracle_sim

pytestmark = pytest.mark.gpu

FORCE_REL = 1e-5


def _force_check(F, Fo, fabs, rel=FORCE_REL):
    err = np.abs(F - Fo).max(axis=1) / (fabs + 1e-30)
    assert err.max() <= rel, f"max rel force error {err.max():.3e} at {err.argmax()}"
    return err.max()


@pytest.mark.parametrize("shape,seed", [((12, 12, 10), 7), ((9, 7, 5), 8), ((20, 20, 3), 9)])
def test_contacts_and_forces_at_identical_state(shape, seed):
    # several tiles of 128 and a ragged last tile; random v and spin; floor sheared
    wl = workloads.dense_block(*shape, seed=seed)
    assert wl.n % 128 != 0
    sim = dem.from_workload(wl)
    F = sim.read(dem.FORCE)
    T = sim.read(dem.TORQUE)
    partner, xi = sim.read_contacts(width=24)
    Fo, To, hist, fabs = oracle_sim(wl).evaluate()
    assert gpu_pairs(partner) == oracle_pairs(hist)
    assert len(oracle_pairs(hist)) > 2 * wl.n
    _force_check(F, Fo, fabs)
    terr = np.abs(T - To).max(axis=1) / (fabs * wl.r + 1e-30)
    assert terr.max() <= FORCE_REL
    # floor contacts: same particles
    wxi = sim.read(dem.WALL_XI)
    on_floor = set(hist[0][hist[1] < 0].tolist())
    assert on_floor  # the block rests on the sheared floor
    # tangential overlaps after the start-up evaluation (non-zero only where the contact slips)
    o = {(int(a), int(b)): x for a, b, x in zip(hist[0], hist[1], hist[2])}
    scale = max(np.abs(hist[2]).max(), 1e-30)
    for i, row in enumerate(partner):
        for t, p in enumerate(row):
            if p < 0:
                break
            key = (min(i, p), max(i, p))
            assert np.abs(xi[i, t] - o[key]).max() <= 1e-4 * np.abs(o[key]).max() + 1e-5 * scale
    for i in on_floor:
        assert np.abs(wxi[i] - o[(i, -1)]).max() <= 1e-4 * np.abs(o[(i, -1)]).max() + 1e-5 * scale


def test_forces_with_imported_history():
    # tangential overlaps given as input (same on both sides), then one evaluation
    wl = workloads.dense_block(10, 10, 6, seed=11)
    pairs = oracle.pairs(oracle_sim(wl).P, wl.x, wl.r, 0.0)
    rng = np.random.default_rng(5)
    hx = rng.normal(0.0, 2e-6, (len(pairs), 3))
    hx = workloads.f32(hx)
    width = 24
    partner = -np.ones((wl.n, width), dtype=np.int32)
    xi = np.zeros((wl.n, width, 3))
    rows = [[] for _ in range(wl.n)]
    for (i, j), h in zip(pairs, hx):
        rows[i].append((j, h))
        rows[j].append((i, h))
    for i, r in enumerate(rows):
        for t, (j, h) in enumerate(sorted(r, key=lambda z: z[0])):
            partner[i, t] = j
            xi[i, t] = h
    sim = dem.from_workload(wl)
    sim.write_contacts(partner, xi)
    F = sim.read(dem.FORCE)
    T = sim.read(dem.TORQUE)
    o = oracle_sim(wl)
    o.set_history(pairs[:, 0], pairs[:, 1], hx)
    Fo, To, hist, fabs = o.evaluate()
    e = _force_check(F, Fo, fabs)
    assert np.abs(T - To).max(axis=1).max() / 1 <= FORCE_REL * (fabs * wl.r).max()
    assert e < FORCE_REL


def test_neighbour_lists_hold_exactly_the_pairs_within_the_skin():
    wl = workloads.dense_block(11, 9, 7, seed=12, squeeze=-0.02)   # loose: gaps of up to the skin
    sim = dem.from_workload(wl)
    cnt = sim.read(dem.NBR_COUNT)
    pairs = oracle.pairs(oracle_sim(wl).P, wl.x, wl.r, wl.skin)
    ref = np.bincount(pairs.ravel(), minlength=wl.n)
    assert np.array_equal(cnt.astype(np.int64), ref)


def _ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("steps", [100])
def test_rollout_positions(steps):
    wl = workloads.dense_block(12, 12, 8, seed=13)
    sim = dem.from_workload(wl)
    sim.step(steps).sync()
    x = sim.read(dem.POS)
    o = oracle_sim(wl).run(steps)
    d = min_image(x - o.x, wl)
    tol = np.maximum(1e-4 * 2 * wl.r[:, None], 64 * _ulp32(o.x))
    assert (np.abs(d) <= tol).all(), np.abs(d).max()
    # the contact network evolved identically
    partner, gxi = sim.read_contacts(width=24)
    # both particles of a pair hold exactly opposite overlaps (reported in the
    # lower ID's frame, the two copies are bit-identical)
    pos_of = {(i, int(p)): t for i, row in enumerate(partner) for t, p in enumerate(row) if p >= 0}
    nsym = 0
    for (i, p), t in pos_of.items():
        if i < p:
            assert np.array_equal(gxi[i, t], gxi[p, pos_of[(p, i)]]), (i, p)
            nsym += 1
    assert nsym > wl.n
    # contact sets: equal on every pair whose overlap (at the oracle's positions) is larger
    # than the band the position differences allow (twice the largest difference plus the
    # float32 resolution of the radii and coordinates); band pairs are counted, not failed
    ha, hb, _, _ = o.history()
    g, r = gpu_pairs(partner), oracle_pairs((ha, hb))
    band = 2 * np.abs(d).max() + 8 * _ulp32(2 * wl.r.max()) + 8 * _ulp32(np.abs(o.x).max())
    inband = 0
    for i, j in g ^ r:
        dd = min_image(o.x[i] - o.x[j], wl)
        delta = o.r[i] + o.r[j] - np.linalg.norm(dd)
        assert abs(delta) < band, (i, j, delta, band)
        inband += 1
    assert inband <= 0.01 * len(r)


@pytest.mark.parametrize("mode", [1, 2])
def test_graph_capture_matches_direct_launches_bitwise(mode):
    # graphs of one step kernel per step (mode 1) and of fused steps (mode 2: one cooperative
    # launch between list builds, a grid barrier between steps) against direct launches
    wl = workloads.dense_block(10, 10, 6, seed=14, vel=0.5)
    a = dem.from_workload(wl)
    b = dem.from_workload(wl)
    a.step(1)
    b.step(1)
    b.set_graph_mode(mode)
    b.set_graph(25)
    assert b.stats()["graph_fused"] == (mode == 2)
    a.step(300).sync()
    b.step(300).sync()
    assert a.stats()["rebuilds"] > 2
    assert np.array_equal(a.read(dem.POS), b.read(dem.POS))
    assert np.array_equal(a.read(dem.VEL), b.read(dem.VEL))


def test_staged_list_build_gives_the_same_lists():
    # the list build with the cell-ordered positions staged in shared memory (per block) builds
    # the same rows as the direct scan: the same bits over many rebuilds, one and several instances
    wl = workloads.dense_block(10, 10, 6, seed=14, vel=0.5)
    wls = [workloads.dense_block(*sh, seed=40 + k, vel=0.4) for k, sh in enumerate([(5, 6, 4), (9, 7, 5), (4, 4, 3)])]

    def batched():
        sim = dem.DEM([dem.desc_from_workload(b) for b in wls])
        sim.write_state(*(np.concatenate([getattr(b, f) for b in wls]) for f in ("x", "v", "w", "r", "m")))
        return sim
    for make in (lambda: dem.from_workload(wl), batched):
        runs = []
        for staged in (0, 1):
            sim = make()
            sim.set_list_build(staged)
            sim.step(1)
            sim.set_graph(25)
            sim.step(300).sync()
            runs.append((sim.read(dem.POS), sim.read(dem.OMEGA), sim.stats()["rebuilds"]))
        assert runs[0][2] == runs[1][2] > 2
        assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_results_do_not_depend_on_cell_size_or_list_width():
    wl = workloads.dense_block(10, 8, 6, seed=15, vel=0.3)
    a = dem.from_workload(wl)
    d = dem.desc_from_workload(wl, r_max=2.0 * float(wl.r.max()))
    b = dem.DEM([d], max_neighbors=24)
    b.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    a.step(120).sync()
    b.step(120).sync()
    assert np.array_equal(a.read(dem.POS), b.read(dem.POS))
    assert np.array_equal(a.read(dem.OMEGA), b.read(dem.OMEGA))


def test_two_instances_in_one_context_equal_each_alone():
    w1 = workloads.dense_block(8, 8, 5, seed=16)
    w2 = workloads.dense_block(7, 9, 4, seed=17, mat=workloads.Material(E=3e7, nu=0.3, e=0.5, mu=0.2, rho=1000))
    both = dem.DEM([dem.desc_from_workload(w1), dem.desc_from_workload(w2)])
    cat = lambda f: np.concatenate([getattr(w1, f), getattr(w2, f)])
    both.write_state(cat("x"), cat("v"), cat("w"), cat("r"), cat("m"))
    both.step(80).sync()
    x = both.read(dem.POS)
    for wl, sl in ((w1, slice(0, w1.n)), (w2, slice(w1.n, None))):
        one = dem.from_workload(wl)
        one.step(80).sync()
        assert np.array_equal(one.read(dem.POS), x[sl])


def test_single_sphere_on_the_floor_matches_oracle():
    wl = workloads.single_sphere()
    sim = dem.from_workload(wl)
    sim.step(400).sync()
    o = oracle_sim(wl).run(400)
    assert np.abs(sim.read(dem.POS) - o.x).max() <= 2e-7
    assert np.abs(sim.read(dem.VEL) - o.v).max() <= 1e-4 * np.abs(o.v).max() + 1e-6


def test_empty_instance_is_fine():
    wl = workloads.dense_block(4, 4, 2, seed=19)
    d0 = dem.desc_from_workload(wl)
    d0.n = 0
    d0.capacity = 64
    sim = dem.DEM([d0, dem.desc_from_workload(wl)])
    sim.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    sim.step(10).sync()
    assert sim.read(dem.POS).shape == (wl.n, 3)


def test_list_overflow_is_reported_not_hung():
    wl = workloads.dense_block(6, 6, 4, seed=20)
    sim = dem.DEM([dem.desc_from_workload(wl)], max_neighbors=3)
    sim.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    sim.step(2)
    assert sim.status() == 2  # DEM_ERR_CAPACITY


def test_nonfinite_input_is_reported():
    wl = workloads.dense_block(6, 6, 4, seed=21)
    v = wl.v.copy()
    v[5, 0] = np.nan
    sim = dem.DEM([dem.desc_from_workload(wl)])
    sim.write_state(wl.x, v, wl.w, wl.r, wl.m)
    sim.step(2)
    assert sim.status() == 4  # DEM_ERR_NONFINITE


@pytest.mark.slow
def test_full_size_million_particle_forces():
    # 1,000,000 particles (100^3 overlapping block) in the bench's launch configuration
    wl = workloads.dense_block(100, 100, 100, seed=22)
    sim = dem.from_workload(wl)
    F = sim.read(dem.FORCE)
    Fo, To, hist, fabs = oracle_sim(wl).evaluate()
    _force_check(F, Fo, fabs)


def test_steady_drift_is_not_biased_by_the_position_grid():
    # free spheres (no gravity, contacts or floor) at constant velocities whose step is a
    # fractional number of position quanta: the positions follow x0 + v t within a random
    # walk of about a quantum times the square root of the step count, not the
    # half-quantum-per-step bias of plain rounding
    import dataclasses
    wl = workloads.single_sphere(z=5e-3, w=(0.0, 0.0, 0.0))
    q = oracle.quantum(wl.lo, wl.hi)
    n, steps = 64, 2000
    x = np.column_stack([np.full(n, 2e-3), np.linspace(0.5e-3, 9.5e-3, n), np.full(n, 5e-3)])
    v = np.zeros((n, 3))
    v[:, 0] = (33.0 + np.linspace(0.05, 0.95, n)) * q / wl.dt        # 33.05 .. 33.95 quanta per step
    v = workloads.f32(v)
    r = workloads.qgrid(np.full(n, 5e-5))                           # 0.1 mm spheres 0.14 mm apart
    m = workloads.sphere_masses(r, wl.material.rho)
    wl = dataclasses.replace(wl, x=workloads.qgrid(x), v=v, w=np.zeros((n, 3)), r=r, m=m, g=(0.0, 0.0, 0.0),
                             floor=False)
    sim = dem.DEM([dem.desc_from_workload(wl)])
    sim.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    sim.step(steps)
    d = min_image(sim.read(dem.POS) - (wl.x + wl.v * wl.dt * steps), wl)
    err = np.abs(d[:, 0]) / q
    assert err.max() < 6 * np.sqrt(steps * 0.25) + 2, err.max()        # plain rounding: up to 900 quanta
    assert np.abs(d[:, 1:]).max() == 0.0


def test_column_of_1000_spheres_over_5000_steps():
    # the FP64-oracle-size plain workload as stated (1,000 spheres on a jittered lattice in a
    # 20 x 20 x 60 mm box, dt = 2e-6 s, 5,000 steps): exact positions while the column falls,
    # then kinetic energy and mean height along the run within 2 % once contacts form
    wl = workloads.column()
    sim = dem.from_workload(wl)
    o = oracle_sim(wl)
    axis = np.array([[0.01, 0.01]])
    done = 0
    for k, upto in enumerate((500, 1000, 2000, 3000, 4000, 5000)):
        sim.step(upto - done)
        o.run(upto - done)
        done = upto
        x = sim.read(dem.POS)
        if k == 0:
            d = min_image(x - o.x, wl)
            tol = np.maximum(1e-4 * 2 * wl.r[:, None], 64 * _ulp32(o.x))
            assert (np.abs(d) <= tol).all(), np.abs(d).max()
        ke_gpu = sim.observables(axis)[0, 0]
        I = 0.4 * wl.m * wl.r ** 2
        ke_orc = 0.5 * np.sum(wl.m[:, None] * o.v ** 2) + 0.5 * np.sum(I[:, None] * o.w ** 2)
        assert ke_gpu == pytest.approx(ke_orc, rel=0.02), (upto, ke_gpu, ke_orc)
        assert x[:, 2].mean() == pytest.approx(o.x[:, 2].mean(), rel=0.02)
    st = sim.stats()
    assert st["contacts"] + st["wall_contacts"] > 0      # the bottom of the column reached the floor


def test_full_size_graph_steps_equal_direct_steps_and_keep_the_exact_contact_set():
    # 1,000,000 particles through the timed path (CUDA graphs of 50 steps with in-graph
    # rebuilds) against direct launches, bit for bit; after 100 steps the contact pairs
    # equal the oracle's pairs at the read-back positions (exact: positions are multiples
    # of the quantum) and both sides of every pair hold the same stored overlap
    wl = workloads.dense_block(100, 100, 100, seed=23, vel=0.2)
    a = dem.from_workload(wl)
    b = dem.from_workload(wl)
    a.step(1)
    b.step(1)
    a.set_graph(50)
    a.step(100)
    b.step(100)
    xa, xb = a.read(dem.POS), b.read(dem.POS)
    assert np.array_equal(xa, xb)
    assert np.array_equal(a.read(dem.VEL), b.read(dem.VEL))
    assert a.stats()["rebuilds"] >= 1
    partner, xi = a.read_contacts(width=24)
    ref = oracle.pairs(oracle_params(wl), xa, a.read(dem.RADIUS), 0.0, method="cells")
    got = gpu_pairs(partner)
    assert got == {(int(i), int(j)) for i, j in ref}
    for i in range(0, wl.n, 997):                   # a sample of rows (the check is per pair)
        for t, p in enumerate(partner[i]):
            if p < 0:
                break
            row = partner[p]
            u = int(np.nonzero(row == i)[0][0])
            assert np.array_equal(xi[i, t], xi[p, u])
