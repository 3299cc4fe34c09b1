"""The silo inputs (Sec. 3) as stated, checked with the oracle on the CPU: particle counts and
sizes of Table 1 and Sec. 3, and a start with no contact at all (no sphere touches another or
a wall), so that the settling begins from rest rather than from overlaps."""
import numpy as np
import pytest

import oracle
from paper_1705_03850_gb300 import workloads
from _util import oracle_params


def _no_contacts(wl, walls):
    P = oracle_params(wl, walls)
    assert len(oracle.pairs(P, wl.x, wl.r, 0.0)) == 0
    _, _, hist, _ = oracle.Sim(P, wl.x, np.zeros_like(wl.v), wl.w, wl.r, wl.m).evaluate()
    assert len(hist[0]) == 0


@pytest.mark.parametrize("alpha,n,d", [(1, 187_504, 2.8e-3), (2, 23_438, 5.6e-3)])
def test_silo_counts_sizes_and_a_contact_free_start(alpha, n, d):
    wl = workloads.silo(alpha)
    assert wl.n == n
    assert np.allclose(2 * wl.r, d, rtol=1e-6)
    m = wl.material
    assert (m.E, m.nu, m.e, m.mu, m.mu_wall, m.rho) == (2.5e7, 0.25, 0.5, 0.2, 0.175, 1000.0)
    assert wl.dt == pytest.approx(1e-6, rel=1e-7)
    _no_contacts(wl, workloads.silo_walls(wl.meta["z_o"], closed=True))


def test_two_level_silo_fine_start():
    coarse, fine, spec = workloads.silo_two_level()
    assert coarse.n == 23_438
    assert 35_000 < fine.n < 50_000                     # Sec. 3: about 44,000 in the lower quarter
    z_o = coarse.meta["z_o"]
    assert np.all(fine.x[:, 2] >= spec["lo"][2]) and np.all(fine.x[:, 2] <= spec["hi"][2])
    _no_contacts(fine, workloads.silo_walls(z_o, closed=True))
    # 8 x 8 surface cells of 2 cm on the top face, a 2 cm transition layer
    w = spec["hi"][0] - spec["lo"][0]
    assert int(np.floor(w / spec["surface_cell"])) == 8


def test_small_vessel_lattice_start_is_contact_free():
    wl = workloads.small_vessel()
    _no_contacts(wl, wl.meta["walls"])
