"""The allocation-free neighbour counter against a context's neighbour-list lengths.

dem_neighbor_counts_noalloc serves callers that cannot hand the library device
memory (a host framework that owns every device byte through its own pool, or
a loop that must not allocate after start-up): its scratch is a fixed device
array inside the library.  Its counts must equal, exactly, the list lengths
that a context built from the same particles reports (DEM_F_NBR_COUNT); two
different inputs in a row check that each call starts from a clean scratch.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1705_03850_gb300 import dem, workloads

pytestmark = pytest.mark.gpu


def _context_counts(wl):
    sim = dem.from_workload(wl)
    c = sim.read(dem.NBR_COUNT).astype(np.int64)
    sim.close()
    return c


def _noalloc_counts(wl):
    import torch
    x = torch.as_tensor(wl.x, dtype=torch.float64, device="cuda")
    r = torch.as_tensor(wl.r, dtype=torch.float64, device="cuda")
    out = dem.neighbor_counts_noalloc(x, r, wl.lo, wl.hi, wl.periodic, wl.skin, float(wl.r.max()))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64)


def test_noalloc_counts_equal_context_list_lengths_on_two_calls_in_a_row():
    first = workloads.dense_block(24, 20, 12, seed=31, squeeze=-0.01)           # 5,760 particles
    second = workloads.dense_block(9, 11, 5, seed=32, squeeze=0.003, rjit=0.1)  # 495 particles, other box
    for wl in (first, second):
        ref = _context_counts(wl)
        got = _noalloc_counts(wl)
        assert ref.sum() > wl.n
        assert np.array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_fixed_maximum():
    import torch
    n = (1 << 18) + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    r = torch.full((n,), 1e-3, dtype=torch.float64, device="cuda")
    with pytest.raises(dem.DemError) as e:
        dem.neighbor_counts_noalloc(x, r, (0, 0, 0), (1, 1, 1), (True, True, False), 1e-4, 1e-3)
    assert e.value.code == 2 and "262144" in str(e.value)
