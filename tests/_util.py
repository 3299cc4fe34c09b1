"""Helpers shared by the tests (no method arithmetic)."""
import numpy as np

import oracle


def oracle_params(wl, walls=None, axis=(0.0, 0.0)):
    """walls: None, or the polyline (rho, z) of axisymmetric walls about the vertical axis through `axis`."""
    m = wl.material
    return oracle.make_params(E=m.E, nu=m.nu, e=m.e, mu=m.mu, mu_wall=m.mu_wall, dt=wl.dt, g=wl.g, lo=wl.lo,
                              hi=wl.hi, periodic=wl.periodic, floor=wl.floor, floor_v=wl.floor_v,
                              walls=None if walls is None else dict(axis=axis, points=walls))


def oracle_sim(wl, walls=None, **kw):
    return oracle.Sim(oracle_params(wl, walls), wl.x, wl.v, wl.w, wl.r, wl.m, **kw)


def gpu_pairs(partner):
    """Set of (i, j), i < j, from per-particle partner rows (-1 padded)."""
    out = set()
    for i, row in enumerate(partner):
        for p in row:
            if p < 0:
                break
            if p > i:
                out.add((i, int(p)))
    return out


def oracle_pairs(hist):
    a, b = hist[0], hist[1]
    keep = b >= 0
    return set(zip(a[keep].tolist(), b[keep].tolist()))


def min_image(d, wl):
    d = d.copy()
    for a in range(3):
        if wl.periodic[a]:
            L = wl.hi[a] - wl.lo[a]
            d[..., a] -= L * np.round(d[..., a] / L)
    return d
