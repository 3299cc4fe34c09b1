"""Seeded synthetic inputs for the DEM workloads.

This module only places particles and draws random numbers: lattices,
jitter, size draws, boxes and material constants.  It holds none of the
method's arithmetic, and both the CUDA path and the FP64 oracle take their
inputs from it (neither imports the other).

Every input is exactly representable on both sides: positions, radii and
box bounds are multiples of GRID = 2**-26 m (about 15 nm), and velocities,
masses, gravity and the time step are rounded to float32 values.  Masses are
those of solid spheres of the stated density.

Workloads (sizes and materials as stated for each configuration):

* ``column``  -- 1,000 spheres d = 2 mm in a 20 x 20 x 60 mm box, periodic in
  x/y, floor at z = 0, E = 1e7 Pa, nu = 0.25, e = 0.9, mu = 0.5,
  rho = 2500 kg/m^3, dt = 2e-6 s.  The box cannot hold a 10 x 10 lattice of
  2 mm spheres without contact, so the start is an 8 x 8 lattice at 2.5 mm
  spacing, layers 2.5 mm apart from z = 1.25 mm, first 1,000 sites, each
  jittered uniformly by +-0.2 mm per axis.
* ``shear_bed`` -- N polydisperse spheres d ~ U[1.6, 2.4] mm (N = 1,000,000 at
  full size) in a 0.2 x 0.2 m footprint (box height 0.6 m), periodic x/y,
  floor; start on an FCC lattice whose nearest-neighbour distance exceeds
  d_max, to be settled under gravity before the floor is sheared at 0.5 m/s.
* ``dense_block`` -- jittered lattice at spacing slightly below 2 r with
  random velocities and spins, so that most neighbours overlap by 0.01-1 %
  of r: the input for single-evaluation force parity.
* ``batch`` -- 256 settling boxes, N_k log-uniform in [2e3, 2e5], d = 2 mm,
  e ~ U[0.5, 0.95], mu ~ U[0.2, 0.8], E log-uniform in [5e6, 5e7] Pa.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GRID = 2.0 ** -26


def qgrid(a):
    """Round lengths to multiples of GRID (exact in float64, float32 and the device's fixed point)."""
    return np.round(np.asarray(a, dtype=np.float64) / GRID) * GRID


def f32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Material:
    E: float = 1.0e7
    nu: float = 0.25
    e: float = 0.9
    mu: float = 0.5
    mu_wall: float | None = None
    rho: float = 2500.0


@dataclass
class Workload:
    name: str
    x: np.ndarray                      # (n, 3) positions [m]
    v: np.ndarray                      # (n, 3) velocities [m/s]
    w: np.ndarray                      # (n, 3) angular velocities [1/s]
    r: np.ndarray                      # (n,) radii [m]
    m: np.ndarray                      # (n,) masses [kg]
    lo: tuple                          # box lower corner [m]
    hi: tuple                          # box upper corner [m]
    periodic: tuple                    # (bool, bool, bool)
    material: Material
    dt: float
    g: tuple = (0.0, 0.0, 0.0)
    floor: bool = True
    floor_v: tuple = (0.0, 0.0, 0.0)
    skin: float = 2.0e-4
    steps: int = 100
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def sphere_masses(r, rho):
    return f32(rho * (4.0 / 3.0) * math.pi * np.asarray(r, dtype=np.float64) ** 3)


def _finish(name, x, v, w, r, mat, lo, hi, periodic, dt, g, floor, floor_v, skin, steps, **meta):
    lo = tuple(qgrid(lo).tolist())
    hi = tuple(qgrid(hi).tolist())
    x = qgrid(x)
    for a in range(3):
        if periodic[a]:
            L = hi[a] - lo[a]
            x[:, a] = lo[a] + np.mod(x[:, a] - lo[a], L)
            x[:, a] = qgrid(x[:, a])
            x[x[:, a] >= hi[a], a] -= L
    r = qgrid(r)
    return Workload(name=name, x=x, v=f32(v), w=f32(w), r=r, m=sphere_masses(r, mat.rho), lo=lo, hi=hi,
                    periodic=tuple(bool(p) for p in periodic), material=mat, dt=float(f32(dt)),
                    g=tuple(f32(g).tolist()), floor=floor, floor_v=tuple(f32(floor_v).tolist()),
                    skin=float(qgrid(skin)), steps=steps, meta=meta)


def column(n: int = 1000, seed: int = 1) -> Workload:
    rng = np.random.default_rng(seed)
    d, sp = 2.0e-3, 2.5e-3
    k = np.arange(n)
    ix, iy, iz = k % 8, (k // 8) % 8, k // 64
    x = np.column_stack([1.25e-3 + sp * ix, 1.25e-3 + sp * iy, 1.25e-3 + sp * iz])
    x += rng.uniform(-0.2e-3, 0.2e-3, (n, 3))
    r = np.full(n, d / 2)
    z = np.zeros((n, 3))
    return _finish("column_1k", x, z, z, r, Material(E=1e7, nu=0.25, e=0.9, mu=0.5, rho=2500.0),
                   (0, 0, 0), (0.02, 0.02, 0.06), (True, True, False), 2e-6, (0, 0, -9.81), True,
                   (0, 0, 0), 0.1 * d, 5000)


def _fcc(nx, ny, a, nlayers):
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    gx, gy, gz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nlayers), indexing="ij")
    cells = np.column_stack([gx.ravel(), gy.ravel(), gz.ravel()]).astype(np.float64)
    pts = (cells[:, None, :] + base[None, :, :]).reshape(-1, 3) * a
    order = np.lexsort((pts[:, 0], pts[:, 1], pts[:, 2]))
    return pts[order]


def shear_bed(n: int = 1_000_000, seed: int = 2, footprint: float = 0.2, height: float = 0.6,
              dmin: float = 1.6e-3, dmax: float = 2.4e-3) -> Workload:
    """Polydisperse bed before settling (see the module docstring)."""
    rng = np.random.default_rng(seed)
    nn = dmax + 0.05e-3                       # nearest-neighbour distance of the start lattice
    ncell = max(1, int(math.floor(footprint / (nn * math.sqrt(2.0)))))
    a = footprint / ncell
    nlayers = int(math.ceil(n / (4 * ncell * ncell)))
    pts = _fcc(ncell, ncell, a, nlayers)[:n]
    pts += np.array([a / 4, a / 4, dmax / 2 + 0.05e-3])
    pts += rng.uniform(-0.02e-3, 0.02e-3, pts.shape)
    d = rng.uniform(dmin, dmax, n)
    z = np.zeros((n, 3))
    return _finish(f"shear_bed_{n}", pts, z, z, d / 2, Material(E=1e7, nu=0.25, e=0.9, mu=0.5, rho=2500.0),
                   (0, 0, 0), (footprint, footprint, height), (True, True, False), 1e-6, (0, 0, -9.81),
                   True, (0, 0, 0), 0.1 * 0.5 * (dmin + dmax), 10_000, lattice_a=a, layers=nlayers)


def dense_block(nx: int = 12, ny: int = 12, nz: int = 10, r: float = 1.0e-3, seed: int = 7,
                squeeze: float = 2e-3, rjit: float = 2e-3, vel: float = 0.05, spin: float = 20.0,
                mat: Material | None = None, floor_v=(0.5, 0.0, 0.0), g=(0.0, 0.0, -9.81),
                dt: float = 1e-6) -> Workload:
    """Overlapping jittered lattice for force parity (random v, spin; floor in contact)."""
    rng = np.random.default_rng(seed)
    sp = 2.0 * r * (1.0 - squeeze)
    gx, gy, gz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = np.column_stack([gx.ravel(), gy.ravel(), gz.ravel()]).astype(np.float64) * sp
    x += np.array([sp / 2, sp / 2, r * (1.0 - squeeze)])
    x += rng.uniform(-0.25, 0.25, x.shape) * squeeze * r
    n = x.shape[0]
    rad = r * (1.0 + rng.uniform(-rjit, rjit, n))
    v = rng.normal(0.0, vel, (n, 3))
    w = rng.normal(0.0, spin, (n, 3))
    return _finish(f"dense_block_{n}", x, v, w, rad, mat or Material(E=1e7, nu=0.25, e=0.6, mu=0.4, rho=2500.0),
                   (0, 0, 0), (nx * sp, ny * sp, nz * sp * 2 + 4 * r), (True, True, False), dt, g, True,
                   floor_v, 0.1 * 2 * r, 100)


def single_sphere(r: float = 1.0e-3, z: float = 0.999e-3, v=(0.2, 0.05, -0.1), w=(30.0, -50.0, 10.0),
                  mat: Material | None = None, dt: float = 1e-6) -> Workload:
    """One sphere just touching the floor of a 10 mm periodic box, sliding and spinning."""
    return _finish("single_sphere", np.array([[5e-3, 5e-3, z]]), np.array([v]), np.array([w]), np.array([r]),
                   mat or Material(E=1e7, nu=0.25, e=0.6, mu=0.4, rho=2500.0), (0, 0, 0), (0.01, 0.01, 0.01),
                   (True, True, False), dt, (0, 0, -9.81), True, (0.3, 0.0, 0.0), 0.1 * 2 * r, 400)


def column_collapse(n: int = 10_000, seed: int = 5, mat: Material | None = None, side: int = 14,
                    spacing: float = 2.1e-3, d: float = 2.0e-3, dt: float = 5e-6, steps: int = 500,
                    box: float = 0.1) -> Workload:
    """A granular column released onto a floor: side x side jittered simple-cubic
    lattice at `spacing` (30 x 30 mm footprint for 14 x 2.1 mm), layers from the
    floor up until n particles; open x/y in a `box` wide domain centred on the column."""
    rng = np.random.default_rng(seed)
    k = np.arange(n)
    x = np.column_stack([(k % side - (side - 1) / 2) * spacing, ((k // side) % side - (side - 1) / 2) * spacing,
                         (k // (side * side)) * spacing + d / 2 + 0.05e-3])
    x += rng.uniform(-0.03e-3, 0.03e-3, x.shape)
    x[:, :2] += box / 2
    top = float(x[:, 2].max()) + 4 * d
    z = np.zeros((n, 3))
    return _finish(f"column_{n}", x, z, z, np.full(n, d / 2), mat or Material(), (0, 0, 0), (box, box, top),
                   (False, False, False), dt, (0, 0, -9.81), True, (0, 0, 0), 0.1 * d, steps,
                   axis=(box / 2, box / 2))


def column_materials(count: int = 64, seed: int = 5) -> list[Material]:
    """Per-instance E log-uniform in [5e6, 5e7] Pa, e ~ U[0.5, 0.95], mu ~ U[0.2, 0.8]."""
    rng = np.random.default_rng(seed + 2000)
    return [Material(E=float(math.exp(rng.uniform(math.log(5e6), math.log(5e7)))), nu=0.25,
                     e=float(rng.uniform(0.5, 0.95)), mu=float(rng.uniform(0.2, 0.8)), rho=2500.0)
            for _ in range(count)]


def coupling_case(seed: int = 50, shift: float = 3.0e-3):
    """A coarse level (d = 4 mm) above and across the top face of a fine region
    (d = 2 mm particles) in a 24 x 24 mm periodic column, for one coupling call:
    coarse positions before (A) and after (B, moved down by `shift`), the fine
    level, and the coupling spec.  Returns (A, B, fine, spec)."""
    rng = np.random.default_rng(seed)
    L, H = 0.024, 0.06
    mat = Material(E=1e7, nu=0.25, e=0.6, mu=0.4, rho=2500.0)
    sp_c = 4.0e-3 * (1 - 2e-3)
    g = np.arange(6) * sp_c + sp_c / 2
    X, Y, Z = np.meshgrid(g, g, np.arange(11) * sp_c + 14.2e-3, indexing="ij")
    xa = np.column_stack([X.ravel(), Y.ravel(), Z.ravel()]) + rng.uniform(-2e-6, 2e-6, (X.size, 3))
    nc = xa.shape[0]
    rc = 2.0e-3 * (1 + rng.uniform(-2e-3, 2e-3, nc))
    vc = rng.normal(0.0, 0.05, (nc, 3)) + np.array([0.0, 0.0, -0.5])
    wc = rng.normal(0.0, 10.0, (nc, 3))
    xb = xa + np.array([0.0, 0.0, -shift]) + rng.uniform(-1e-5, 1e-5, xa.shape)
    A = _finish("coarse_A", xa, vc, wc, rc, mat, (0, 0, 0), (L, L, H), (True, True, False), 1e-6, (0, 0, -9.81),
                True, (0, 0, 0), 0.4e-3, 15)
    B = _finish("coarse_B", xb, vc, wc, rc, mat, (0, 0, 0), (L, L, H), (True, True, False), 1e-6, (0, 0, -9.81),
                True, (0, 0, 0), 0.4e-3, 15)
    sp_f = 2.0e-3 * (1 - 2e-3)
    gf = np.arange(12) * sp_f + sp_f / 2
    Xf, Yf, Zf = np.meshgrid(gf, gf, np.arange(9) * sp_f + 2.0e-3, indexing="ij")   # top within the fade zone
    xf = np.column_stack([Xf.ravel(), Yf.ravel(), Zf.ravel()]) + rng.uniform(-1e-6, 1e-6, (Xf.size, 3))
    # the top layer (inside the controller's fade zone) covers half the face only,
    # so that the other half has room for inserted particles
    top = Zf.ravel() > Zf.max() - 1e-4
    xf = xf[~top | (Xf.ravel() < L / 2)]
    nf = xf.shape[0]
    rf = 1.0e-3 * (1 + rng.uniform(-2e-3, 2e-3, nf))
    fine = _finish("fine", xf, rng.normal(0.0, 0.05, (nf, 3)), rng.normal(0.0, 10.0, (nf, 3)), rf, mat, (0, 0, 0),
                   (L, L, H), (True, True, False), 1e-6, (0, 0, -9.81), True, (0, 0, 0), 0.2e-3, 15)
    spec = dict(lo=(0.0, 0.0, 0.0), hi=(L, L, 0.02), feed_faces=1 << 5, drain_faces=0, surface_cell=12e-3,
                layer=12e-3, corr_cell=8e-3, interval=15, bins=16, alpha=2.0, kp=1.0, ki=1.0 / (10 * 15e-6), kv=0.5,
                mode=1, max_attempts=100, seed=1234, mass_unit=1e-15, max_insert=256, dt=B.dt)
    return A, B, fine, spec


def batch_sizes(count: int = 256, seed: int = 4, nmin: float = 2e3, nmax: float = 2e5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(nmin), math.log(nmax), count))).astype(np.int64)


def settling_box(n: int, seed: int, mat: Material, d: float = 2.0e-3, spacing: float = 2.1e-3,
                 phi: float = 0.45, dt: float = 1e-6, steps: int = 2000) -> Workload:
    """One settling box: footprint s x s with s = (n V_p / phi)^(1/3), periodic x/y, floor;
    jittered simple-cubic lattice at the given spacing; box height = lattice top + 4 d."""
    rng = np.random.default_rng(seed)
    vp = math.pi / 6.0 * d ** 3
    s = (n * vp / phi) ** (1.0 / 3.0)
    per = max(4, int(math.floor(s / spacing)))     # at least 3 cells across for any tuned cell width
    s = per * spacing
    k = np.arange(n)
    x = np.column_stack([(k % per + 0.5) * spacing, ((k // per) % per + 0.5) * spacing,
                         (k // (per * per)) * spacing + d / 2 + 0.05e-3])
    x += rng.uniform(-0.03e-3, 0.03e-3, x.shape)
    height = float(x[:, 2].max()) + 4 * d       # particles only settle: the cell grid need not reach higher
    z = np.zeros((n, 3))
    return _finish(f"box_{n}", x, z, z, np.full(n, d / 2), mat, (0, 0, 0), (s, s, height),
                   (True, True, False), dt, (0, 0, -9.81), True, (0, 0, 0), 0.1 * d, steps)


def batch(count: int = 256, seed: int = 4, scale: float = 1.0, steps: int = 2000) -> list[Workload]:
    """The batched workload: `count` independent boxes (sizes scaled by `scale` for small tests)."""
    sizes = np.maximum(8, np.round(batch_sizes(count, seed) * scale).astype(np.int64))
    rng = np.random.default_rng(seed + 1000)
    out = []
    for k, nk in enumerate(sizes):
        mat = Material(E=float(math.exp(rng.uniform(math.log(5e6), math.log(5e7)))), nu=0.25,
                       e=float(rng.uniform(0.5, 0.95)), mu=float(rng.uniform(0.2, 0.8)), rho=2500.0)
        out.append(settling_box(int(nk), seed + k, mat, steps=steps))
    return out


def _fcc_fill(lo, hi, periodic, d, gap, z_top, rng, jitter=0.01e-3):
    """FCC sites (nearest-neighbour distance >= d + gap) filling [lo, hi] in x/y from the floor up to
    z_top (centres).  Periodic axes take a lattice constant that tiles the period exactly (slightly
    above (d + gap) sqrt 2); open axes keep d/2 + gap/2 clear of the faces."""
    nn = d + gap
    a0 = nn * math.sqrt(2.0)
    a, n, start = [0.0, 0.0], [0, 0], [0.0, 0.0]
    for ax in range(2):
        L = hi[ax] - lo[ax]
        if periodic[ax]:
            n[ax] = max(1, int(math.floor(L / a0)))
            a[ax] = L / n[ax]
            start[ax] = lo[ax] + a[ax] / 4
        else:
            n[ax] = max(1, int(math.floor((L - nn) / a0)) + 1)
            a[ax] = a0
            start[ax] = lo[ax] + nn / 2
    az = a0
    nl = max(1, int(math.floor((z_top - nn / 2) / (az / 2))) + 1)
    pts = []
    for k in range(nl):
        z = nn / 2 + gap + k * az / 2
        ox = 0.0 if k % 2 == 0 else 0.5
        for sx, sy in ((0.0, 0.0), (0.5, 0.5)):
            gx, gy = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="ij")
            px = start[0] + (gx.ravel() + (sx + ox) % 1.0) * a[0]
            py = start[1] + (gy.ravel() + sy) * a[1]
            keep = np.ones(px.shape, dtype=bool)
            if not periodic[0]:
                keep &= px <= hi[0] - nn / 2
            if not periodic[1]:
                keep &= py <= hi[1] - nn / 2
            pts.append(np.column_stack([px[keep], py[keep], np.full(keep.sum(), z)]))
    x = np.vstack(pts)
    x = x[np.lexsort((x[:, 0], x[:, 1], x[:, 2]))]
    return x + rng.uniform(-jitter, jitter, x.shape)


def chute(length: float = 11.0, width: float = 0.3, height: float = 0.3, bed: float = 0.227,
          regions=((2.0, 0.70), (2.30, 0.18)), diameters=(8.0e-3, 4.0e-3, 2.0e-3), seed: int = 3,
          incline_deg: float = 30.0, u0: float = 0.5, dt: float = 1e-6, interval: int = 15,
          clear: float = 1.0, multirate: bool = False, gap: float = 0.05e-3):
    """Three nested coarse-graining levels of an inclined chute (Sec. 2.3 coupling, one dt for all levels).

    Level 0 (d = 8 mm, alpha = 4 against the 2 mm base) fills the whole chute, periodic along the
    flow (x) and across it (y), floor at z = 0, to the bed height.  Level 1 (4 mm) fills the region
    regions[0] = (x start, length) over the full cross-section, level 2 (2 mm) the region
    regions[1] nested inside it.  Each level starts on an FCC lattice (gap 0.05 mm) that is to be
    settled under vertical gravity; the flow then runs with gravity tilted by incline_deg about y
    and every particle given u0 along x (gap: the lattice's clearance between neighbours; a negative
    gap starts the bed compressed, every neighbour pair in contact).  The lattice of a finer level starts `clear` diameters of
    the level above it downstream of its feed face, room for the first inserted particles.
    multirate: level k runs dt times its grain ratio to the finest level (8 mm: 4 dt, 4 mm: 2 dt),
    and `interval` counts steps of the finest level (a multiple of 4 keeps every level whole).  At the default sizes the levels hold about 2.0M, 1.0M and
    2.0M particles.  Returns (levels, specs): three Workloads (gravity already tilted, velocities
    zero) and the two coupling specs (level 0 -> 1, level 1 -> 2): feed through the upstream face,
    drain through the downstream one, cells of three coarse diameters."""
    rng = np.random.default_rng(seed)
    mat = Material(E=1e7, nu=0.25, e=0.9, mu=0.5, rho=2500.0)
    th = math.radians(incline_deg)
    g = (9.81 * math.sin(th), 0.0, -9.81 * math.cos(th))
    boxes = [((0.0, 0.0, 0.0), (length, width, height), (True, True, False))]
    for x0, L in regions:
        boxes.append(((x0, 0.0, 0.0), (x0 + L, width, height), (False, True, False)))
    levels = []
    ratio = [round(d / diameters[-1]) if multirate else 1 for d in diameters]
    for k, (d, (lo, hi, per)) in enumerate(zip(diameters, boxes)):
        flo = lo if k == 0 else (lo[0] + clear * diameters[k - 1], lo[1], lo[2])
        x = _fcc_fill(flo, hi, per, d, gap, bed - d / 2, rng)
        n = x.shape[0]
        z = np.zeros((n, 3))
        levels.append(_finish(f"chute_level{k}", x, z, z, np.full(n, d / 2), mat, lo, hi, per, dt * ratio[k], g,
                              True, (0, 0, 0), 0.1 * d, 5000, diameter=d, u0=u0))
    specs = []
    Tc = interval * float(f32(dt))
    for k in range(len(diameters) - 1):
        lo, hi, _ = boxes[k + 1]
        dc = diameters[k]
        fine_dt = levels[k + 1].dt
        specs.append(dict(lo=tuple(qgrid(lo).tolist()), hi=tuple(qgrid(hi).tolist()), feed_faces=1 << 0,
                          drain_faces=1 << 1, surface_cell=3 * dc, layer=3 * dc, corr_cell=3 * dc,
                          interval=int(round(Tc / fine_dt)), bins=16, alpha=diameters[k] / diameters[k + 1],
                          kp=1.0, ki=1.0 / (10 * Tc), kv=0.5, mode=0, max_attempts=100, seed=seed * 1000 + k,
                          mass_unit=1e-12, max_insert=256, dt=fine_dt))
    return levels, specs


def nested_levels(levels: int = 5, d_fine: float = 1.0e-3, length: float = 11.0, width: float = 0.3,
                  height: float = 0.3, bed: float = 0.227, start: float = 2.0, seed: int = 6, u0: float = 0.5,
                  dt: float = 1e-6, multirate: bool = True):
    """Recursive nesting in the manner of the paper's projection (Sec. 3, runtimes): `levels`
    coarse-graining levels with alpha_l = 2^(l-1) (the coarsest first: d = 2^(levels-1) d_fine ...
    d_fine), each embedded in the next coarser one with a quarter of its filled volume (the
    region length quartered, the cross-section kept), so that each finer level holds about twice
    the particles of the coarser one.  Built on `chute` (30-degree chute, periodic along the flow);
    multi-rate by default, coupling every 16 finest steps."""
    diameters = tuple(d_fine * 2.0 ** (levels - 1 - k) for k in range(levels))
    regions, x0, L = [], start, length
    for k in range(1, levels):
        L = L / 4.0
        regions.append((x0, L))
        x0 = x0 + 0.25 * L            # the next region starts a quarter into this one
    return chute(length=length, width=width, height=height, bed=bed, regions=tuple(regions), diameters=diameters,
                 seed=seed, u0=u0, dt=dt, interval=16, multirate=multirate)


# The silo of Sec. 3 (Table 1): E = 2.5e7 Pa, nu = 0.25, e = 0.5, mu = 0.2 (particle-particle),
# 0.175 (particle-wall), rho = 1000 kg/m^3, d = 2.8 mm, dt = 1e-6 s.
SILO_MATERIAL = Material(E=2.5e7, nu=0.25, e=0.5, mu=0.2, mu_wall=0.175, rho=1000.0)


def silo_walls(z_o: float, r_o: float = 0.02, R: float = 0.135, h_cone: float = 0.2, h_cyl: float = 0.2,
               closed: bool = True):
    """Polyline (rho, z) of the silo wall: a cone from the orifice radius r_o at z_o up to R over
    h_cone, then a cylinder of radius R for h_cyl more; closed: a disk (0, z_o) - (r_o, z_o) shuts
    the orifice (the filling phase)."""
    pts = [(r_o, z_o), (R, z_o + h_cone), (R, z_o + h_cone + h_cyl)]
    if closed:
        pts = [(0.0, z_o)] + pts
    return qgrid(np.asarray(pts, dtype=np.float64))


def _fcc_in_vessel(nn, r_wall, z_lo, z_hi, R, clear, n, rng, jitter):
    """The n lowest (n None: all) FCC sites (nearest-neighbour distance nn) about the vertical axis at the origin
    whose distance from the axis stays `clear` inside r_wall(z) (a horizontal distance: a sphere
    clears a sloped wall only where clear times the cosine of the wall's slope exceeds its
    radius), from z_lo + clear up."""
    a = nn * math.sqrt(2.0)
    m = int(math.ceil(R / a)) + 1
    kz = int(math.ceil((z_hi - z_lo) / a)) + 1
    i, j, k = np.meshgrid(np.arange(-m, m + 1), np.arange(-m, m + 1), np.arange(kz), indexing="ij")
    base = np.column_stack([i.ravel(), j.ravel(), k.ravel()]).astype(np.float64) * a
    pts = np.vstack([base + np.array(o) * a for o in ((0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5))])
    pts[:, 2] += z_lo + clear
    rho = np.hypot(pts[:, 0], pts[:, 1])
    keep = (rho <= r_wall(pts[:, 2]) - clear) & (pts[:, 2] <= z_hi - clear)
    pts = pts[keep]
    pts = pts[np.lexsort((pts[:, 0], pts[:, 1], pts[:, 2]))]
    if n is None:                                # all sites
        n = pts.shape[0]
    if pts.shape[0] < n:
        raise ValueError(f"the vessel holds {pts.shape[0]} lattice sites, {n} asked")
    return pts[:n] + rng.uniform(-jitter, jitter, (n, 3))


def silo(alpha: int = 1, n_ref: int = 187_504, d_ref: float = 2.8e-3, seed: int = 17, z_o: float = 0.05,
         gap: float = 0.3, v_rand: float = 0.1, dt: float = 1e-6):
    """The silo of Sec. 3: 40 cm tall, the upper half a cylinder of diameter 27 cm, the lower half a
    cone narrowing to a 4 cm orifice at height z_o above the box floor (the orifice closed by a disk
    while filling).  Filled with n_ref / alpha^3 spheres of d = alpha d_ref (alpha = 1: the
    reference, 187,504 x 2.8 mm; alpha = 2: the coarse-grain model, 23,438 x 5.6 mm) on an FCC
    lattice (nearest-neighbour distance (1 + gap) d) inside the vessel with d of clearance, lowest
    sites first, each jittered by +-0.01 d and given a velocity uniform in +-v_rand per axis: the
    synthetic stand-in for the paper's pouring from the top, to be settled under gravity.  No box
    floor; the box spans the vessel with 2 d of margin and z from 0."""
    rng = np.random.default_rng(seed + alpha)
    d = alpha * d_ref
    n = int(round(n_ref / alpha ** 3))
    r_o, R, h_cone, h_cyl = 0.02, 0.135, 0.2, 0.2

    def r_wall(z):
        return np.where(z < z_o + h_cone, r_o + (R - r_o) * (z - z_o) / h_cone, R)

    x = _fcc_in_vessel((1.0 + gap) * d, r_wall, z_o, z_o + h_cone + h_cyl, R, d, n, rng, 0.01 * d)
    v = rng.uniform(-v_rand, v_rand, (n, 3))
    m = R + 2 * d
    wl = _finish(f"silo_alpha{alpha}", x, v, np.zeros((n, 3)), np.full(n, d / 2), SILO_MATERIAL, (-m, -m, 0.0),
                 (m, m, z_o + h_cone + h_cyl + 0.05), (False, False, False), dt, (0.0, 0.0, -9.81), False,
                 (0, 0, 0), 0.1 * d, 0, alpha=alpha, diameter=d, z_o=z_o, r_o=r_o, R=R, h_cone=h_cone,
                 h_cyl=h_cyl)
    return wl


def small_vessel(seed: int = 21, n: int = 600, d: float = 2.0e-3, closed: bool = True, packed: bool = True):
    """A small cone-and-cylinder vessel (orifice radius 4 mm at z = 10 mm, cone to 12 mm over 10 mm,
    cylinder to z = 40 mm), for parity: packed = True fills it from the bottom on an FCC lattice
    (nearest neighbour 1.1 d; centres 0.65 d from the wall horizontally and above the orifice, so
    that no sphere starts in contact with the cone, whose normal is 39 degrees from horizontal)
    with random velocities of +-0.5 m/s; packed =
    False scatters n spheres uniformly over the vessel's bounding cylinder, so that many overlap a
    wall, a rim or the orifice disk (and some lie outside the wall): the input for the
    single-evaluation force parity.  Material of Table 1 with d = 2 mm."""
    rng = np.random.default_rng(seed)
    z_o, r_o, R, h_cone, h_cyl = 0.01, 0.004, 0.012, 0.01, 0.02

    def r_wall(z):
        return np.where(z < z_o + h_cone, r_o + (R - r_o) * (z - z_o) / h_cone, R)

    if packed:
        x = _fcc_in_vessel(1.1 * d, r_wall, z_o, z_o + h_cone + h_cyl, R, 0.65 * d, n, rng, 0.01 * d)
        v = rng.uniform(-0.5, 0.5, (n, 3))
        w = np.zeros((n, 3))
    else:
        rho = (R + 0.5 * d) * np.sqrt(rng.uniform(0.0, 1.0, n))
        ph = rng.uniform(0.0, 2.0 * math.pi, n)
        z = rng.uniform(z_o - 0.5 * d, z_o + h_cone + h_cyl + 0.5 * d, n)
        x = np.column_stack([rho * np.cos(ph), rho * np.sin(ph), z])
        v = rng.uniform(-0.5, 0.5, (n, 3))
        w = rng.uniform(-100.0, 100.0, (n, 3))
    pts = [(r_o, z_o), (R, z_o + h_cone), (R, z_o + h_cone + h_cyl)]
    if closed:
        pts = [(0.0, z_o)] + pts
    m = R + 2 * d
    wl = _finish("small_vessel", x, v, w, np.full(n, d / 2), SILO_MATERIAL, (-m, -m, 0.0), (m, m, 0.05),
                 (False, False, False), 1e-6, (0.0, 0.0, -9.81), False, (0, 0, 0), 0.1 * d, 0, z_o=z_o,
                 walls=qgrid(np.asarray(pts, dtype=np.float64)))
    return wl


def vessel_sphere(case: str = "cone", d: float = 2.0e-3, overlap: float = 2.0e-7):
    """One sphere against the small vessel's wall (orifice radius 4 mm at z = 10 mm, cone to 12 mm
    over 10 mm, cylinder above), for parity of a wall contact carried over many steps:

    * ``cone``: halfway up the cone, pressed into it by `overlap`, moving azimuthally at 0.3 m/s
      (it runs round the cone under gravity);
    * ``kink``: in the corner where the cone meets the cylinder, `overlap` into both;
    * ``rim``: with the orifice open, leaning on the rim's edge from inside the hole (centre
      below the cone's normal at the rim, so the edge is its only contact), `overlap` into it:
      it slides off the edge and falls through."""
    z_o, r_o, R, h_cone = 0.01, 0.004, 0.012, 0.01
    r = d / 2
    s = (R - r_o) / h_cone                       # d rho / d z of the cone
    c = 1.0 / math.sqrt(1.0 + s * s)             # the cone's inward normal is (-c, s c) in (rho, z)
    pts = [(r_o, z_o), (R, z_o + h_cone), (R, z_o + 2 * h_cone)]
    v = np.zeros((1, 3))
    w = np.zeros((1, 3))
    a = r - overlap
    if case == "cone":
        zc = z_o + 0.5 * h_cone
        rc = r_o + s * (zc - z_o)
        rho, z = rc - a * c, zc + a * s * c
        v[0] = (0.0, 0.3, 0.0)
    elif case == "kink":
        # a from the cylinder (rho = R - a) and a from the cone: the contact point on the cone
        # at height zc satisfies r_o + s (zc - z_o) - a c = R - a
        zc = z_o + (R - r_o - a * (1.0 - c)) / s
        rho, z = R - a, zc + a * s * c
    elif case == "rim":
        e = a / math.sqrt(1.25)                  # centre (r_o - e, z_o + e / 2), |.| = a from the edge
        rho, z = r_o - e, z_o + 0.5 * e
    else:
        raise ValueError(case)
    x = np.array([[rho, 0.0, z]])
    m = R + 2 * d
    return _finish(f"vessel_sphere_{case}", x, v, w, np.full(1, r), SILO_MATERIAL, (-m, -m, 0.0), (m, m, 0.05),
                   (False, False, False), 1e-6, (0.0, 0.0, -9.81), False, (0, 0, 0), 0.1 * d, 0,
                   walls=qgrid(np.asarray(pts, dtype=np.float64)))


def silo_two_level(seed: int = 17, z_o: float = 0.05, h_fine: float = 0.10, cell: float = 0.0199,
                   dt: float = 1e-6, interval: int = 15):
    """The multi-level silo of Sec. 3: the coarse-grain silo of ``silo(2)`` (23,438 x 5.6 mm) over
    its whole height, and a fine level (2.8 mm) in the lower quarter, the region |x|, |y| <= 8 cm
    (the cone's radius there is at most 7.75 cm), z_o - 2 cm <= z <= z_o + h_fine, coupled through
    its top face; the correction cells below the orifice couple the coarse particles that passed
    it to the fine velocity alone, those above it to the fine mass flow (Sec. 3).  Surface, transition-layer (one cell deep) and correction cells are 2 cm cubes (the
    paper's grid of 2 cm cells: a top layer for the transition, the cells below for the mass-flow
    correction; `cell` is the least side, the region's 16 x 16 x 10 cm divide into 8 x 8 x 5 cells
    of 2 cm); the controller acts every `interval` = 15 steps (Sec. 3).  The
    fine level starts on an FCC lattice (nearest neighbour 1.05 d, a packing fraction of 0.64)
    filling the region inside the cone up to one diameter below its top face (about 44,000
    spheres), with the coarse level's start otherwise; both are to be settled together.
    Returns (coarse, fine, spec)."""
    coarse = silo(2, seed=seed, z_o=z_o, dt=dt)
    rng = np.random.default_rng(seed + 100)
    d = 2.8e-3
    r_o, R, h_cone = coarse.meta["r_o"], coarse.meta["R"], coarse.meta["h_cone"]

    def r_wall(z):
        return np.where(z < z_o + h_cone, r_o + (R - r_o) * (z - z_o) / h_cone, R)

    # every lattice site of the region inside the cone with d of clearance
    x = _fcc_in_vessel(1.05 * d, r_wall, z_o, z_o + h_fine, 0.08, d, None, rng, 0.01 * d)
    n = x.shape[0]
    v = rng.uniform(-0.1, 0.1, (n, 3))
    m = 0.09
    fine = _finish("silo_fine", x, v, np.zeros((n, 3)), np.full(n, d / 2), SILO_MATERIAL, (-m, -m, 0.0),
                   (m, m, z_o + h_fine + 0.03), (False, False, False), dt, (0.0, 0.0, -9.81), False, (0, 0, 0),
                   0.1 * d, 0, diameter=d, z_o=z_o)
    Tc = interval * float(f32(dt))
    # the region reaches one cell below the orifice: coarse particles that passed it are
    # coupled to the fine velocity alone (Sec. 3), those above it to the fine mass flow
    spec = dict(lo=tuple(qgrid((-0.08, -0.08, z_o - 0.02)).tolist()),
                hi=tuple(qgrid((0.08, 0.08, z_o + h_fine)).tolist()),
                feed_faces=1 << 5, drain_faces=0, surface_cell=cell, layer=cell, corr_cell=cell, interval=interval,
                bins=16, alpha=2.0, kp=1.0, ki=1.0 / (10 * Tc), kv=0.5, mode=1, max_attempts=100, seed=seed * 1000,
                mass_unit=1e-12, max_insert=256, dt=fine.dt, velocity_below=float(qgrid(z_o)))
    return coarse, fine, spec
