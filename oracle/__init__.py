"""Plain FP64 CPU oracle for the DEM hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The
product path (``paper_1705_03850_gb300``) never imports it, and it imports
nothing from the product path.

The arithmetic lives in ``dem_oracle.c`` and ``dem_oracle_dyn.h`` (plain C,
double precision), compiled here with gcc into ``oracle/_build/liboracle.so``
and called through ctypes.  ``dem_oracle_cs.c`` compiles the same dynamics
with complex numbers for complex-step derivatives (the FP64 reference
gradient of rollouts with respect to E, e and mu).
What it follows, by section and equation of Queteschiner et al. (2017):

* Sec. 2.1, Eqs. 1-2: Newton's equations for translation and rotation,
  advanced by velocity Verlet (the paper names no integrator).
* Eqs. 3-4: damped normal and tangential spring-dashpot forces, with the
  tangential overlap carried over a contact's life.
* Eq. 5: Coulomb truncation of the tangential overlap, |f_t| <= mu |f_n|.
* Eq. 6: non-linear damped Hertz coefficients and beta(e).
* Sec. 2.2: coarse-grain scaling (r -> alpha r with rho, e, E, mu kept).

Pins (tests/test_oracle_*.py) tie it to closed forms and invariants rather
than to itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("dem_oracle.c", "dem_oracle_cs.c", "dem_oracle_couple.c")]
_HDRS = [os.path.join(_HERE, f) for f in ("dem_oracle_common.h", "dem_oracle_dyn.h")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lib = None
_lib_omp = None

NPARAM = 43


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle's C source with gcc (plain -O2, no fast-math).  openmp: the same
    source with OpenMP, which runs the per-pair contact law on all host cores (the sums over
    pairs stay serial, so the results are bit-identical to the serial build)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP_PATH if openmp else _LIB_PATH
    newest = max(os.path.getmtime(f) for f in _SRCS + _HDRS)
    if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off"] +
                              (["-fopenmp"] if openmp else []) + ["-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, path)
    return path


def _load(openmp: bool = False):
    global _lib, _lib_omp
    if openmp and _lib_omp is not None:
        return _lib_omp
    if not openmp and _lib is not None:
        return _lib
    lib = ctypes.CDLL(build(openmp=openmp))
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64 = ctypes.c_int64
    lib.orc_beta.restype = ctypes.c_double
    lib.orc_beta.argtypes = [ctypes.c_double]
    lib.orc_pair_coeffs.restype = None
    lib.orc_pair_coeffs.argtypes = [dp] + [ctypes.c_double] * 5 + [ctypes.c_int32, dp]
    for fn in (lib.orc_pairs_brute, lib.orc_pairs_cells):
        fn.restype = i64
        fn.argtypes = [dp, i64, dp, dp, ctypes.c_double, i64, i64p, i64p]
    lib.orc_eval.restype = i64
    lib.orc_eval.argtypes = [dp, i64, dp, dp, dp, dp, dp, i64p, dp, i64, i64p, i64p, dp,
                             ctypes.c_double, ctypes.c_int32, dp, dp, i64, i64p, i64p, dp,
                             i32p, dp]
    lib.orc_cs_run_derivative.restype = ctypes.c_int32
    lib.orc_cs_run_derivative.argtypes = [dp, ctypes.c_int32, ctypes.c_double, i64, dp, dp, dp, dp, dp, i64p, i64,
                                          ctypes.c_int32, i64] + [dp] * 10
    u64 = ctypes.c_uint64
    lib.orc_couple.restype = ctypes.c_int32
    lib.orc_couple.argtypes = ([dp, u64, ctypes.c_int32, dp, i64, dp, dp, dp, dp, dp, i64p, i64, i64p, i64p, dp,
                                dp, i64, dp, dp, dp, dp, dp, i64p, i64, i64p, i64p, dp, ctypes.c_double, ctypes.c_double, dp, i32p, i64p, dp, ctypes.c_double,
                                ctypes.c_double, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_uint32), dp, dp, dp, dp,
                                dp, dp, i32p, dp, dp, i32p, i32p])
    lib.orc_run.restype = ctypes.c_int32
    lib.orc_run.argtypes = [dp, i64, dp, dp, dp, dp, dp, i64p, dp, i64p, i64, i64p, i64p, dp,
                            i32p, dp, dp, i64, ctypes.c_int32, ctypes.c_int32]
    if openmp:
        _lib_omp = lib
    else:
        _lib = lib
    return lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def make_params(*, E, nu, e, mu, dt, g=(0.0, 0.0, 0.0), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                periodic=(False, False, False), mu_wall=None, floor=False, floor_z=0.0,
                floor_v=(0.0, 0.0, 0.0), clamp_fn=False, walls=None) -> np.ndarray:
    """The oracle's flat parameter block (layout documented in dem_oracle.c).  walls: None or
    dict(axis=(x, y), points=[(rho, z), ...]) -- axisymmetric walls, the surface of revolution
    of the polyline about the vertical axis (at most 8 points)."""
    P = np.zeros(NPARAM, dtype=np.float64)
    P[0], P[1], P[2], P[3] = E, nu, e, mu
    P[4] = mu if mu_wall is None else mu_wall
    P[5] = dt
    P[6:9] = g
    P[9:12] = lo
    P[12:15] = hi
    P[15:18] = [1.0 if p else 0.0 for p in periodic]
    P[18] = 1.0 if floor else 0.0
    P[19] = floor_z
    P[20:23] = floor_v
    P[23] = 1.0 if clamp_fn else 0.0
    if walls is not None:
        pts = np.asarray(walls["points"], dtype=np.float64).reshape(-1, 2)
        if not 2 <= len(pts) <= 8:
            raise ValueError("2 to 8 wall profile points")
        P[24] = len(pts)
        P[25:27] = walls["axis"]
        P[27:27 + 2 * len(pts)] = pts.ravel()
    return P


def beta(e: float) -> float:
    """beta(e) = ln e / sqrt(ln^2 e + pi^2) (Eq. 6)."""
    return _load().orc_beta(float(e))


def pair_coeffs(P, ri, rj, mi, mj, delta, wall=False) -> dict:
    """E_eff, G_eff, R_eff, m_eff, k_n, gamma_n, k_t, gamma_t of one contact (Eq. 6)."""
    out = np.zeros(8)
    _load().orc_pair_coeffs(_d(np.ascontiguousarray(P, dtype=np.float64)), ri, rj, mi, mj,
                            delta, 1 if wall else 0, _d(out))
    keys = ["Eeff", "Geff", "Reff", "meff", "kn", "gn", "kt", "gt"]
    return dict(zip(keys, out.tolist()))


def pairs(P, x, r, extra=0.0, method="cells") -> np.ndarray:
    """Index pairs (i < j) with |x_ij| < r_i + r_j + extra, sorted; shape (n, 2)."""
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    r = np.ascontiguousarray(r, dtype=np.float64)
    fn = lib.orc_pairs_brute if method == "brute" else lib.orc_pairs_cells
    cap = max(16, 8 * len(r))
    while True:
        pi = np.zeros(cap, dtype=np.int64)
        pj = np.zeros(cap, dtype=np.int64)
        cnt = fn(_d(P), len(r), _d(x), _d(r), float(extra), cap, _i64(pi), _i64(pj))
        if cnt <= cap:
            return np.stack([pi[:cnt], pj[:cnt]], axis=1)
        cap = int(cnt)


PARAM_INDEX = {"E": 0, "e": 1, "mu": 2}


def rollout_derivative(P, x, v, w, r, m, nsteps, param, h=None, ids=None, use_cells=True):
    """State after `nsteps` from (x, v, w) with empty history, and its derivative with
    respect to one material parameter ("E", "e" or "mu") by a complex step.

    Returns dict with x, v, w, F, T (step nsteps) and dx, dv, dw, dF, dT.
    """
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    which = PARAM_INDEX[param]
    base = float(P[[0, 2, 3][which]])
    h = h if h is not None else 1e-30 * max(abs(base), 1e-300)
    ids = np.arange(n, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    outs = {k: np.zeros((n, 3)) for k in ("x", "v", "w", "F", "T", "dx", "dv", "dw", "dF", "dT")}
    rc = lib.orc_cs_run_derivative(_d(P), which, float(h), n, _d(x), _d(np.ascontiguousarray(v, dtype=np.float64)),
                                   _d(np.ascontiguousarray(w, dtype=np.float64)),
                                   _d(np.ascontiguousarray(r, dtype=np.float64)),
                                   _d(np.ascontiguousarray(m, dtype=np.float64)), _i64(ids), int(nsteps),
                                   1 if use_cells else 0, max(64, 16 * n),
                                   *[_d(outs[k]) for k in ("x", "v", "w", "F", "T", "dx", "dv", "dw", "dF", "dT")])
    if rc != 0:
        raise RuntimeError("oracle history capacity exceeded")
    return outs


def quantum(lo, hi):
    """Length unit of a level's integer positions: the smallest power of two with
    (largest box extent) / q <= 2^30 (the rule the library documents)."""
    import math
    emax = max(h - l for l, h in zip(lo, hi))
    q = 2.0 ** math.ceil(math.log2(emax / 2.0 ** 30))
    while emax / q > 2.0 ** 30:
        q *= 2.0
    return q


class Coupler:
    """FP64 oracle of the coarse/fine coupling (see dem_oracle_couple.c).

    spec: dict with the fields of dem_coupling; Pc, Pf: parameter blocks of the
    levels; rmax_f: the fine level's largest radius (the range of the radius
    histogram) [m]; rho_f: fine density; idcap: coarse IDs; band: insertion
    decisions whose clearance is within (-band, band) [m] are reported per cell
    in out["border"] (first such attempt, -1: none).
    """

    def __init__(self, spec, Pc, Pf, rmax_f, rho_f, idcap, band=0.0):
        self.CP = np.zeros(24)
        self.CP[0:3] = spec["lo"]
        self.CP[3:6] = spec["hi"]
        self.CP[6] = spec["feed_faces"]
        self.CP[7] = spec.get("drain_faces", 0)
        self.CP[8] = spec["surface_cell"]
        self.CP[9] = spec["layer"]
        self.CP[10] = spec["corr_cell"]
        self.CP[11] = spec["interval"]
        self.CP[12] = spec["bins"]
        self.CP[13] = spec["alpha"]
        self.CP[14] = spec["kp"]
        self.CP[15] = spec["ki"]
        self.CP[16] = spec["kv"]
        self.CP[17] = spec["mode"]
        self.CP[18] = spec["max_attempts"]
        vb = spec.get("velocity_below", None)
        self.CP[19] = -np.inf if vb is None or np.isnan(vb) else vb
        self.CP[20] = spec["mass_unit"]
        self.CP[21] = spec["max_insert"]
        self.CP[22] = spec["dt"]
        self.CP[23] = rho_f
        self.seed = int(spec["seed"])
        self.Pc = np.ascontiguousarray(Pc, dtype=np.float64)
        self.Pf = np.ascontiguousarray(Pf, dtype=np.float64)
        self.rmax_f = float(rmax_f)
        self.band = float(band)
        self.prev = np.zeros((idcap, 3))
        self.prev_ok = np.zeros(idcap, dtype=np.int32)
        self.calls = 0
        self.S = None

    def _sizes(self):
        lo, hi, sc, cc = self.CP[0:3], self.CP[3:6], self.CP[8], self.CP[10]
        S = 0
        for bit in range(6):
            if not (int(self.CP[6]) >> bit) & 1:
                continue
            a = bit // 2
            b, c = sorted(((a + 1) % 3, (a + 2) % 3))
            S += max(1, int(np.floor((hi[b] - lo[b]) / sc))) * max(1, int(np.floor((hi[c] - lo[c]) / sc)))
        C = 1
        for a in range(3):
            C *= max(1, int(np.floor((hi[a] - lo[a]) / cc)))
        return S, C

    def record(self, xc, idc):
        for i, k in enumerate(np.asarray(idc)):
            self.prev[k] = xc[i]
            self.prev_ok[k] = 1

    def call(self, coarse, fine, dth_c, dth_f):
        """coarse, fine: dicts x, v, w, r, m, id (float64 / int64 arrays) and optionally the
        contact history hist = (a, b, xi) as Sim.history() gives it (none: no stored overlaps).
        Returns a dict of outputs."""
        lib = _load()
        S, C = self._sizes()
        if self.S is None:
            self.S = S
            self.carry = np.zeros(S, dtype=np.int64)
            self.integ = np.zeros(S)
        self.calls += 1
        bins, mi = int(self.CP[12]), int(self.CP[21])
        nc, nf = len(coarse["r"]), len(fine["r"])
        out = dict(cross=np.zeros(S, dtype=np.uint64), hist=np.zeros(S * bins, dtype=np.uint32), fav=np.zeros(S * 4),
                   lay=np.zeros(2 * S * 11), ctrl=np.zeros(S * 3), cor=np.zeros(2 * C * 5), fext_c=np.zeros(nc * 3),
                   fext_f=np.zeros(nf * 3), removed=np.zeros(nf, dtype=np.int32),
                   ins_x=np.zeros(S * mi * 4), ins_m=np.zeros(S * mi), nins=np.zeros(S, dtype=np.int32),
                   border=np.zeros(S, dtype=np.int32))
        def hist(lv):
            a, b, x = lv.get("hist", (np.zeros(0), np.zeros(0), np.zeros((0, 3))))[:3]
            return (len(a), np.ascontiguousarray(a, dtype=np.int64), np.ascontiguousarray(b, dtype=np.int64),
                    np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3)))
        hc, hf = hist(coarse), hist(fine)
        c = {k: np.ascontiguousarray(v, dtype=np.int64 if k == "id" else np.float64) for k, v in coarse.items()
             if k != "hist"}
        f = {k: np.ascontiguousarray(v, dtype=np.int64 if k == "id" else np.float64) for k, v in fine.items()
             if k != "hist"}
        u64p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        u32p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        lib.orc_couple(_d(self.CP), self.seed, self.calls, _d(self.Pc), nc, _d(c["x"]), _d(c["v"]), _d(c["w"]),
                       _d(c["r"]), _d(c["m"]), _i64(c["id"]), hc[0], _i64(hc[1]), _i64(hc[2]), _d(hc[3]),
                       _d(self.Pf), nf, _d(f["x"]), _d(f["v"]), _d(f["w"]),
                       _d(f["r"]), _d(f["m"]), _i64(f["id"]), hf[0], _i64(hf[1]), _i64(hf[2]), _d(hf[3]),
                       self.rmax_f, self.band, _d(self.prev),
                       _i32(self.prev_ok), _i64(self.carry), _d(self.integ), float(dth_c), float(dth_f),
                       u64p(out["cross"]), u32p(out["hist"]), _d(out["fav"]), _d(out["lay"]), _d(out["ctrl"]),
                       _d(out["cor"]), _d(out["fext_c"]), _d(out["fext_f"]), _i32(out["removed"]), _d(out["ins_x"]),
                       _d(out["ins_m"]), _i32(out["nins"]), _i32(out["border"]))
        out["carry"] = self.carry.copy()
        out["hist"] = out["hist"].reshape(S, bins)
        out["fav"] = out["fav"].reshape(S, 4)
        out["lay"] = out["lay"].reshape(2, S, 11)
        out["ctrl"] = out["ctrl"].reshape(S, 3)
        out["cor"] = out["cor"].reshape(2, C, 5)
        out["ins_x"] = out["ins_x"].reshape(S, mi, 4)
        out["ins_m"] = out["ins_m"].reshape(S, mi)
        out["fext_c"] = out["fext_c"].reshape(nc, 3)
        out["fext_f"] = out["fext_f"].reshape(nf, 3)
        return out


class Sim:
    """A DEM system advanced by the oracle (all arrays float64 / int64, SI units).

    State at an integer step n: x, v, w (angular velocity), and -- once
    evaluated -- F, T and the contact history (one record per contact, keyed by
    the particle IDs (a < b), or (a, -1) for the floor).
    """

    def __init__(self, P, x, v, w, r, m, ids=None, use_cells=True, openmp=False):
        self.openmp = bool(openmp)
        self.P = np.ascontiguousarray(P, dtype=np.float64)
        self.x = np.array(x, dtype=np.float64).reshape(-1, 3)
        n = self.x.shape[0]
        self.v = np.array(v, dtype=np.float64).reshape(n, 3)
        self.w = np.array(w, dtype=np.float64).reshape(n, 3)
        self.r = np.array(r, dtype=np.float64).reshape(n)
        self.m = np.array(m, dtype=np.float64).reshape(n)
        self.id = (np.arange(n, dtype=np.int64) if ids is None
                   else np.array(ids, dtype=np.int64).reshape(n))
        self.use_cells = 1 if use_cells else 0
        self.cap = max(64, 16 * n)
        self.ha = np.zeros(self.cap, dtype=np.int64)
        self.hb = np.zeros(self.cap, dtype=np.int64)
        self.hxi = np.zeros((self.cap, 3), dtype=np.float64)
        self.slip = np.zeros(self.cap, dtype=np.int32)
        self.nh = np.zeros(1, dtype=np.int64)
        self.F = np.zeros((n, 3))
        self.T = np.zeros((n, 3))
        self.primed = 0
        # held external force per particle [N] (None: none), added at every evaluation
        self.fext = None

    def _fext(self):
        if self.fext is None:
            return None
        self.fext = np.ascontiguousarray(self.fext, dtype=np.float64).reshape(self.n, 3)
        return _d(self.fext)

    @property
    def n(self):
        return self.x.shape[0]

    def set_history(self, a, b, xi):
        """Replace the stored history by records (a, b, xi); sorted here."""
        a = np.asarray(a, dtype=np.int64)
        b = np.asarray(b, dtype=np.int64)
        order = np.lexsort((b, a))
        k = len(a)
        self.ha[:k] = a[order]
        self.hb[:k] = b[order]
        self.hxi[:k] = np.asarray(xi, dtype=np.float64).reshape(-1, 3)[order]
        self.nh[0] = k

    def history(self):
        k = int(self.nh[0])
        return self.ha[:k].copy(), self.hb[:k].copy(), self.hxi[:k].copy(), self.slip[:k].copy()

    def checkpoint(self):
        """A copy of the whole state: x, v, w, r, m, IDs, the forces of the last evaluation,
        the contact history and whether that evaluation has been done."""
        ha, hb, hxi, slip = self.history()
        return dict(x=self.x.copy(), v=self.v.copy(), w=self.w.copy(), r=self.r.copy(), m=self.m.copy(),
                    id=self.id.copy(), F=self.F.copy(), T=self.T.copy(), ha=ha, hb=hb, hxi=hxi, slip=slip,
                    primed=self.primed, use_cells=self.use_cells)

    @classmethod
    def restore(cls, P, ck):
        """A simulation continuing from a checkpoint() (same parameters P)."""
        s = cls(P, ck["x"], ck["v"], ck["w"], ck["r"], ck["m"], ids=ck["id"], use_cells=bool(ck["use_cells"]))
        k = len(ck["ha"])
        s.ha[:k], s.hb[:k], s.hxi[:k], s.slip[:k] = ck["ha"], ck["hb"], ck["hxi"], ck["slip"]
        s.nh[0] = k
        s.F[:] = ck["F"]
        s.T[:] = ck["T"]
        s.primed = ck["primed"]
        return s

    def evaluate(self, dt_hist=0.0):
        """Forces at the current state without changing it.

        Returns (F, T, (a, b, xi, slip), fabs) where fabs[i] = sum_j |F_ij| + |m_i g|.
        """
        lib = _load(self.openmp)
        n = self.n
        F = np.zeros((n, 3))
        T = np.zeros((n, 3))
        fabs = np.zeros(n)
        ha = np.zeros(self.cap, dtype=np.int64)
        hb = np.zeros(self.cap, dtype=np.int64)
        hxi = np.zeros((self.cap, 3))
        slip = np.zeros(self.cap, dtype=np.int32)
        c = lib.orc_eval(_d(self.P), n, _d(self.x), _d(self.v), _d(self.w), _d(self.r), _d(self.m),
                         _i64(self.id), self._fext(), int(self.nh[0]), _i64(self.ha), _i64(self.hb), _d(self.hxi),
                         float(dt_hist), self.use_cells, _d(F), _d(T), self.cap, _i64(ha), _i64(hb),
                         _d(hxi), _i32(slip), _d(fabs))
        if c < 0:
            raise RuntimeError("oracle history capacity exceeded")
        return F, T, (ha[:c], hb[:c], hxi[:c], slip[:c]), fabs

    def run(self, nsteps: int):
        lib = _load(self.openmp)
        rc = lib.orc_run(_d(self.P), self.n, _d(self.x), _d(self.v), _d(self.w), _d(self.r),
                         _d(self.m), _i64(self.id), self._fext(), _i64(self.nh), self.cap, _i64(self.ha),
                         _i64(self.hb), _d(self.hxi), _i32(self.slip), _d(self.F), _d(self.T),
                         int(nsteps), self.primed, self.use_cells)
        if rc != 0:
            raise RuntimeError("oracle history capacity exceeded")
        self.primed = 1
        return self


def grid_fields(x, v, r, m, lo, h, n):
    """Volume averages on a uniform grid (the plain definition): per cell (x fastest) the
    solid volume of the particles whose centre lies in it over the cell volume, their mass
    and their mass-weighted mean velocity (0 in empty cells).  Returns (n2, n1, n0, 5)."""
    x = np.asarray(x, dtype=np.float64)
    idx = np.floor((x - np.asarray(lo, dtype=np.float64)) / h).astype(np.int64)
    ok = np.all((idx >= 0) & (idx < np.asarray(n)), axis=1)
    out = np.zeros((n[2], n[1], n[0], 5))
    vol = 4.0 / 3.0 * np.pi * np.asarray(r, dtype=np.float64) ** 3
    for i in np.nonzero(ok)[0]:
        c = out[idx[i, 2], idx[i, 1], idx[i, 0]]
        c[0] += vol[i]
        c[1] += m[i]
        c[2:5] += m[i] * v[i]
    out[..., 0] /= h ** 3
    mass = out[..., 1:2]
    out[..., 2:5] = np.where(mass > 0, out[..., 2:5] / np.where(mass > 0, mass, 1.0), 0.0)
    return out
