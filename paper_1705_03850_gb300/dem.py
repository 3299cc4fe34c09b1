"""Thin ctypes binding of the C ABI in include/dem.h (argument marshalling only).

Every step of the computation runs in the CUDA library ``_build/libcgdem.so``;
this module only allocates the caller-owned workspace with PyTorch, passes
PyTorch's current stream, and converts arrays.  There is no CPU fallback: if
the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
import sys

import numpy as np

from .build import LIB, LIB_CHECKED

# field ids (dem_field)
POS, VEL, OMEGA, RADIUS, MASS, FORCE, TORQUE, WALL_XI, NBR_COUNT, FEXT = range(10)
_WIDTH = {POS: 3, VEL: 3, OMEGA: 3, RADIUS: 1, MASS: 1, FORCE: 3, TORQUE: 3, WALL_XI: 3, NBR_COUNT: 1, FEXT: 3}
STATUS = {0: "DEM_OK", 1: "DEM_ERR_ARG", 2: "DEM_ERR_CAPACITY", 3: "DEM_ERR_CUDA", 4: "DEM_ERR_NONFINITE",
          5: "DEM_ERR_ESCAPED", 6: "DEM_ERR_TIMEOUT", 7: "DEM_ERR_STATE", 8: "DEM_ERR_BOUNDS"}


class DemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class InstanceDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("capacity", ctypes.c_int64), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("periodic", ctypes.c_int32 * 3), ("floor_on", ctypes.c_int32),
                ("floor_v", ctypes.c_double * 3), ("g", ctypes.c_double * 3), ("dt", ctypes.c_double),
                ("skin", ctypes.c_double), ("r_max", ctypes.c_double), ("E", ctypes.c_double),
                ("nu", ctypes.c_double), ("e", ctypes.c_double), ("mu", ctypes.c_double),
                ("mu_wall", ctypes.c_double), ("rho", ctypes.c_double), ("clamp_fn", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int32), ("max_neighbors", ctypes.c_int32),
                ("inst", ctypes.POINTER(InstanceDesc))]


class InstanceInfo(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("ncell", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32), ("n", ctypes.c_int64),
                ("capacity", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rebuilds", ctypes.c_int64), ("list_entries", ctypes.c_int64),
                ("contacts", ctypes.c_int64), ("particles", ctypes.c_int64), ("wall_contacts", ctypes.c_int64),
                ("step_threads", ctypes.c_int32), ("step_lanes", ctypes.c_int32), ("graph_fused", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class CouplingSpec(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("feed_faces", ctypes.c_int32),
                ("drain_faces", ctypes.c_int32), ("surface_cell", ctypes.c_double), ("layer", ctypes.c_double),
                ("corr_cell", ctypes.c_double), ("interval", ctypes.c_int32), ("bins", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("kp", ctypes.c_double), ("ki", ctypes.c_double), ("kv", ctypes.c_double),
                ("mode", ctypes.c_int32), ("max_attempts", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("mass_unit", ctypes.c_double), ("max_insert", ctypes.c_int32), ("add_forces", ctypes.c_int32),
                ("velocity_below", ctypes.c_double), ("velocity_below_on", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


# coupler fields (dem_coupler_field)
CPL_SURFACE_MASS, CPL_SURFACE_CARRY, CPL_SURFACE_INSERTED, CPL_SURFACE_VEL, CPL_SURFACE_HIST, CPL_LAYER_STRESS, \
    CPL_LAYER_PHI, CPL_LAYER_VEL, CPL_LAYER_VMAX, CPL_LAYER_CTRL, CPL_CORR_PHI, CPL_CORR_VEL, CPL_SIZES = range(13)

_lib = None


def lib_path() -> str:
    """libcgdem.so, or with CGDEM_CHECKED=1 in the environment its bounds-checked build (the
    step kernel's gathered indices and the list build's cell codes tested in the kernels; an
    index out of range is reported as DEM_ERR_BOUNDS)."""
    return LIB_CHECKED if os.environ.get("CGDEM_CHECKED", "0") not in ("", "0") else LIB


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "dem_query_workspace": [ctypes.POINTER(Config), ctypes.POINTER(i64)],
        "dem_create": [ctypes.POINTER(Config), vp, i64, vp, ctypes.POINTER(vp)],
        "dem_destroy": [vp],
        "dem_write": [vp, i32, vp, i64],
        "dem_read": [vp, i32, vp, i64],
        "dem_read_contacts": [vp, vp, vp, i32, i64],
        "dem_write_contacts": [vp, vp, vp, i32, i64],
        "dem_read_neighbors": [vp, vp, i32, i64],
        "dem_step": [vp, i64],
        "dem_sync_status": [vp],
        "dem_instance_info_get": [vp, i32, ctypes.POINTER(InstanceInfo)],
        "dem_stats": [vp, ctypes.POINTER(Stats)],
        "dem_set_graph": [vp, i32],
        "dem_set_step_block": [vp, i32],
        "dem_set_step_lanes": [vp, i32],
        "dem_set_graph_mode": [vp, i32],
        "dem_test_stall_barrier": [vp],
        "dem_set_list_build": [vp, i32],
        "dem_graph_step_kernel_ms": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)],
        "dem_rollout_workspace": [vp, i64, i64, ctypes.POINTER(i64)],
        "dem_rollout_forward": [vp, i64, i64, vp, i64],
        "dem_rollout_adjoint": [vp, vp, vp, vp],
        "dem_observables": [vp, vp, vp],
        "dem_set_material": [vp, vp],
        "dem_coupler_workspace": [vp, vp, ctypes.POINTER(CouplingSpec), ctypes.POINTER(i64)],
        "dem_coupler_create": [vp, vp, ctypes.POINTER(CouplingSpec), vp, i64, ctypes.POINTER(vp)],
        "dem_couple": [vp],
        "dem_coupler_read": [vp, i32, vp, i64],
        "dem_coupler_destroy": [vp],
        "dem_counts": [vp, vp, vp],
        "dem_clear_external_force": [vp],
        "dem_grid_fields": [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.POINTER(i32), vp, i64],
        "dem_set_walls": [vp, i32, ctypes.POINTER(ctypes.c_double), i32, ctypes.POINTER(ctypes.c_double),
                          ctypes.c_double],
        "dem_wall_removed": [vp, i32, ctypes.POINTER(ctypes.c_double)],
        "dem_neighbor_counts_noalloc": [vp, vp, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(i32), ctypes.c_double, ctypes.c_double, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.dem_last_error.argtypes = [vp]
    L.dem_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def exported_symbols():
    return ["dem_query_workspace", "dem_create", "dem_destroy", "dem_write", "dem_read", "dem_read_contacts", "dem_read_neighbors",
            "dem_write_contacts", "dem_step", "dem_sync_status", "dem_instance_info_get", "dem_stats",
            "dem_set_graph", "dem_set_step_block", "dem_set_step_lanes", "dem_set_graph_mode", "dem_test_stall_barrier", "dem_set_list_build", "dem_graph_step_kernel_ms", "dem_neighbor_counts_noalloc", "dem_rollout_workspace",
            "dem_rollout_forward", "dem_rollout_adjoint", "dem_observables", "dem_set_material",
            "dem_coupler_workspace", "dem_coupler_create", "dem_couple", "dem_coupler_read", "dem_coupler_destroy",
            "dem_counts", "dem_clear_external_force", "dem_grid_fields", "dem_set_walls", "dem_wall_removed",
            "dem_last_error"]


def desc(*, n, lo, hi, periodic, dt, skin, r_max, E, nu, e, mu, rho, g=(0, 0, 0), floor=True,
         floor_v=(0, 0, 0), mu_wall=None, capacity=None, clamp_fn=False) -> InstanceDesc:
    d = InstanceDesc()
    d.n = int(n)
    d.capacity = int(capacity if capacity is not None else max(1, n))
    for a in range(3):
        d.lo[a], d.hi[a] = float(lo[a]), float(hi[a])
        d.periodic[a] = 1 if periodic[a] else 0
        d.floor_v[a] = float(floor_v[a])
        d.g[a] = float(g[a])
    d.floor_on = 1 if floor else 0
    d.dt, d.skin, d.r_max = float(dt), float(skin), float(r_max)
    d.E, d.nu, d.e, d.mu = float(E), float(nu), float(e), float(mu)
    d.mu_wall = -1.0 if mu_wall is None else float(mu_wall)
    d.rho = float(rho)
    d.clamp_fn = 1 if clamp_fn else 0
    return d


def desc_from_workload(wl, capacity=None, r_max=None) -> InstanceDesc:
    m = wl.material
    return desc(n=wl.n, lo=wl.lo, hi=wl.hi, periodic=wl.periodic, dt=wl.dt, skin=wl.skin,
                r_max=r_max if r_max is not None else float(np.max(wl.r)) if wl.n else 1e-3,
                E=m.E, nu=m.nu, e=m.e, mu=m.mu, rho=m.rho, g=wl.g, floor=wl.floor, floor_v=wl.floor_v,
                mu_wall=m.mu_wall, capacity=capacity)


class DEM:
    """A context of one or more DEM instances on the current CUDA device."""

    def __init__(self, descs, max_neighbors=32, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("DEM needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.L = lib()
        self.device = torch.device(device or "cuda")
        if isinstance(descs, InstanceDesc):
            descs = [descs]
        self._descs = (InstanceDesc * len(descs))(*descs)
        self.cfg = Config(len(descs), int(max_neighbors), self._descs)
        nbytes = ctypes.c_int64()
        self._check(self.L.dem_query_workspace(ctypes.byref(self.cfg), ctypes.byref(nbytes)), "query workspace")
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            self.stream = stream or torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        self._check(self.L.dem_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                      self.workspace_bytes, ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(h)), "create")
        self.h = h
        self.counts_ = [int(d.n) for d in descs]
        self._count_stale = False                     # a coupling call changed the counts on the device
        self.dts = [float(d.dt) for d in descs]       # time step of each instance [s]

    # ------------------------------------------------------------------
    def _check(self, rc, what):
        if rc != 0:
            msg = self.L.dem_last_error(getattr(self, "h", None)).decode()
            raise DemError(rc, f"{what}: {msg}")

    @property
    def n(self):
        if self._count_stale:                         # refreshed only when needed (synchronises)
            self._count_stale = False
            self.counts_ = [int(self.info(k)["n"]) for k in range(len(self.counts_))]
        return sum(self.counts_)

    def close(self):
        if getattr(self, "h", None):
            self.L.dem_destroy(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():      # the CUDA runtime may already be torn down
            return
        try:
            self.close()
        except Exception:
            pass

    def _as_f64(self, a, width):
        torch = self.torch
        if isinstance(a, torch.Tensor):
            t = a.to(dtype=torch.float64).contiguous()
        else:
            t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64)))
        if t.numel() != self.n * width:
            raise ValueError(f"expected {self.n * width} values, got {t.numel()}")
        return t

    def write(self, field, values):
        t = self._as_f64(values, _WIDTH[field])
        self._check(self.L.dem_write(self.h, field, ctypes.c_void_p(t.data_ptr()), self.n), "write")
        self._keep = t  # device-side source must outlive the asynchronous copy kernel
        return self

    def write_state(self, x, v, w, r, m=None):
        self.write(POS, x).write(VEL, v).write(OMEGA, w).write(RADIUS, r)
        if m is not None:
            self.write(MASS, m)
        return self

    def read(self, field, out=None, host=True):
        """Read a field; returns a float64 numpy array (host) or CUDA tensor."""
        torch = self.torch
        shape = (self.n, 3) if _WIDTH[field] == 3 else (self.n,)
        if out is None:
            out = (torch.empty(shape, dtype=torch.float64, device=self.device) if not host
                   else torch.empty(shape, dtype=torch.float64).pin_memory())
        self._check(self.L.dem_read(self.h, field, ctypes.c_void_p(out.data_ptr()), self.n), "read")
        return out.numpy() if host and out.device.type == "cpu" else out

    def read_contacts(self, width=16):
        torch = self.torch
        partner = torch.empty((self.n, width), dtype=torch.int32, device=self.device)
        xi = torch.empty((self.n, width, 3), dtype=torch.float64, device=self.device)
        self._check(self.L.dem_read_contacts(self.h, ctypes.c_void_p(partner.data_ptr()),
                                             ctypes.c_void_p(xi.data_ptr()), width, self.n), "read contacts")
        self.sync()
        return partner.cpu().numpy(), xi.cpu().numpy()

    def read_neighbors(self, width=32):
        """(n, width) int32 partner IDs of every neighbour-list entry, ascending, -1 padded."""
        torch = self.torch
        partner = torch.empty((self.n, width), dtype=torch.int32, device=self.device)
        self._check(self.L.dem_read_neighbors(self.h, ctypes.c_void_p(partner.data_ptr()), width, self.n),
                    "read neighbors")
        self.sync()
        return partner.cpu().numpy()

    def write_contacts(self, partner, xi):
        torch = self.torch
        p = torch.as_tensor(np.ascontiguousarray(partner, dtype=np.int32)).to(self.device)
        x = torch.as_tensor(np.ascontiguousarray(xi, dtype=np.float64)).to(self.device)
        width = p.shape[1]
        self._check(self.L.dem_write_contacts(self.h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                              width, self.n), "write contacts")
        self.sync()
        return self

    def step(self, nsteps=1):
        self._check(self.L.dem_step(self.h, int(nsteps)), "step")
        return self

    def sync(self):
        self._check(self.L.dem_sync_status(self.h), "sync")
        return self

    def status(self):
        return self.L.dem_sync_status(self.h)

    def set_graph(self, steps_per_graph):
        self._check(self.L.dem_set_graph(self.h, int(steps_per_graph)), "set graph")
        return self

    def set_step_block(self, threads):
        """Threads per block of the step kernel: 0 (automatic, the default), 64, 128, 256 or 896
        (one block per SM; single-instance contexts)."""
        self._check(self.L.dem_set_step_block(self.h, int(threads)), "set step block")
        return self

    def set_step_lanes(self, lanes):
        """Lanes per particle of the step kernel: 1 (default), 2, 4 or 8 (more than one at the
        128-thread block), or 0 to choose by size; for systems too small to fill the GPU with one
        thread per particle."""
        self._check(self.L.dem_set_step_lanes(self.h, int(lanes)), "set step lanes")
        return self

    def set_graph_mode(self, mode):
        """How a captured graph runs its steps: 0 fused when the context fits (default), 1 one
        kernel per step, 2 fused (one cooperative launch between list builds)."""
        self._check(self.L.dem_set_graph_mode(self.h, int(mode)), "set graph mode")
        return self

    def set_list_build(self, staged):
        """Neighbour-list build: 0 direct scan of the 27 cells (default), 1 staged in shared memory."""
        self._check(self.L.dem_set_list_build(self.h, int(staged)), "set list build")
        return self

    def test_stall_barrier(self):
        """Make the next fused launch's barrier wait run out (tests of DEM_ERR_TIMEOUT)."""
        self._check(self.L.dem_test_stall_barrier(self.h), "test stall barrier")
        return self

    def graph_step_kernel_ms(self):
        """(sum of step-kernel CUDA-event times in the last graph launch [ms], number of step kernels)."""
        t, c = ctypes.c_double(), ctypes.c_int32()
        self._check(self.L.dem_graph_step_kernel_ms(self.h, ctypes.byref(t), ctypes.byref(c)), "kernel times")
        return t.value, c.value

    # ---- differentiable rollouts -------------------------------------------------
    @staticmethod
    def _host(a, shape):
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))
        return arr, ctypes.c_void_p(arr.ctypes.data)

    def set_material(self, params):
        """params (B, 3) = {E, e, mu} per instance."""
        arr, ptr = self._host(params, (len(self.counts_), 3))
        self._check(self.L.dem_set_material(self.h, ptr), "set material")
        return self

    def rollout_forward(self, nsteps, checkpoint_every):
        torch = self.torch
        nb = ctypes.c_int64()
        self._check(self.L.dem_rollout_workspace(self.h, int(nsteps), int(checkpoint_every), ctypes.byref(nb)),
                    "rollout workspace")
        if getattr(self, "_ro_ws", None) is None or self._ro_ws.numel() < nb.value:
            self._ro_ws = None
            self._ro_ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        self._check(self.L.dem_rollout_forward(self.h, int(nsteps), int(checkpoint_every),
                                               ctypes.c_void_p(self._ro_ws.data_ptr()), int(self._ro_ws.numel())),
                    "rollout forward")
        return self

    def observables(self, axis):
        """(B, 2) = {kinetic energy, runout} at the current step; axis (B, 2) [m]."""
        B = len(self.counts_)
        ax, axp = self._host(axis, (B, 2))
        out = np.zeros((B, 2))
        self._check(self.L.dem_observables(self.h, axp, ctypes.c_void_p(out.ctypes.data)), "observables")
        return out

    def rollout_adjoint(self, weights, axis):
        """(B, 3) gradient of sum_k w_KE KE_k + w_R runout_k w.r.t. {E, e, mu} per instance."""
        B = len(self.counts_)
        w, wp = self._host(weights, (B, 2))
        ax, axp = self._host(axis, (B, 2))
        grad = np.zeros((B, 3))
        self._check(self.L.dem_rollout_adjoint(self.h, wp, axp, ctypes.c_void_p(grad.ctypes.data)), "rollout adjoint")
        return grad

    def counts(self):
        """(live, ids) per instance; refreshes the binding's idea of the particle count."""
        B = len(self.counts_)
        live = np.zeros(B, dtype=np.int64)
        ids = np.zeros(B, dtype=np.int64)
        self._check(self.L.dem_counts(self.h, ctypes.c_void_p(live.ctypes.data), ctypes.c_void_p(ids.ctypes.data)),
                    "counts")
        self.counts_ = [int(x) for x in ids]
        return live, ids

    def grid_fields(self, lo, h, n, k=0):
        """(n2, n1, n0, 5) CUDA tensor: solid volume fraction, mass, Favre velocity per cell."""
        torch = self.torch
        n = [int(v) for v in n]
        out = torch.empty((n[2], n[1], n[0], 5), dtype=torch.float64, device=self.device)
        lo3 = (ctypes.c_double * 3)(*[float(v) for v in lo])
        n3 = (ctypes.c_int32 * 3)(*n)
        self._check(self.L.dem_grid_fields(self.h, int(k), lo3, float(h), n3, ctypes.c_void_p(out.data_ptr()),
                                           out.numel()), "grid fields")
        return out

    def clear_external_force(self):
        self._check(self.L.dem_clear_external_force(self.h), "clear external force")
        return self

    def info(self, k=0):
        inf = InstanceInfo()
        self._check(self.L.dem_instance_info_get(self.h, k, ctypes.byref(inf)), "info")
        return dict(q=inf.q, lo=tuple(inf.lo), hi=tuple(inf.hi), ncell=tuple(inf.ncell), n=inf.n,
                    capacity=inf.capacity)

    def set_walls(self, k=0, axis=(0.0, 0.0), points=(), z_remove=-math.inf):
        """Axisymmetric walls of instance k: the surface of revolution of the polyline
        points [(rho, z), ...] about the vertical axis through `axis`; particles whose centre
        falls below z_remove are removed (see dem_set_walls)."""
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 2))
        ax = (ctypes.c_double * 2)(*[float(a) for a in axis])
        pp = pts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if len(pts) else None
        self._check(self.L.dem_set_walls(self.h, int(k), ax, int(len(pts)), pp, float(z_remove)), "set walls")
        return self

    def wall_removed(self, k=0):
        """(count, mass [kg]) removed below the removal height of instance k so far."""
        out = (ctypes.c_double * 2)()
        self._check(self.L.dem_wall_removed(self.h, int(k), out), "wall removed")
        return int(out[0]), float(out[1])

    def stats(self):
        st = Stats()
        self._check(self.L.dem_stats(self.h, ctypes.byref(st)), "stats")
        return dict(steps=st.steps, rebuilds=st.rebuilds, list_entries=st.list_entries, contacts=st.contacts,
                    particles=st.particles, wall_contacts=st.wall_contacts, step_threads=st.step_threads,
                    step_lanes=st.step_lanes, graph_fused=st.graph_fused)


def neighbor_counts_noalloc(x, r, lo, hi, periodic, skin, r_max, out=None, stream=None):
    """Neighbour counts through the allocation-free entry point (see include/dem.h).

    x (n,3) and r (n,) are float64 CUDA tensors; the result is an int32 CUDA tensor
    (the caller's `out` if given).  The library allocates nothing for this call.
    """
    import torch
    L = lib()
    n = int(r.shape[0])
    if out is None:
        out = torch.empty((n,), dtype=torch.int32, device=r.device)
    st = stream or torch.cuda.current_stream(r.device)
    lo3 = (ctypes.c_double * 3)(*[float(v) for v in lo])
    hi3 = (ctypes.c_double * 3)(*[float(v) for v in hi])
    per3 = (ctypes.c_int32 * 3)(*[1 if p else 0 for p in periodic])
    rc = L.dem_neighbor_counts_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(r.data_ptr()), n, lo3, hi3,
                                       per3, float(skin), float(r_max), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise DemError(rc, L.dem_last_error(None).decode())
    return out


class Coupler:
    """Two-way coupling of a coarse and a fine single-instance context (dem_coupler_*)."""

    def __init__(self, coarse, fine, **spec):
        import torch
        self.L = lib()
        self.coarse, self.fine = coarse, fine
        sp = CouplingSpec()
        for a in range(3):
            sp.lo[a], sp.hi[a] = float(spec["lo"][a]), float(spec["hi"][a])
        for k in ("feed_faces", "drain_faces", "interval", "bins", "mode", "max_attempts", "max_insert", "add_forces"):
            setattr(sp, k, int(spec.get(k, 0)))
        for k in ("surface_cell", "layer", "corr_cell", "alpha", "kp", "ki", "kv", "mass_unit"):
            setattr(sp, k, float(spec[k]))
        sp.seed = int(spec.get("seed", 0))
        vb = spec.get("velocity_below", None)
        if vb is not None and not math.isnan(float(vb)) and float(vb) > -math.inf:
            sp.velocity_below, sp.velocity_below_on = float(vb), 1
        self.spec = sp
        nb = ctypes.c_int64()
        rc = self.L.dem_coupler_workspace(coarse.h, fine.h, ctypes.byref(sp), ctypes.byref(nb))
        if rc:
            raise DemError(rc, self.L.dem_last_error(None).decode())
        self.ws = torch.empty(int(nb.value), dtype=torch.uint8, device=fine.device)
        h = ctypes.c_void_p()
        rc = self.L.dem_coupler_create(coarse.h, fine.h, ctypes.byref(sp), ctypes.c_void_p(self.ws.data_ptr()),
                                       int(nb.value), ctypes.byref(h))
        if rc:
            raise DemError(rc, self.L.dem_last_error(None).decode())
        self.h = h
        sz = self.read(CPL_SIZES)
        self.S, self.C = int(sz[0]), int(sz[2])

    def couple(self):
        rc = self.L.dem_couple(self.h)
        if rc:
            raise DemError(rc, self.L.dem_last_error(self.fine.h).decode())
        # the IDs handed out changed on the device; the host copy is refreshed when next needed
        self.fine._count_stale = True
        return self

    def read(self, field):
        S, C = getattr(self, "S", 0), getattr(self, "C", 0)
        bins = self.spec.bins
        shapes = {CPL_SIZES: (4,), CPL_SURFACE_MASS: (S,), CPL_SURFACE_CARRY: (S,), CPL_SURFACE_INSERTED: (S,),
                  CPL_SURFACE_VEL: (S, 3), CPL_SURFACE_HIST: (S, bins), CPL_LAYER_STRESS: (S, 2, 6),
                  CPL_LAYER_PHI: (S, 2), CPL_LAYER_VEL: (S, 2, 3), CPL_LAYER_VMAX: (S, 2), CPL_LAYER_CTRL: (S, 3),
                  CPL_CORR_PHI: (C, 2), CPL_CORR_VEL: (C, 2, 3)}
        out = np.zeros(shapes[field])
        rc = self.L.dem_coupler_read(self.h, field, ctypes.c_void_p(out.ctypes.data), out.size)
        if rc:
            raise DemError(rc, self.L.dem_last_error(self.fine.h).decode())
        return out

    def close(self):
        if getattr(self, "h", None):
            self.L.dem_coupler_destroy(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def from_workload(wl, max_neighbors=32, capacity=None, **kw) -> DEM:
    """A single-instance context loaded with a workload's state."""
    d = DEM([desc_from_workload(wl, capacity=capacity)], max_neighbors=max_neighbors, **kw)
    d.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
    return d
