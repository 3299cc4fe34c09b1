"""Throughput of the DEM hot path on GB300: particle-steps/s at 1,000,000 particles.

Workload (plain, single instance): 1,000,000 polydisperse spheres, d ~ U[1.6, 2.4] mm,
E = 1e7 Pa, nu = 0.25, e = 0.9, mu = 0.5, rho = 2500 kg/m^3, in a 0.2 x 0.2 x 0.6 m box
periodic in x/y with a floor; dt = 1e-6 s, skin 0.1 d.  The bed starts on an FCC
lattice, settles under gravity for --settle steps (not timed), then the floor is
sheared at 0.5 m/s and --steps steps are timed.  One bench step = one DEM time step
of the whole hot path (neighbour-list rebuild when due, contact forces, integration).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs its own replica (the plain system is one problem;
replicas only), and the value is the particle-steps of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/sec and HBM GB/s fraction at 1M particles; batched & adjoint vs plain"
UNIT = "particle-steps/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--settle", type=int, default=30_000, help="settling steps at dt 5e-6, e 0.5 (not timed)")
    ap.add_argument("--graph", type=int, default=50, help="largest number of steps per captured CUDA graph (the "
                    "graph length is the largest divisor of --steps up to this; 0: direct launches)")
    ap.add_argument("--run-in", type=int, default=2000, help="untimed steps of the sheared bed before the warm-up "
                    "(part of the workload: the shear flow develops and the lists are rebuilt several times)")
    ap.add_argument("--repeats", type=int, default=5, help="timed repeats of --steps steps (median reported)")
    ap.add_argument("--settle-graph", type=int, default=50, help="steps per graph while settling")
    ap.add_argument("--lmax", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the reference arm's sample")
    ap.add_argument("--cpu-bed-steps", type=int, default=10, help="oracle steps on the settled bed (CPU baseline)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--adjoint-instances", type=int, default=64)
    ap.add_argument("--batched-steps", type=int, default=2000)
    ap.add_argument("--batched-scale", type=float, default=1.0, help="scale of the 256 box sizes (1 = as stated)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batched-settle", type=int, default=8000, help="settling steps before the settled batched "
                    "measurement (0: skip it)")
    ap.add_argument("--no-coupled", action="store_true")
    ap.add_argument("--no-nested", action="store_true")
    ap.add_argument("--silo", action="store_true", help="add the silo discharge validation (alpha 1 and 2, ~70 s)")
    ap.add_argument("--nested-periods", type=int, default=60, help="timed coupling periods of the five-level line")
    ap.add_argument("--profile-range", default="plain", choices=["plain", "batched", "adjoint", "coupled"],
                    help="which line's timed region `ncu --profile-from-start off` sees")
    ap.add_argument("--coupled-intervals", type=int, default=100, help="timed coupling intervals of 15 steps")
    ap.add_argument("--coupled-settle", type=int, default=4000, help="settling steps per level (dt 5e-6)")
    ap.add_argument("--save-state", default=None, help="save the settled bed (.npz) for later --load-state runs")
    ap.add_argument("--load-state", default=None, help="start from a saved settled bed instead of settling")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _profile(args, line, start):
    """Start or stop the profiler range (cudaProfilerStart/Stop) around one line's timed region."""
    if args.profile_range != line:
        return
    import torch
    if start:
        torch.cuda.profiler.start()
    else:
        torch.cuda.profiler.stop()


def max_over_ranks(x, device):
    """The largest of a per-rank float over all ranks (the time of the slowest replica)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks (weak scaling: each rank its own replica) per second of the slowest."""
    return units_per_rank * world / seconds


def _profile_traffic(kernel_src_hash):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "k_step_shear_bed.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch_at_1M:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_src_hash:
        return None
    return float(m.group(1))


def graph_length(steps, cap):
    """Steps per captured graph: the largest divisor of `steps` up to `cap`, so that a timed run of
    exactly `steps` steps is whole graphs (0: direct launches)."""
    if cap <= 0:
        return 0
    return max(d for d in range(1, min(cap, steps) + 1) if steps % d == 0)


def _kernel_hash():
    """Hash of the step kernel's source (its definition in dem.cu and the headers it is built
    from); a profile taken from another version gives no traffic."""
    csrc = os.path.join(ROOT, "paper_1705_03850_gb300", "csrc")
    src = open(os.path.join(csrc, "dem.cu")).read()
    # from the block-size helper before the step pass to the end of the per-step kernel (the
    # fused kernel after it is not part of the timed launch)
    i0 = src.index("constexpr int step_minb()")
    i0 = src.rindex("template", 0, i0)
    m = re.search(r"__global__ void __launch_bounds__\(.*\) k_step\(", src[i0:])   # the kernel is in range
    i1 = src.index("\n}\n", i0 + m.end()) + 3
    h = hashlib.sha256(src[i0:i1].encode())
    h.update(re.search(r"#define DEM_STEP_MINB \d+", src).group(0).encode())   # its launch bound
    for f in ("dem_internal.cuh", "dem_contact.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# --------------------------------------------------------------- CPU oracle

def _oracle_timed(sim, steps):
    sim.run(0)                           # start-up evaluation (not timed)
    t0 = time.perf_counter()
    sim.run(steps)
    return time.perf_counter() - t0


def cpu_oracle_baseline(bed, bed_steps):
    """The FP64 oracle as it stands, timed on this host's cores: the 1,000-sphere column in full
    (5,000 steps) and `bed_steps` steps of the GPU line's own settled and sheared 1M bed (its
    state read back from the device, empty contact history), each on one thread and with the
    OpenMP build on every core (the per-pair contact law in parallel; identical results)."""
    import oracle
    from paper_1705_03850_gb300 import workloads
    cores = os.cpu_count() or 1
    runs = []
    col = workloads.column()
    m = col.material
    Pc = oracle.make_params(E=m.E, nu=m.nu, e=m.e, mu=m.mu, dt=col.dt, g=col.g, lo=col.lo, hi=col.hi,
                            periodic=col.periodic, floor=col.floor, floor_v=col.floor_v)
    x, v, w, r, mass, P = bed
    for threads, omp in ((1, False), (cores, True)):
        os.environ["OMP_NUM_THREADS"] = str(threads)
        t = _oracle_timed(oracle.Sim(Pc, col.x, col.v, col.w, col.r, col.m, openmp=omp), 5000)
        runs.append({"workload": "1,000-sphere column (d = 2 mm, 20 x 20 x 60 mm), 5,000 steps of 2e-6 s",
                     "threads": threads, "seconds": t, "value": col.n * 5000 / t})
        t = _oracle_timed(oracle.Sim(P, x, v, w, r, mass, openmp=omp), bed_steps)
        runs.append({"workload": f"the settled, sheared 1M bed of the GPU line, {bed_steps} steps of 1e-6 s",
                     "threads": threads, "seconds": t, "value": len(r) * bed_steps / t})
    head = runs[3]
    return {"value": head["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle (OpenMP build, {cores} threads) for {bed_steps} steps of the GPU line's own "
                      f"settled 1M bed ({head['seconds']:.1f} s); all runs below",
            "runs": runs, "host": os.uname().machine, "nproc": cores}


def _oracle_block(nx, ny, nz):
    import oracle
    from paper_1705_03850_gb300 import workloads
    wl = workloads.dense_block(nx, ny, nz, seed=2, rjit=0.2, vel=0.05, spin=5.0)
    m = wl.material
    P = oracle.make_params(E=m.E, nu=m.nu, e=m.e, mu=m.mu, dt=wl.dt, g=wl.g, lo=wl.lo, hi=wl.hi,
                           periodic=wl.periodic, floor=wl.floor, floor_v=wl.floor_v)
    return wl, oracle.Sim(P, wl.x, wl.v, wl.w, wl.r, wl.m, openmp=True)


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host, W untimed and K timed steps of
    a dense polydisperse block (the stand-in for the settled 1M bed, which a CPU cannot settle),
    its size chosen so that the K timed steps take about two minutes at most."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    K, W = max(1, args.steps), max(0, args.warmup)
    cores = os.cpu_count() or 1
    os.environ["OMP_NUM_THREADS"] = str(cores)
    wl, sim = _oracle_block(20, 20, 20)            # calibration: 8,000 particles
    sim.run(0)
    t0 = time.perf_counter()
    sim.run(3)
    rate = wl.n * 3 / (time.perf_counter() - t0)
    n_target = rate * min(120.0, max(10.0, args.cpu_seconds * 8)) / K
    side = int(max(8, min(60, round((n_target / 0.667) ** (1.0 / 3.0)))))
    wl, sim = _oracle_block(side, side, max(4, int(round(side * 0.667))))
    sim.run(0)
    sim.run(W)
    t0 = time.perf_counter()
    sim.run(K)
    t = time.perf_counter() - t0
    value = wl.n * K / t
    sample = (f"FP64 C oracle (OpenMP build, {cores} threads), {W} untimed + {K} timed steps of a {wl.n}-particle "
              f"dense polydisperse block (d in [1.6, 2.4] mm, overlapping jittered lattice, cell-list contacts; a "
              f"host cannot settle the 1M bed in a bench run), {t:.1f} s")
    cpu = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
           "host": os.uname().machine, "nproc": os.cpu_count()}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": t / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"shear_bed stand-in: {wl.n:,}-particle dense polydisperse block "
                                   "(oracle sample; ms_per_step is per step of that sample)",
                       "n_particles": wl.n},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- GPU

def run_ours(args):
    import numpy as np
    import torch

    from paper_1705_03850_gb300 import dem, workloads

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    K = max(1, args.steps)
    W = max(3, args.warmup)
    S = graph_length(K, args.graph)

    # ---- build and settle the bed (not timed): larger step and more damping
    # than the sheared run, so that the lattice collapses into a dense bed quickly
    wl = workloads.shear_bed(args.n, seed=2)
    desc = dem.desc_from_workload(wl, r_max=1.2e-3)
    if args.load_state:
        z = np.load(args.load_state)
        x, v, w, r, m = (torch.from_numpy(z[k]).to(dev) for k in ("x", "v", "w", "r", "m"))
        if x.shape[0] != wl.n:
            raise SystemExit(f"{args.load_state} holds {x.shape[0]} particles, not {wl.n}")
    else:
        sdesc = dem.desc_from_workload(wl, r_max=1.2e-3)
        sdesc.dt, sdesc.e = 5e-6, 0.5
        settle = dem.DEM([sdesc], max_neighbors=args.lmax, device=dev)
        settle.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
        settle.step(1)
        if args.settle_graph > 0:
            settle.set_graph(args.settle_graph)
        settle.step(max(0, args.settle - 1))
        settle.sync()
        x = settle.read(dem.POS, host=False)
        v = settle.read(dem.VEL, host=False)
        w = settle.read(dem.OMEGA, host=False)
        r = settle.read(dem.RADIUS, host=False)
        m = settle.read(dem.MASS, host=False)
        settle.close()
        del settle
    if args.save_state and rank == 0:
        np.savez(args.save_state, x=x.cpu().numpy(), v=v.cpu().numpy(), w=w.cpu().numpy(), r=r.cpu().numpy(),
                 m=m.cpu().numpy())

    # ---- sheared bed: floor moves at 0.5 m/s in x; the run-in (untimed, part of the workload)
    # lets the shear flow develop through several list rebuilds, then W warm-up steps
    desc.floor_v[0] = 0.5
    sim = dem.DEM([desc], max_neighbors=args.lmax, device=dev)
    sim.write_state(x, v, w, r, m)
    sim.step(1)
    if S > 0:
        sim.set_graph(S)
    sim.step(max(0, args.run_in - 1))
    sim.step(W)
    sim.sync()
    st0 = sim.stats()

    # ---- timed: `repeats` x exactly K steps (inputs larger than L2), median reported
    reps = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        for rep in range(max(1, args.repeats)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize(dev)
            if rep == 0:
                _profile(args, "plain", True)    # marks the timed region for `ncu --profile-from-start off`
            e0.record(stream)
            sim.step(K)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if rep == 0:
                _profile(args, "plain", False)
            kms, kn = sim.graph_step_kernel_ms() if S > 0 else (float("nan"), 1)
            reps.append((max_over_ranks(e0.elapsed_time(e1), dev), kms / max(1, kn), kn))
    st1 = sim.stats()
    sim.sync()
    order = sorted(range(len(reps)), key=lambda i: reps[i][0])
    ms = reps[order[len(order) // 2]][0]
    kern_sorted = sorted(t for _, t, _ in reps)
    t_kernel_ms = kern_sorted[len(kern_sorted) // 2]
    n = wl.n
    value = whole_job_rate(n * K, world, ms / 1e3)
    L = st1["list_entries"] / max(1, st1["particles"])
    C = st1["contacts"] / max(1, st1["particles"])
    Wc = st1["wall_contacts"] / max(1, st1["particles"])
    rebuilds = st1["rebuilds"] - st0["rebuilds"]
    # algorithmic bytes per particle-step of the step kernel:
    # 48 B own state read + 48 B written, per list entry 4 B index + 12 B history read + 12 B written
    B_step = 96.0 + 28.0 * L
    # what this design must move at least: the same state, count and history mask,
    # indices of every entry, history only of entries in contact, floor history
    B_design = 96.0 + 4.0 + 8.0 + 4.0 * L + 24.0 * (C - Wc) + 32.0 * Wc
    t_kernel = t_kernel_ms / 1e3
    achieved = n * B_step / t_kernel / 1e9
    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    traffic = _profile_traffic(_kernel_hash())
    # per graph of S steps: one condition-setting kernel and S step kernels, plus the
    # 11-kernel rebuild chain when a rebuild runs; direct launches run the chain every step
    # (per timed repeat of K steps; rebuilds averaged over the repeats)
    nrep = max(1, args.repeats)
    launches = round(K + K // S + 11 * rebuilds / nrep) if S > 0 else 12 * K

    # the bed as it stands after the timed region (host copies, for the CPU baseline)
    bed = tuple(sim.read(f) for f in (dem.POS, dem.VEL, dem.OMEGA, dem.RADIUS, dem.MASS)) if world == 1 else None

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hx = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        hv = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        hw = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        hr = torch.empty((n,), dtype=torch.float64).pin_memory()
        hm = torch.empty((n,), dtype=torch.float64).pin_memory()
        hx.copy_(x.cpu()); hv.copy_(v.cpu()); hw.copy_(w.cpu()); hr.copy_(r.cpu()); hm.copy_(m.cpu())
        ox = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        ov = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        ow = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sim.write_state(hx, hv, hw, hr, hm)
        sim.step(K)
        sim.read(dem.POS, out=ox)
        sim.read(dem.VEL, out=ov)
        sim.read(dem.OMEGA, out=ow)
        torch.cuda.synchronize(dev)
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        h2d = (hx.numel() + hv.numel() + hw.numel() + hr.numel() + hm.numel()) * 8
        d2h = (ox.numel() + ov.numel() + ow.numel()) * 8
        e2e = {"value": whole_job_rate(n * K, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K, "chunk_steps": K,
               "what": "dem_write(POS,VEL,OMEGA,RADIUS,MASS) from pinned host, dem_step(K), "
                       "dem_read(POS,VEL,OMEGA) to pinned host; bytes per DEM step = chunk bytes / K"}

    # the batched, adjoint and coupled lines are single-GPU measurements (rank 0 alone reports;
    # under several ranks only the plain replicas are timed)
    single = world == 1
    batched = run_batched(args, dev, value) if single and not args.no_batched else None
    adj = run_adjoint(args, dev, value) if single and not args.no_adjoint else None
    coupled = run_coupled(args, dev, value) if single and not args.no_coupled else None
    nested = run_nested(args, dev, value) if single and not args.no_nested else None
    silo = None
    if single and args.silo:
        from paper_1705_03850_gb300 import silo as silo_mod
        silo = [silo_mod.run(a, device=dev) for a in (1, 2)]

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        import oracle
        mt = wl.material
        P_bed = oracle.make_params(E=mt.E, nu=mt.nu, e=mt.e, mu=mt.mu, dt=wl.dt, g=wl.g, lo=wl.lo, hi=wl.hi,
                                   periodic=wl.periodic, floor=wl.floor, floor_v=(0.5, 0.0, 0.0))
        cpu = cpu_oracle_baseline(bed + (P_bed,), args.cpu_bed_steps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"shear_bed: {n:,} polydisperse spheres, settled then floor-sheared",
                   "n_particles": n, "dt": wl.dt, "skin_m": wl.skin,
                   "settle_steps": 0 if args.load_state else args.settle,
                   "settle": (f"loaded from {os.path.basename(args.load_state)}" if args.load_state
                              else "dt 5e-6 s, e 0.5, from the FCC start"),
                   "run_in_steps": args.run_in, "steps_per_graph": S, "max_neighbors": args.lmax,
                   "repeats": len(reps), "ms_per_step_repeats": [t / K for t, _, _ in reps],
                   "ms_per_step_mean": sum(t for t, _, _ in reps) / (K * len(reps)),
                   "timing": f"CUDA events around each repeat of exactly {K} steps after {args.run_in} untimed "
                             f"run-in and {W} warm-up steps; value and ms_per_step from the median repeat",
                   "l2": "inputs larger than L2 (state + lists + histories > 129 MB)",
                   "mean_list_length": L, "mean_contacts_per_particle": C,
                   "rebuilds_in_timed_region": rebuilds, "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src, "kernel": f"k_step<0, false, {st1['step_threads']}> (fused force + Verlet, the variant without walls; "
                               f"{st1['step_threads']} threads per block)",
                     "bytes_per_particle_step": B_step, "kernel_ms_avg": t_kernel * 1e3,
                     "kernel_ms_repeats": [t for _, t, _ in reps],
                     "kernel_timing": "median over the repeats of the mean CUDA-event duration of every fifth "
                                      "step kernel of the repeat's last graph",
                     "design_bytes_per_particle_step": B_design,
                     "design_achieved": n * B_design / t_kernel / 1e9,
                     "kernel_share_of_step": t_kernel * 1e3 / (ms / K)},
        "clocks": clocks.summary(),
        "e2e": e2e,
        "batched": batched,
        "adjoint": adj,
        "coupled": coupled,
        "nested": nested,
        "silo": silo,
        "gpu_launches": launches,
        "cpu_baseline": cpu,
    }
    # the lines beside the plain step, repeated compactly at the end of the line
    g = lambda d, *ks: None if d is None else (g(d.get(ks[0]), *ks[1:]) if len(ks) > 1 else d.get(ks[0]))
    line["summary"] = {"plain": value, "roofline_frac": achieved / peak, "e2e": g(e2e, "value"),
                       "batched": g(batched, "value"), "batched_settled": g(batched, "settled", "value"),
                       "adjoint": g(adj, "value"), "coupled": g(coupled, "value"),
                       "coupled_multirate": g(coupled, "multirate", "value"), "nested": g(nested, "value"),
                       "cpu_oracle_all_cores": g(cpu, "value"), "unit": UNIT}
    print(json.dumps(line), flush=True)


def run_batched(args, dev, plain_value):
    """256 independent settling boxes advanced together (one persistent step launch per
    step, inside captured CUDA graphs); settings chosen by the autotuner first."""
    import torch

    from paper_1705_03850_gb300 import autotune, dem, workloads
    wls = workloads.batch(256, seed=4, scale=args.batched_scale, steps=args.batched_steps)
    state = [torch.as_tensor(a, dtype=torch.float64, device=dev) for a in autotune.concat_state(wls)]
    t0 = time.perf_counter()
    best, allc = autotune.tune(wls, window=args.batched_steps, sample=32, device=dev)
    t_tune = time.perf_counter() - t0
    sim = autotune.make_context(wls, best, device=dev, state=state)
    n = sum(w.n for w in wls)
    S = best.graph_steps
    K = max(S, (args.batched_steps // S) * S)
    st0 = sim.stats()
    sim.set_graph(S)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    _profile(args, "batched", True)
    e0.record(sim.stream)
    sim.step(1)               # start-up evaluation and first list build of all 256 boxes
    sim.step(K - 1 - ((K - 1) % S))
    sim.step((K - 1) % S)
    e1.record(sim.stream)
    torch.cuda.synchronize(dev)
    _profile(args, "batched", False)
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    sim.sync()
    sim.close()
    value = n * K / (ms / 1e3)
    settled = None if args.batched_settle <= 0 else _batched_settled(args, dev, wls)
    return {"value": value, "unit": UNIT, "workload": "256 settling boxes, N_k log-uniform in [2e3, 2e5] "
            "(seed 4), d = 2 mm, per-box E, e, mu", "n_instances": len(wls), "n_particles": n, "steps": K,
            "ms_per_step": ms / K, "vs_plain": value / plain_value, "rebuilds": st1["rebuilds"] - st0["rebuilds"],
            "mean_list_length": st1["list_entries"] / max(1, st1["particles"]),
            "mean_contacts_per_particle": st1["contacts"] / max(1, st1["particles"]),
            "timed": "all K steps from the lattice start, including the first list build (in 2 ms the lattice "
                     "barely moves: few contacts)",
            "tuned": best.as_dict(), "tuning_seconds": t_tune, "candidates": len(allc),
            "tuning": "each candidate timed on 32 of the boxes (spread over sizes) for the full step count",
            "settled": settled}


def _batched_settled(args, dev, wls):
    """The same 256 boxes after settling (dt 5e-6 s, e 0.5, not timed), retuned, then timed for the
    same number of steps at the stated dt: every particle in contact with its neighbours."""
    import torch

    from paper_1705_03850_gb300 import autotune, dem
    base = autotune.Choice(0.1, 1.0, 50, 32)
    descs = autotune.descs_for(wls, base)
    for dsc in descs:
        dsc.dt, dsc.e = 5e-6, 0.5
    st = dem.DEM(descs, max_neighbors=32, device=dev)
    st.write_state(*[torch.as_tensor(a, dtype=torch.float64, device=dev) for a in autotune.concat_state(wls)])
    st.step(1)
    st.set_graph(50)
    st.step(args.batched_settle - 1)
    st.sync()
    state = [st.read(f, host=False) for f in (dem.POS, dem.VEL, dem.OMEGA, dem.RADIUS, dem.MASS)]
    st.close()
    best, allc = autotune.tune(wls, window=args.batched_steps, sample=32, device=dev, state=state)
    sim = autotune.make_context(wls, best, device=dev, state=state)
    n = sum(w.n for w in wls)
    S = best.graph_steps
    K = max(S, (args.batched_steps // S) * S)
    sim.step(1)
    sim.set_graph(S)
    sim.step(S)
    torch.cuda.synchronize(dev)
    st0 = sim.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    sim.step(K)
    e1.record(sim.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    sim.close()
    return {"value": n * K / (ms / 1e3), "unit": UNIT, "steps": K, "ms_per_step": ms / K,
            "settle_steps": args.batched_settle, "rebuilds": st1["rebuilds"] - st0["rebuilds"],
            "mean_list_length": st1["list_entries"] / max(1, st1["particles"]),
            "mean_contacts_per_particle": st1["contacts"] / max(1, st1["particles"]), "tuned": best.as_dict()}


def run_adjoint(args, dev, plain_value):
    """64 granular columns of 10,000 spheres: 500-step forward with checkpoints every 50
    steps, then the adjoint gradients of final kinetic energy and runout with respect to
    (E, e, mu) of every column.  Throughput counts the forward and the backward pass."""
    import numpy as np
    import torch

    from paper_1705_03850_gb300 import dem, workloads
    B = args.adjoint_instances
    mats = workloads.column_materials(B, seed=5)
    wls = [workloads.column_collapse(10_000, seed=5 + k, mat=mats[k], steps=args.adjoint_steps) for k in range(B)]
    sim = dem.DEM([dem.desc_from_workload(w) for w in wls], max_neighbors=16, device=dev)
    cat = lambda f: np.concatenate([getattr(w, f) for w in wls])
    state = [torch.as_tensor(cat(f), dtype=torch.float64, device=dev) for f in ("x", "v", "w", "r", "m")]
    params = np.array([[m.E, m.e, m.mu] for m in mats])
    axis = np.array([w.meta["axis"] for w in wls])
    n = sum(w.n for w in wls)
    N, K = args.adjoint_steps, 50
    # plain forward of the same workload (graphs, lists rebuilt as needed), for comparison
    sim.set_material(params).write_state(*state)
    sim.step(1)
    sim.set_graph(50)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sim.step(N - 1)
    sim.sync()
    t_plain = time.perf_counter() - t0
    # differentiable rollout: forward with checkpoints + adjoint
    sim.set_material(params).write_state(*state)
    torch.cuda.synchronize(dev)
    _profile(args, "adjoint", True)
    t0 = time.perf_counter()
    sim.rollout_forward(N, K)
    t1 = time.perf_counter()
    obs = sim.observables(axis)
    grad = sim.rollout_adjoint(np.ones((B, 2)), axis)
    t2 = time.perf_counter()
    _profile(args, "adjoint", False)
    sim.close()
    value = n * N / (t2 - t0)
    return {"value": value, "unit": "adjoint particle-steps/s (forward with checkpoints + backward)",
            "workload": f"{B} granular columns x 10,000 spheres (d = 2 mm, 30 x 30 mm footprint), "
                        f"{N} steps at dt 5e-6 s, checkpoints every {K}",
            "n_particles": n, "steps": N, "seconds_forward": t1 - t0, "seconds_backward": t2 - t1,
            "plain_forward_particle_steps_per_s": n * (N - 1) / t_plain, "vs_plain_1M": value / plain_value,
            "gradient_example": {"dKE_dE": grad[0, 0], "dKE_de": grad[0, 1], "dKE_dmu": grad[0, 2]},
            "observables_example": {"KE": obs[0, 0], "runout": obs[0, 1]},
            "timing": "wall clock around the C-ABI calls (they synchronise)"}


def run_coupled(args, dev, plain_value):
    """Three nested coarse-graining levels of a 30-degree chute (8, 4 and 2 mm spheres; about
    2.0M + 1.0M + 2.0M), coupled pairwise every 15 steps (stress and velocity controllers,
    insertion, removal).  Each level first settles on its own under vertical gravity (not timed)."""
    import torch

    from paper_1705_03850_gb300 import dem, levels, workloads
    lv, specs = workloads.chute(u0=0.5)
    states = _settle_levels(args, dev, lv)
    single = _coupled_flow(args, dev, lv, specs, states, args.coupled_intervals, profile=True)
    # multi-rate: time steps scaled with the grain (4, 2, 1 x 1e-6 s), periods of 16 finest steps,
    # about the same physical time as the single-rate run
    lvm, specm = workloads.chute(u0=0.5, multirate=True, interval=16)
    periods = max(1, round(args.coupled_intervals * 15 / 16))
    multi = _coupled_flow(args, dev, lvm, specm, states, periods, profile=False)
    value = single["value"]
    line = dict(single)
    line.update({"value": value, "unit": UNIT, "metric": "particle-steps/s summed over the coupled levels",
                 "workload": "30-degree chute, 11 m periodic along the flow, 0.3 x 0.3 m section: level 0 d = 8 mm "
                             "everywhere, level 1 d = 4 mm in a 0.70 m region, level 2 d = 2 mm in a 0.18 m region "
                             "nested in it; plug flow 0.5 m/s at the start",
                 "vs_plain": value / plain_value, "settle_steps": args.coupled_settle,
                 "timing": "wall clock around the periods (no host wait inside; one stream per level); level "
                           "steps in CUDA graphs of one period; coupling_share from 20 more periods with the host "
                           "waiting around the coupling calls",
                 "multirate": dict(multi, speedup_in_simulated_time=single["wall_s_per_simulated_ms"] /
                                   multi["wall_s_per_simulated_ms"],
                                   what="dt 4e-6 / 2e-6 / 1e-6 s for the 8 / 4 / 2 mm levels (Sec. 3: the time "
                                        "step may scale with the grain), coupling every 16 us")})
    return line


def _settle_levels(args, dev, lv):
    """Each level settled on its own under vertical gravity (dt 5e-6 s, e 0.5; not timed)."""
    from paper_1705_03850_gb300 import dem
    states = []
    for wl in lv:
        sd = dem.desc_from_workload(wl)
        sd.dt, sd.e = 5e-6, 0.5
        sd.g[0], sd.g[1], sd.g[2] = 0.0, 0.0, -9.81
        st = dem.DEM([sd], max_neighbors=24, device=dev)
        st.write_state(wl.x, wl.v, wl.w, wl.r, wl.m)
        st.step(1)
        st.set_graph(50)
        st.step(max(0, args.coupled_settle - 1))
        st.sync()
        states.append([st.read(f, host=False) for f in (dem.POS, dem.VEL, dem.OMEGA, dem.RADIUS, dem.MASS)])
        st.close()
    return states


def run_nested(args, dev, plain_value):
    """Five nested levels (alpha = 16, 8, 4, 2, 1; d = 16 .. 1 mm; filled volume quartered per
    level, about 6.9M particles) of the 11 m chute, multi-rate, coupled every 16 us.  Beside the
    measured wall time per simulated millisecond: the same physical time for the whole chute at
    the finest resolution, estimated from the plain line's measured throughput."""
    from paper_1705_03850_gb300 import workloads
    lv, specs = workloads.nested_levels()
    states = _settle_levels(args, dev, lv)
    r = _coupled_flow(args, dev, lv, specs, states, args.nested_periods, profile=False)
    # the whole chute at 1 mm: the finest level's particle density times the full length
    n_full = lv[-1].n * (lv[0].hi[0] - lv[0].lo[0]) / (lv[-1].hi[0] - lv[-1].lo[0])
    est_full = n_full * (1e-3 / lv[-1].dt) / plain_value        # wall seconds per simulated ms
    r.update({"workload": "11 m chute, five levels d = 16, 8, 4, 2, 1 mm in nested regions of 11, 2.75, 0.69, "
                          "0.17, 0.043 m (cross-section kept), time steps 16, 8, 4, 2, 1 us",
              "unit": UNIT, "single_level_fine_particles_estimate": n_full,
              "single_level_fine_wall_s_per_simulated_ms_estimate": est_full,
              "speedup_estimate": est_full / r["wall_s_per_simulated_ms"],
              "estimate": "whole chute at d = 1 mm (finest level's density), stepped at the plain line's measured "
                          "particle-steps/s; an extrapolation, not a run"})
    return r


def _coupled_flow(args, dev, lv, specs, states, periods, profile):
    """Timed run of a level hierarchy from settled states: particle-steps/s and wall time per
    simulated millisecond."""
    import torch

    from paper_1705_03850_gb300 import dem, levels
    ctx = []
    for k, (wl, (x, v, w, r, m)) in enumerate(zip(lv, states)):
        cap = None if k == 0 else wl.n + 60_000
        # one stream per level: the levels' steps within a period run concurrently
        d = dem.DEM([dem.desc_from_workload(wl, capacity=cap)], max_neighbors=24, device=dev,
                    stream=torch.cuda.Stream(dev))
        v = v.clone()
        v[:, 0] += wl.meta["u0"]
        torch.cuda.synchronize(dev)       # the state tensors were made on the default stream
        d.write_state(x, v, w, r, m)
        ctx.append(d)
    h = levels.Hierarchy(ctx, specs)
    h.advance(3)
    torch.cuda.synchronize(dev)
    n0 = h.counts()
    st0 = [c.stats() for c in ctx]
    if profile:
        _profile(args, "coupled", True)
    t0 = time.perf_counter()
    h.advance(periods)                    # no host wait inside: the coupling calls run on the streams
    torch.cuda.synchronize(dev)
    t = time.perf_counter() - t0
    if profile:
        _profile(args, "coupled", False)
    n1 = h.counts()
    st1 = [c.stats() for c in ctx]
    # share of the coupling calls: a few periods with the host waiting around them
    t_step = t_couple = 0.0
    for _ in range(min(periods, 20)):
        ta = time.perf_counter()
        for c, n in zip(ctx, h.steps):
            c.step(n)
        torch.cuda.synchronize(dev)
        tb = time.perf_counter()
        for c in ctx:
            c.clear_external_force()
        for cp in h.couplers:
            cp.couple()
        torch.cuda.synchronize(dev)
        t_step += tb - ta
        t_couple += time.perf_counter() - tb
    inserted = [int(c.counts()[1][0]) - wl.n for c, wl in zip(ctx[1:], lv[1:])]
    h.close()
    for c in ctx:
        c.close()
    psteps = sum(0.5 * (a + b) * n * periods for a, b, n in zip(n0, n1, h.steps))
    sim_ms = periods * h.period * 1e3
    return {"value": psteps / t, "particles_per_level_start": n0, "particles_per_level_end": n1,
            "inserted_per_fine_level": inserted, "periods": periods, "steps_per_period": h.steps,
            "simulated_ms": sim_ms, "seconds": t, "wall_s_per_simulated_ms": t / sim_ms,
            "coupling_share": t_couple / (t_step + t_couple), "ms_per_step": t / (periods * h.steps[-1]) * 1e3,
            "rebuilds_per_level": [b["rebuilds"] - a["rebuilds"] for a, b in zip(st0, st1)]}


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
