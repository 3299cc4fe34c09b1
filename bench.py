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
    ap.add_argument("--graph", type=int, default=50, help="steps per captured CUDA graph (0: direct launches)")
    ap.add_argument("--settle-graph", type=int, default=50, help="steps per graph while settling")
    ap.add_argument("--lmax", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--adjoint-instances", type=int, default=64)
    ap.add_argument("--batched-steps", type=int, default=2000)
    ap.add_argument("--batched-scale", type=float, default=1.0, help="scale of the 256 box sizes (1 = as stated)")
    ap.add_argument("--no-cpu", action="store_true")
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


def _kernel_hash():
    p = os.path.join(ROOT, "paper_1705_03850_gb300", "csrc", "dem.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# --------------------------------------------------------------- CPU oracle

def cpu_oracle_sample(target_seconds):
    """Time the FP64 oracle (single thread) on a dense polydisperse block, the bounded CPU sample."""
    import oracle
    from paper_1705_03850_gb300 import workloads
    wl = workloads.dense_block(60, 60, 40, seed=2, rjit=0.2, vel=0.05, spin=5.0)
    m = wl.material
    P = oracle.make_params(E=m.E, nu=m.nu, e=m.e, mu=m.mu, dt=wl.dt, g=wl.g, lo=wl.lo, hi=wl.hi,
                           periodic=wl.periodic, floor=wl.floor, floor_v=wl.floor_v)
    sim = oracle.Sim(P, wl.x, wl.v, wl.w, wl.r, wl.m)
    sim.run(0)                       # start-up evaluation, not timed
    t0 = time.perf_counter()
    steps = 0
    while True:
        sim.run(1)
        steps += 1
        if time.perf_counter() - t0 >= target_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": wl.n * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 C oracle, 1 thread, {steps} steps of a {wl.n}-particle dense polydisperse block "
                      f"(d in [1.6, 2.4] mm, overlapping jittered lattice, cell-list contacts), {dt:.1f} s",
            "host": os.uname().machine, "nproc": os.cpu_count()}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    steps = max(1, args.steps)
    cpu = cpu_oracle_sample(args.cpu_seconds)
    line = {"impl": "reference", "metric": METRIC, "value": cpu["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "shear_bed_1M stand-in: dense polydisperse block (oracle sample)",
                       "n_particles": args.n},
            "cpu_baseline": cpu,
            "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    S = args.graph
    K = max(S, (args.steps // S) * S) if S > 0 else max(1, args.steps)
    W = max(3, args.warmup)

    # ---- build and settle the bed (not timed): larger step and more damping
    # than the sheared run, so that the lattice collapses into a dense bed quickly
    wl = workloads.shear_bed(args.n, seed=2)
    desc = dem.desc_from_workload(wl, r_max=1.2e-3)
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

    # ---- sheared bed: floor moves at 0.5 m/s in x
    desc.floor_v[0] = 0.5
    sim = dem.DEM([desc], max_neighbors=args.lmax, device=dev)
    sim.write_state(x, v, w, r, m)
    sim.step(1)
    if S > 0:
        sim.set_graph(S)
        sim.step(((W + S - 1) // S) * S)
    else:
        sim.step(W)
    sim.sync()
    st0 = sim.stats()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    kern_ms, kern_n = sim.graph_step_kernel_ms() if S > 0 else (float("nan"), 1)
    st1 = sim.stats()
    sim.sync()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    n = wl.n
    value = n * K * world / (ms / 1e3)
    L = st1["list_entries"] / max(1, st1["particles"])
    C = st1["contacts"] / max(1, st1["particles"])
    Wc = st1["wall_contacts"] / max(1, st1["particles"])
    rebuilds = st1["rebuilds"] - st0["rebuilds"]
    # algorithmic bytes per particle-step of the step kernel, SURVEY.md 8(d):
    # 48 B own state read + 48 B written, per list entry 4 B index + 12 B history read + 12 B written
    B_step = 96.0 + 28.0 * L
    # what this design must move at least: the same state, count and history mask,
    # indices of every entry, history only of entries in contact, floor history
    B_design = 96.0 + 4.0 + 8.0 + 4.0 * L + 24.0 * (C - Wc) + 32.0 * Wc
    t_kernel = kern_ms / max(1, kern_n) / 1e3
    achieved = n * B_step / t_kernel / 1e9
    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    traffic = _profile_traffic(_kernel_hash())
    launches = K + (K // S if S > 0 else 9 * K) + 9 * rebuilds

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
        t_e2e = time.perf_counter() - t0
        h2d = (hx.numel() + hv.numel() + hw.numel() + hr.numel() + hm.numel()) * 8
        d2h = (ox.numel() + ov.numel() + ow.numel()) * 8
        e2e = {"value": n * K / t_e2e * world, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K, "chunk_steps": K,
               "what": "dem_write(POS,VEL,OMEGA,RADIUS,MASS) from pinned host, dem_step(K), "
                       "dem_read(POS,VEL,OMEGA) to pinned host; bytes per DEM step = chunk bytes / K"}

    batched = None if args.no_batched else run_batched(args, dev, value)
    adj = None if args.no_adjoint else run_adjoint(args, dev, value)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_oracle_sample(args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"shear_bed: {n:,} polydisperse spheres, settled then floor-sheared",
                   "n_particles": n, "dt": wl.dt, "skin_m": wl.skin, "settle_steps": args.settle,
                   "settle": "dt 5e-6 s, e 0.5, from the FCC start",
                   "steps_per_graph": S, "max_neighbors": args.lmax,
                   "l2": "inputs larger than L2 (state + lists + histories > 129 MB)",
                   "mean_list_length": L, "mean_contacts_per_particle": C, "rebuilds_in_timed_region": rebuilds,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src, "kernel": "k_step<0> (fused force + Verlet)",
                     "bytes_per_particle_step": B_step, "kernel_ms_avg": t_kernel * 1e3,
                     "design_bytes_per_particle_step": B_design,
                     "design_achieved": n * B_design / t_kernel / 1e9,
                     "kernel_share_of_step": t_kernel * 1e3 / (ms / K)},
        "clocks": clocks.summary(),
        "e2e": e2e,
        "batched": batched,
        "adjoint": adj,
        "gpu_launches": launches,
        "cpu_baseline": cpu,
    }
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
    e0.record(sim.stream)
    sim.step(1)               # start-up evaluation and first list build of all 256 boxes
    sim.step(K - 1 - ((K - 1) % S))
    sim.step((K - 1) % S)
    e1.record(sim.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    sim.sync()
    sim.close()
    value = n * K / (ms / 1e3)
    return {"value": value, "unit": UNIT, "workload": "256 settling boxes, N_k log-uniform in [2e3, 2e5] "
            "(seed 4), d = 2 mm, per-box E, e, mu", "n_instances": len(wls), "n_particles": n, "steps": K,
            "ms_per_step": ms / K, "vs_plain": value / plain_value, "rebuilds": st1["rebuilds"] - st0["rebuilds"],
            "mean_list_length": st1["list_entries"] / max(1, st1["particles"]),
            "timed": "all K steps from the lattice start, including the first list build",
            "tuned": best.as_dict(), "tuning_seconds": t_tune, "candidates": len(allc),
            "tuning": "each candidate timed on 32 of the boxes (spread over sizes) for the full step count"}


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
    t0 = time.perf_counter()
    sim.rollout_forward(N, K)
    t1 = time.perf_counter()
    obs = sim.observables(axis)
    grad = sim.rollout_adjoint(np.ones((B, 2)), axis)
    t2 = time.perf_counter()
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
