"""The silo of Sec. 3 on the GPU: filling and settling with the orifice closed, then discharge
through the orifice, the discharge rate measured 1 cm below it at 100 Hz (Table 2 gives
0.400 +- 0.007 kg/s for the 2.8 mm reference and 0.315 +- 0.028 kg/s for the coarse-grain model,
alpha = 2).

The walls are the axisymmetric cone and cylinder of dem_set_walls; the measurement plane is the
removal height, so the mass removed per 10 ms sampling interval is the mass that crossed the
plane.  The filling is the synthetic lattice start of ``workloads.silo`` settled under gravity
(the paper pours particles in from the top for 0.47 s and lets them settle until 0.7 s).

    python -m paper_1705_03850_gb300.silo [--alpha 1 2] [--settle 0.3] [--discharge 0.6] [--two-level]

prints one JSON line per alpha (and one for the two-level silo).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import dem, workloads

PAPER_RATE = {1: (0.400, 0.007), 2: (0.315, 0.028)}   # Table 2, kg/s (mean, standard deviation)
PAPER_RATE_TWO_LEVEL = {"fine": (0.390, 0.009), "coarse": (0.391, 0.026)}   # Table 2, MLCG rows
PLANE_BELOW = 0.01   # the discharge rate is measured this far below the orifice [m] (Sec. 3)


def run(alpha: int = 1, settle_s: float = 0.3, discharge_s: float = 0.6, skip_s: float = 0.1,
        sample_s: float = 0.01, graph: int = 200, seed: int = 17, device=None) -> dict:
    """Settle the silo for settle_s with the orifice closed, open it and discharge for
    discharge_s; the rate is averaged over the sampling intervals after the first skip_s."""
    import torch

    wl = workloads.silo(alpha, seed=seed)
    sim = dem.from_workload(wl, max_neighbors=24, device=device)
    z_o = wl.meta["z_o"]
    sim.set_walls(0, (0.0, 0.0), workloads.silo_walls(z_o, closed=True))
    sim.set_step_lanes(0)                      # by size: the coarse grain runs fused steps, four lanes
    sim.set_graph(graph)
    dt = wl.dt
    g = max(graph, 1)
    steps_settle = int(round(settle_s / dt / g)) * g
    steps_sample = int(round(sample_s / dt / g)) * g
    nsample = int(round(discharge_s / sample_s))
    torch.cuda.synchronize(sim.device)
    t0 = time.perf_counter()
    sim.step(steps_settle).sync()
    t_settle = time.perf_counter() - t0
    st0 = sim.stats()
    # open the orifice; everything below the measurement plane 1 cm under it is removed
    sim.set_walls(0, (0.0, 0.0), workloads.silo_walls(z_o, closed=False), z_o - PLANE_BELOW)
    removed = []
    t0 = time.perf_counter()
    for _ in range(nsample):
        sim.step(steps_sample)
        removed.append(sim.wall_removed())
    t_dis = time.perf_counter() - t0
    st1 = sim.stats()
    live, _ = sim.counts()
    # the step kernel (the variant with walls) over the last graph: CUDA-event time of every
    # fifth launch, and the bytes one particle-step moves as the bench counts them (state 96 B,
    # 28 B per list entry) plus the two wall-history slots written (32 B)
    kms, kn = sim.graph_step_kernel_ms() if graph > 0 else (float("nan"), 1)
    L = st1["list_entries"] / max(1, st1["particles"])
    B = 96.0 + 28.0 * L + 32.0
    sim.close()
    mass = np.array([m for _, m in removed])
    rates = np.diff(np.concatenate([[0.0], mass])) / (steps_sample * dt)
    use = rates[int(round(skip_s / sample_s)):]
    steps = steps_settle + nsample * steps_sample
    psteps = wl.n * steps_settle + 0.5 * (wl.n + int(live[0])) * nsample * steps_sample
    ref = PAPER_RATE.get(alpha)
    return {
        "alpha": alpha, "diameter_m": wl.meta["diameter"], "particles": wl.n, "dt": dt,
        "settle_s": steps_settle * dt, "discharge_s": nsample * steps_sample * dt, "sample_s": steps_sample * dt,
        "rate_mean_kg_s": float(use.mean()), "rate_std_kg_s": float(use.std()),
        "rates_kg_s": [round(float(x), 4) for x in rates],
        "paper_rate_kg_s": None if ref is None else ref[0], "paper_std_kg_s": None if ref is None else ref[1],
        "removed_particles": int(removed[-1][0]), "removed_mass_kg": float(mass[-1]),
        "mass_kg": float(wl.m.sum()),
        "wall_s_settle": t_settle, "wall_s_discharge": t_dis,
        "particle_steps_per_s": psteps / (t_settle + t_dis), "steps": steps,
        "rebuilds_discharge": st1["rebuilds"] - st0["rebuilds"],
        "step_kernel_ms": kms / max(1, kn), "mean_list_length": L,
        "contacts_per_particle": st1["contacts"] / max(1, st1["particles"]),
        "bytes_per_particle_step": B,
        # modelled bytes over event time (not a DRAM measurement): the rows the last graph's step
        # kernels walked, from the same statistics snapshot as the list length
        "step_kernel_gbs_modelled": int(st1["particles"]) * B / (kms / max(1, kn) * 1e-3) / 1e9,
    }


def run_two_level(settle_s: float = 0.3, discharge_s: float = 0.6, skip_s: float = 0.1, sample_s: float = 0.01,
                  seed: int = 17, device=None) -> dict:
    """The multi-level silo (``workloads.silo_two_level``): both levels settle together with the
    orifice closed, then discharge; each level's rate is measured 1 cm below the orifice."""
    import torch

    from . import levels
    cw, fw, spec = workloads.silo_two_level(seed=seed)
    dev = torch.device(device or "cuda")
    # one stream per level: the two levels' steps of a coupling period run concurrently (the
    # coupling call orders the streams and ends with a host synchronisation)
    coarse = dem.DEM([dem.desc_from_workload(cw)], max_neighbors=24, device=dev, stream=torch.cuda.Stream(dev))
    coarse.write_state(cw.x, cw.v, cw.w, cw.r, cw.m)
    fine = dem.DEM([dem.desc_from_workload(fw, capacity=fw.n + 100_000)], max_neighbors=24, device=dev,
                   stream=torch.cuda.Stream(dev))
    fine.write_state(fw.x, fw.v, fw.w, fw.r, fw.m)
    z_o = cw.meta["z_o"]
    for lv in (coarse, fine):
        lv.set_walls(0, (0.0, 0.0), workloads.silo_walls(z_o, closed=True))
    h = levels.Hierarchy([coarse, fine], [spec])
    T = h.period
    n_settle = int(round(settle_s / T))
    per_sample = int(round(sample_s / T))
    nsample = int(round(discharge_s / (per_sample * T)))
    torch.cuda.synchronize(coarse.device)
    t0 = time.perf_counter()
    h.advance(n_settle)
    torch.cuda.synchronize(coarse.device)
    t_settle = time.perf_counter() - t0
    n_after_fill = h.counts()
    for lv in (coarse, fine):
        lv.set_walls(0, (0.0, 0.0), workloads.silo_walls(z_o, closed=False), z_o - PLANE_BELOW)
    removed = {"coarse": [], "fine": []}
    counts = []
    t0 = time.perf_counter()
    for _ in range(nsample):
        h.advance(per_sample)
        removed["coarse"].append(coarse.wall_removed()[1])
        removed["fine"].append(fine.wall_removed()[1])
        counts.append(h.counts())
    t_dis = time.perf_counter() - t0
    inserted = int(fine.counts()[1][0]) - fw.n
    h.close()
    coarse.close()
    fine.close()
    out = {"workload": "two-level silo: alpha = 2 over the whole silo, 2.8 mm in the lower quarter",
           "particles_start": [cw.n, fw.n], "particles_after_fill": n_after_fill, "particles_end": counts[-1],
           "fine_inserted": inserted, "period_s": T, "settle_s": n_settle * T,
           "discharge_s": nsample * per_sample * T, "sample_s": per_sample * T,
           "wall_s_settle": t_settle, "wall_s_discharge": t_dis}
    for name in ("fine", "coarse"):
        mass = np.array(removed[name])
        rates = np.diff(np.concatenate([[0.0], mass])) / (per_sample * T)
        use = rates[int(round(skip_s / (per_sample * T))):]
        out[name] = {"rate_mean_kg_s": float(use.mean()), "rate_std_kg_s": float(use.std()),
                     "rates_kg_s": [round(float(x), 4) for x in rates],
                     "paper_rate_kg_s": PAPER_RATE_TWO_LEVEL[name][0], "paper_std_kg_s": PAPER_RATE_TWO_LEVEL[name][1]}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--alpha", type=int, nargs="*", default=[1, 2])
    ap.add_argument("--settle", type=float, default=0.3, help="settling time with the orifice closed [s]")
    ap.add_argument("--discharge", type=float, default=0.6, help="discharge time [s]")
    ap.add_argument("--skip", type=float, default=0.1, help="start-up interval left out of the average [s]")
    ap.add_argument("--graph", type=int, default=200)
    ap.add_argument("--two-level", action="store_true", help="also run the two-level (alpha 2 / 1) silo")
    a = ap.parse_args(argv)
    for alpha in a.alpha:
        r = run(alpha, settle_s=a.settle, discharge_s=a.discharge, skip_s=a.skip, graph=a.graph)
        print(json.dumps(r), flush=True)
    if a.two_level:
        print(json.dumps(run_two_level(settle_s=a.settle, discharge_s=a.discharge, skip_s=a.skip)), flush=True)


if __name__ == "__main__":
    main()
