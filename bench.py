#!/usr/bin/env python
"""Benchmark of the implicit bonded-DEM step (GB300).

Workload: the ceramic-plate fracture scene (hexagonal-close-packed disk, 219,314 particles, 1,092,558 bonds, E = 5e9,
dt = 5e-4, tensile break strain 1e-3, dropped at 3 m/s onto the ground with penalty contact), FP32-mixed path.
A "step" is one full time step (prediction, contact candidates, the Newton loop with its PCG solves and line
searches, velocity update, fracture). Metric: particle-Newton-iterations per second (sum over steps of
particles x Newton iterations, divided by time); sim steps/s is reported beside it, and the FP64 GPU path is timed
on the same workload for the mixed-over-FP64 speedup at equal Newton residual (1e-6 relative).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the workload (replicas only: the path has no
cross-GPU exchange); the wall time is the maximum over ranks and the value counts every rank's work.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-Newton-iters/s & sim steps/s, FP32-mixed vs FP64 GPU at 1e-6 residual"
UNIT = "particle-Newton-iters/s"
WORKLOAD = ("ceramic plate fracture: HCP disk R=0.284 m, 3 layers, r=1 mm, bonds within 1.05*2r, jitter 1e-5 m, "
            "E=5e9 Pa, nu=0.3, rho=2500, break strain 1e-3, dropped at 3 m/s tilted 10 deg, ground and self "
            "penalty contact k=E*r, dt=5e-4 s, Newton tol 1e-6 relative")
SAMPLE_R = 0.01  # radius of the bounded CPU sample of the same plate construction (272 particles)
SAMPLE_CYCLE = 6  # the sample's steps: the first SAMPLE_CYCLE landing steps, restarted from the initial state
OTHER_WORKLOADS = {  # extra measurement lines (not the benchmark's workload), selected with --workload
    "batched": "64 independent Poisson-disk boxes, 2K-50K particles each (log-uniform, seed 4), r=2 mm, bonds within "
               "1.1*2r, drops 0.1-1 m, E=1e8 Pa, break strain 2e-3, ground and self contact k=E*r, dt=1e-3 s",
    "impact": "1M-particle Poisson-disk slab (r=2 mm, bond cutoff for mean degree 12, E=1e9 Pa, break strain 1e-3) hit "
              "by a 2,000-particle unbreakable ball (E=1e10 Pa) at 20 m/s, ground and self contact, dt=2e-4 s",
}


# ------------------------------------------------------------------------------------------------
# algorithmic bytes of one PCG iteration (the dominant kernel)
# ------------------------------------------------------------------------------------------------

def pcg_bytes_per_iter(n, nb, n_contact_entries, w):
    """Bytes one PCG iteration must move from memory at minimum in this layout (Chronopoulos-Gear arrangement): the
    factored bond blocks (33 words per bond, read once), the diagonal blocks and their inverses (2 x 21 words per
    particle), fourteen 6-word vector streams per particle (w = H z: read z r, write w; update: read z w p s x r,
    write p s x r z), and the active contact entries (index 4 B + rank-one block 4 words)."""
    return nb * 33 * w + n * (42 * w + 84 * w) + n_contact_entries * (4 + 4 * w)


def pcg_bytes_per_launch_fixed(n, nb):
    """Bytes one PCG launch reads once and keeps on chip for the whole solve: the two incidence entries of every
    bond (8 B each) and each row's start, active-contact count and kinematic flag (9 B)."""
    return nb * 16 + n * 9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


PCG_REGION = ("template <int NW>\n__device__ __forceinline__ void load_words(const float* src",
              "// per-scene reductions outside the PCG")


def pcg_source_hash():
    """sha256 of the source text of the PCG kernel and the device helpers it uses."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2308_10459_gb300", "csrc", "bdem_kernels.cu")).read()
    a, b = src.index(PCG_REGION[0]), src.index(PCG_REGION[1])
    return hashlib.sha256(src[a:b].encode()).hexdigest()


def traffic_record():
    """ncu DRAM bytes of the PCG kernel per iteration (and staged once per launch) for the product variants and lanes
    per row captured, if captured for the current kernel source."""
    path = os.path.join(ROOT, "profiles", "k_pcg_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("pcg_source_sha256") != pcg_source_hash():
            return None
        return rec
    except Exception:
        return None


def traffic_for_shape(trec, shape):
    """The captured record of the launch shape's product variant (the same lanes per row if captured, else another
    lanes setting of that variant, which moves the same data; None: the variant was not captured)."""
    if trec is None or shape is None:
        return None
    recs = [r for r in trec.get("records", []) if r["product"] == shape["product"]]
    for r in recs:
        if r["lanes_per_row"] == shape["lanes_per_row"]:
            return r
    return recs[0] if recs else None


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------------
# distributed helpers (replicas only)
# ------------------------------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_timing(elapsed_s, units, world):
    """Max of the timed region over ranks, sum of the work units (torch.distributed must be initialised if
    world > 1)."""
    if world <= 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------------
# CPU oracle legs
# ------------------------------------------------------------------------------------------------

def host_cpu():
    """Model name and logical core count of the host CPU (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"model": model or "unknown", "logical_cores": os.cpu_count()}


class OracleSample:
    """The bounded CPU sample of the plate workload: the same plate construction at R = SAMPLE_R m, advanced by the
    oracle (single thread) through the first SAMPLE_CYCLE time steps of its landing (dropped at 3 m/s onto the ground,
    ground and self contact, ~20 Newton iterations per step) and restarted from its initial state after each cycle, so
    that every sample step is a landing step like the GPU's timed steps and the run's length is bounded."""

    def __init__(self):
        import oracle
        from paper_2308_10459_gb300 import scenes
        oracle.build()
        self.oracle = oracle
        self.sc = scenes.c2_plate_small(R=SAMPLE_R)
        self.k = 0
        self.o = None

    def step(self):
        """One sample step; returns the particle-Newton-iterations it did."""
        if self.k % SAMPLE_CYCLE == 0:
            self.o = self.oracle.OracleSim(self.sc)
        self.k += 1
        st = self.o.step(1)[0][0]
        return self.sc.n * st["newton_iters"]

    def describe(self, steps):
        return (f"{steps} oracle time steps (one host core, FP64) of the same plate construction at R={SAMPLE_R} m "
                f"({self.sc.n} particles, {self.sc.nb} bonds): steps 1-{SAMPLE_CYCLE} of its landing, cycled from the "
                f"initial state")


def oracle_sample_rate(n_steps):
    """The CPU oracle (single thread) on n_steps sample steps; returns (rate, seconds, description)."""
    smp = OracleSample()
    t0 = time.perf_counter()
    units = sum(smp.step() for _ in range(n_steps))
    t = time.perf_counter() - t0
    return units / t, t, smp.describe(n_steps)


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    smp = OracleSample()
    for _ in range(args.warmup):
        smp.step()
    t0 = time.perf_counter()
    units = sum(smp.step() for _ in range(args.steps))
    t = time.perf_counter() - t0
    value = units / t
    sample = smp.describe(args.steps) + f", after {args.warmup} warm-up steps"
    cpu = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "sim_steps_per_s": args.steps / t,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host_cpu": cpu["model"], "host_logical_cores": cpu["logical_cores"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# main (our CUDA path)
# ------------------------------------------------------------------------------------------------

def timed_steps(sim, K, world, torch, sizes, profile):
    """K steps between barriers, timed with CUDA events. profile=False: the default step (one captured graph per
    step); profile=True: the host-driven loop with CUDA events around every phase and PCG launch."""
    launches0 = sim.launch_count()
    graph0 = sim.graph_steps()
    sim.profile_enable(profile)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = []
    for _ in range(K):
        stats.append(sim.step(1))
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    prof = sim.profile_read() if profile else None
    sim.profile_enable(False)
    units = sum(int(sizes[k]) * int(st[k]["newton_iters"]) for st in stats for k in range(len(sizes)))
    newton = sum(int(st[k]["newton_iters"]) for st in stats for k in range(len(sizes)))
    pcg = sum(int(st[k]["pcg_iters"]) for st in stats for k in range(len(sizes)))
    refine = sum(int(st[k]["refine_rounds"]) for st in stats for k in range(len(sizes)))
    res = [float(st[k]["lin_rel_residual"]) for st in stats for k in range(len(sizes)) if st[k]["lin_rel_residual"] >= 0]
    return dict(elapsed=elapsed, prof=prof, launches=sim.launch_count() - launches0, stats=stats, units=units,
                newton=newton, pcg=pcg, graph_steps=sim.graph_steps() - graph0, refine=refine,
                lin_res=(max(res) if res else None))


def pcg_probe(args, sc, sim, pkg, torch):
    """One PCG solve of exactly N iterations (eps_r = 0) on the system at the state after `warmup` steps; prints the
    time per iteration and the algorithmic bytes (the command the k_pcg ncu captures use)."""
    import numpy as np
    if args.warmup:
        sim.step(args.warmup)
    if args.pcg_lanes:
        sim.set_pcg_product(args.pcg_product)
        sim.set_pcg_shape(args.pcg_lanes, args.pcg_blocks)
    st = sim.read_state()
    dt = sc.config["dt"]
    sys_ = sim.bdem_debug_system(st["pos"] + dt * st["vel"], st["quat"] + dt * st["quat_vel"], want_bonds=False)
    b = -sys_["g"]
    sim.profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, it = sim.bdem_debug_pcg(b, 0.0, args.pcg_probe)
    t = time.perf_counter() - t0
    line = {"probe": "pcg", "iters": int(it[0]), "seconds_incl_transfers": t, "n": sc.n, "nb": sc.nb,
            "algorithmic_bytes_per_iter_without_contacts": pcg_bytes_per_iter(sc.n, sc.nb, 0, 4),
            "fixed_bytes_per_launch": pcg_bytes_per_launch_fixed(sc.n, sc.nb),
            "lanes": args.pcg_lanes, "shape": sim.pcg_shape()}
    print(json.dumps(line), flush=True)
    return 0


def pcg_roofline(sc, rrun, sizes, trec, shape):
    """Roofline of the persistent PCG kernel from a profiled pass: algorithmic bytes per launch (per scene and step:
    its PCG iterations x its bytes per iteration with the intact bonds after the step, plus the active contact entries
    actually in the systems, plus the once-per-launch staging) over the mean launch time from CUDA events."""
    prof = rrun["prof"]
    pcg_launches = max(prof["intervals"]["pcg"], 1)
    pcg_iters_launch = prof["pcg_iters"] / pcg_launches
    pcg_ms_launch = prof["ms"]["pcg"] / pcg_launches
    alg = 0.0
    for st in rrun["stats"]:
        for k in range(len(sizes)):
            alg += int(st[k]["pcg_iters"]) * pcg_bytes_per_iter(int(sizes[k]), int(st[k]["intact_bonds"]), 0, 4)
            alg += int(st[k]["contact_entry_pcg_iters"]) * (4 + 4 * 4)
    bytes_launch = alg / pcg_launches + pcg_bytes_per_launch_fixed(sc.n, sc.nb)
    bytes_iter = pcg_bytes_per_iter(sc.n, sum(int(rrun["stats"][-1][k]["intact_bonds"]) for k in range(len(sizes))),
                                    0, 4)
    achieved = bytes_launch / (pcg_ms_launch * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    tr = traffic_for_shape(trec, shape)
    traffic = None if tr is None else tr["dram_bytes_per_pcg_iter"] * pcg_iters_launch + tr["dram_bytes_once"]
    return {"bound": "hbm", "kernel": "k_pcg (persistent PCG)", "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_launch,
            "algorithmic_bytes_per_pcg_iter_without_contacts": bytes_iter,
            "pcg_iters_per_launch": pcg_iters_launch, "launch_ms": pcg_ms_launch,
            "timing": "CUDA events around each PCG launch on the library stream, in a second pass over the same steps "
                      "(same starting state) through the host-driven loop"}


def measure_mixed(sc, args, steps, world, torch, pkg, amg, trec, e2e_on, clocks=None):
    """The FP32-mixed path on one workload: `warmup` steps, PCG autotuning, one step that captures the step graph,
    then three passes over the same `steps` steps from the same committed state: (1) the default path (one graph launch
    per step), timed with CUDA events -> value; (2) the host-driven loop with phase events -> roofline of the PCG;
    (3) end to end through the C ABI with pinned host buffers (write_state + step + read_state every step) -> e2e."""
    import numpy as np
    pcfg = dict(preconditioner=pkg.BDEM_PRECOND_AMG if amg else pkg.BDEM_PRECOND_BLOCK_JACOBI)
    if args.no_refine:
        pcfg["pcg_refine"] = 0
    sim = pkg.Sim(sc, precision=pkg.BDEM_MIXED, config=pcfg)
    sim.step(args.warmup)
    if amg:
        shape = None  # the AMG-preconditioned solve runs as host-driven kernels, not the persistent PCG
    elif args.pcg_lanes:
        sim.set_pcg_product(args.pcg_product)
        sim.set_pcg_shape(args.pcg_lanes, args.pcg_blocks)
        shape = dict(sim.pcg_shape(), autotuned=False)
    else:
        sim.autotune_pcg(30)
        shape = dict(sim.pcg_shape(), autotuned=True)
    if shape is not None:
        shape["bond_hessian"] = sim.autotune_bonds(3)  # tile and register variant of the bond-Hessian kernel
    sizes = np.diff(sc.scene_offsets)
    sim.step(1)  # captures the step graph for the chosen PCG shape outside the timed region
    ck = sim.read_state()
    if clocks:
        clocks.start()
    run = timed_steps(sim, steps, world, torch, sizes, profile=False)
    clk = clocks.stop() if clocks else None
    t_max, units = reduce_timing(run["elapsed"], run["units"], world)
    # (2) profiled pass from the same state
    sim.write_state(ck["pos"], ck["quat"], ck["vel"], ck["quat_vel"], ck["broken"])
    rrun = timed_steps(sim, steps, world, torch, sizes, profile=True)
    same_work = all(a[k]["newton_iters"] == b[k]["newton_iters"] and a[k]["pcg_iters"] == b[k]["pcg_iters"]
                    for a, b in zip(run["stats"], rrun["stats"]) for k in range(len(sizes)))
    prof = rrun["prof"]
    roof = None if amg else pcg_roofline(sc, rrun, sizes, trec, shape)
    # (3) end to end from the same state, host copies inside the timed region
    e2e = None
    if e2e_on:
        n, nb = sc.n, sc.nb
        pin = {k: torch.empty(v.shape, dtype=torch.float64 if v.dtype == np.float64 else torch.uint8,
                              pin_memory=True).numpy() for k, v in ck.items()}
        for k in pin:
            pin[k][...] = ck[k]
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        pni = 0
        e2e_stats = []
        for _ in range(steps):
            sim.write_state(pin["pos"], pin["quat"], pin["vel"], pin["quat_vel"], pin["broken"])
            s = sim.step(1)
            e2e_stats.append(s)
            pni += sum(int(sizes[k]) * int(s[k]["newton_iters"]) for k in range(len(sizes)))
            sim.read_state(pin)
        t_e2e = time.perf_counter() - t0
        barrier(world)
        e2e_same = all(a[k]["newton_iters"] == b[k]["newton_iters"] and a[k]["pcg_iters"] == b[k]["pcg_iters"]
                       for a, b in zip(run["stats"], e2e_stats) for k in range(len(sizes)))
        t_e2e, pni = reduce_timing(t_e2e, pni, world)
        e2e = {"value": pni / t_e2e, "unit": UNIT, "h2d_bytes_per_step": n * (3 + 4 + 3 + 4) * 8 + nb,
               "d2h_bytes_per_step": n * (3 + 4 + 3 + 4) * 8 + nb, "steps": steps,
               "same_steps_as_value": e2e_same,
               "timing": "host wall clock; every step writes the state from pinned host buffers, steps through "
                         "bdem_step and reads the state back, over the same steps from the same state as value"}
    sim.close()
    return {"value": units / t_max, "t_max": t_max, "run": run, "rrun": rrun, "same_work": same_work, "prof": prof,
            "shape": shape, "roofline": roof, "e2e": e2e, "clocks": clk}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=5,
                    help="steps of the 64-scene batched workload measured beside the plate (0: skip)")
    ap.add_argument("--pcg-lanes", type=int, default=0, help="lanes per row of the PCG product (0: autotune)")
    ap.add_argument("--pcg-blocks", type=int, default=0, help="PCG grid size with --pcg-lanes (0: all resident)")
    ap.add_argument("--pcg-product", type=int, default=1, choices=[0, 1, 2, 3],
                    help="with --pcg-lanes: 3 one grid barrier per iteration (update fused into the next product), "
                         "2 double-buffered and 1 single-buffered warp-cooperative staging of the bond blocks, 0 "
                         "per-lane loads")
    ap.add_argument("--pcg-probe", type=int, default=0,
                    help="time N PCG iterations of one solve (eps 0) on the workload's system and exit (profiling)")
    ap.add_argument("--workload", default="plate", choices=["plate", "batched", "impact"],
                    help="plate: the benchmark workload; batched / impact: extra measurement lines")
    ap.add_argument("--precond", default="block-jacobi", choices=["block-jacobi", "amg"],
                    help="PCG preconditioner: block Jacobi (the benchmark path) or the aggregation AMG (comparison)")
    ap.add_argument("--no-refine", action="store_true",
                    help="mixed path without the FP64-residual refinement of its linear solves (comparison)")
    ap.add_argument("--radius", type=float, default=0.284,
                    help="plate radius; anything but 0.284 m is a smaller profiling case, not the benchmark workload")
    args = ap.parse_args()
    if args.warmup < 3 and not args.pcg_probe:
        args.warmup = 3
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        import torch
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    import paper_2308_10459_gb300 as pkg
    from paper_2308_10459_gb300 import build as bmod
    from paper_2308_10459_gb300 import scenes

    torch.cuda.set_device(local)
    bmod.build()
    pkg.load()
    if args.workload == "batched":
        sc = scenes.c4_batched()
    elif args.workload == "impact":
        sc = scenes.c5_impact()
    else:
        sc = scenes.c2_plate(R=args.radius)

    amg = args.precond == "amg"
    pcfg = dict(preconditioner=pkg.BDEM_PRECOND_AMG if amg else pkg.BDEM_PRECOND_BLOCK_JACOBI)
    if args.pcg_probe:
        sim = pkg.Sim(sc, precision=pkg.BDEM_MIXED, config=pcfg)
        return pcg_probe(args, sc, sim, pkg, torch)
    # the ncu record is of the plate's PCG: it scales to the plate's launches only
    trec = traffic_record() if args.workload == "plate" and args.radius == 0.284 else None
    m = measure_mixed(sc, args, args.steps, world, torch, pkg, amg, trec, not args.no_e2e, ClockSampler(local))
    run, prof = m["run"], m["prof"]

    # ---- FP64 GPU path on the same workload ----
    fp64 = None
    if args.fp64_steps > 0:
        sizes = np.diff(sc.scene_offsets)
        sim64 = pkg.Sim(sc, precision=pkg.BDEM_FP64, config=pcfg)
        sim64.step(args.warmup)
        r64 = timed_steps(sim64, args.fp64_steps, world, torch, sizes, profile=False)
        t64, u64 = reduce_timing(r64["elapsed"], r64["units"], world)
        fp64 = {"value": u64 / t64, "unit": UNIT, "steps": args.fp64_steps, "ms_per_step": 1e3 * t64 / args.fp64_steps,
                "sim_steps_per_s": args.fp64_steps * world / t64,
                "newton_iters_per_step": r64["newton"] / args.fp64_steps,
                "pcg_iters_per_newton": r64["pcg"] / max(r64["newton"], 1), "graph_steps": r64["graph_steps"],
                "window": f"steps {args.warmup + 1}-{args.warmup + args.fp64_steps} of the workload"}
        sim64.close()

    # ---- the 64-scene batched workload (uneven scenes in the same launches), beside the plate ----
    batched = None
    if args.workload == "plate" and args.radius == 0.284 and args.batched_steps > 0 and not amg:
        scb = scenes.c4_batched()
        mb = measure_mixed(scb, args, args.batched_steps, world, torch, pkg, False, None, False)
        rb = mb["run"]
        batched = {"workload": OTHER_WORKLOADS["batched"], "n_scenes": scb.n_scenes, "n_particles": scb.n,
                   "n_bonds": scb.nb, "value": mb["value"], "unit": UNIT, "steps": args.batched_steps,
                   "ms_per_step": 1e3 * mb["t_max"] / args.batched_steps,
                   "newton_iters_per_step": rb["newton"] / args.batched_steps,
                   "pcg_iters_per_newton": rb["pcg"] / max(rb["newton"], 1), "graph_steps": rb["graph_steps"],
                   "refinement_rounds_per_newton": rb["refine"] / max(rb["newton"], 1),
                   "pcg_shape": mb["shape"], "roofline": mb["roofline"], "same_work": mb["same_work"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "plate":
        rate, secs, desc = oracle_sample_rate(SAMPLE_CYCLE)
        hc = host_cpu()
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc + f" ({secs:.1f} s)",
               "host_cpu": hc["model"], "host_logical_cores": hc["logical_cores"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * m["t_max"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": (OTHER_WORKLOADS[args.workload] if args.workload != "plate" else
                                    WORKLOAD if args.radius == 0.284 else f"profiling case R={args.radius} m"),
                       "n_scenes": sc.n_scenes,
                       "precision": "FP32-mixed (f32 Hessian/PCG, f64 gradient/reductions/state)",
                       "n_particles": sc.n, "n_bonds": sc.nb, "replicas": world,
                       "preconditioner": args.precond,
                       "timed_steps": f"steps {args.warmup + 2}-{args.warmup + 1 + args.steps} of the workload",
                       "l2": "working set of every timed stage exceeds the 129 MB L2; no flush between steps"},
            "sim_steps_per_s": args.steps * world / m["t_max"],
            "newton_iters_per_step": run["newton"] / args.steps,
            "pcg_iters_per_newton": run["pcg"] / max(run["newton"], 1),
            "refinement": {"rounds_per_newton": run["refine"] / max(run["newton"], 1),
                           "max_true_rel_residual_of_last_solves": run["lin_res"],
                           "on": not args.no_refine and not amg},
            "graph_steps": run["graph_steps"],
            "host_loop_pass": {"ms_per_step": 1e3 * m["rrun"]["elapsed"] / args.steps, "same_work": m["same_work"],
                               "phase_ms_per_step": {k: v / max(prof["steps"], 1) for k, v in prof["ms"].items()}},
            "pcg_shape": m["shape"],
            "roofline": m["roofline"],
            "fp64": fp64,
            "mixed_over_fp64": (m["value"] / fp64["value"]) if fp64 else None,
            "batched": batched,
            "cpu_baseline": cpu,
            "e2e": m["e2e"],
            "gpu_launches": run["launches"],
            "clocks": m["clocks"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
