"""Throughput of the event-based transport hot path on one GB300.

One step = one batch of the workload through the whole hot path (source,
sort, lookup, advance, surface, collision, tallies) in one device-driven
run of libgbmc.  Default workload: the 17x17 pin lattice with 68 + 3
synthetic nuclides of 10k-60k grid points, binary64 tables, 1e6 particles
per batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbmc|reference]
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25       # GB300 dense FP64 (recipe table)
# FP64-pipe work of one micro lookup in DFMA issue slots: 9 add/sub/mul plus
# one division, which costs ~9.2 DFMA slots (measured: 65 G div/s vs 598 G
# DFMA/s on this GPU)
FP64_SLOTS_PER_MICRO = 9 + 9.2
BRACKET_BYTES = {0: 32, 1: 16}    # E_j, E_j+1, s_j, s_j+1
LOOKUP_IO_BYTES = 36              # queue index 4, E 8, material 4, sigma_t/a 16, advance-queue 4

WORKLOADS = {
    1: "infinite medium, 4 nuclides x 2000 log-spaced points, 1e5 particles/batch",
    2: "17x17 pin lattice (r 0.4, p 1.26, H 100), pin 68 + moderator 3 nuclides x 10k-60k "
       "points, binary64 tables, 1e6 particles/batch",
    3: "17x17 pin lattice, binary32 tables, sorted, 1e7 particles/batch",
    4: "64 independent lattices (3x3..17x17, 4-68 pin nuclides, 1e4-1e6 particles each, "
       "log-uniform), binary32 tables, one device-driven graph launch, autotuned",
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p:
            time.sleep(0.3)
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(f) > 5 + k and f[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(prob, budget_s, threads, batch=0, cap=None):
    """Particles/s of the CPU oracle on a bounded sample (first ids of a batch)."""
    import oracle
    n = 2000
    t = time.perf_counter()
    oracle.run(prob, seed=prob.seed, batch=batch, n=n, threads=threads)
    dt = time.perf_counter() - t
    n = int(max(2000, min(budget_s / max(dt, 1e-6) * n, cap or prob.n_particles[0])))
    t = time.perf_counter()
    oracle.run(prob, seed=prob.seed, batch=batch, n=n, threads=threads)
    dt = time.perf_counter() - t
    return n / dt, n, dt


def run_reference(args, prob, rank):
    if rank != 0:
        return
    threads = len(os.sched_getaffinity(0))
    import oracle
    # size a step to ~budget seconds of oracle work
    _, n, dt = oracle_rate(prob, args.ref_step_s, threads)
    for w in range(args.warmup):
        oracle.run(prob, seed=prob.seed, batch=100 + w, n=min(n, 2000), threads=threads)
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        oracle.run(prob, seed=prob.seed, batch=k, n=n, threads=threads)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = n * args.steps / tot
    line = {
        "impl": "reference", "metric": "particles/s", "value": value, "unit": "particles/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, prob),
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": threads,
                         "kind": "oracle",
                         "sample": f"first {n} histories of batches 0..{args.steps - 1}"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(args, prob):
    return {"workload": prob.name, "description": WORKLOADS.get(args.config, ""),
            "problems": len(prob.geoms),
            "particles_per_batch": int(sum(args.particles or n for n in prob.n_particles)),
            "table_precision": "fp32" if args.precision == 1 else "fp64",
            "nuclides": int(prob.n_nuc), "grid_points": int(prob.grid_off[-1]),
            "table_bytes": int(prob.table_bytes(args.precision)),
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas{args.gpus}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbmc", choices=["gbmc", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--particles", type=int, default=0)
    ap.add_argument("--precision", type=int, default=-1)
    ap.add_argument("--max-in-flight", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--sort", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--ref-step-s", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=-1,
                    help="1: autotune launch settings before timing (default: config 4 only)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    prob = synth.make_config(args.config, n_particles=args.particles or None)
    if args.precision < 0:
        args.precision = prob.precision
    npart = prob.n_particles[0]

    if args.impl == "reference":
        run_reference(args, prob, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2403_12345_gb300 import gbmc, replicas

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()

    opts = dict(precision=args.precision, sort=args.sort)
    if args.max_in_flight:
        opts["max_in_flight"] = args.max_in_flight
    if args.blocks_per_sm:
        opts["blocks_per_sm"] = args.blocks_per_sm
    ctx = gbmc.Context(local, **opts)
    ctx.load(prob, (args.precision,))
    n_geo = len(prob.geoms)
    geoms = [gbmc.geometry_from(g) for g in prob.geoms]
    counts = [args.particles or prob.n_particles[k] for k in range(n_geo)]
    npart = sum(counts)

    def problems(batch):
        # replicas: each rank runs its own batches (weak scaling)
        return [gbmc.problem(geoms[k], prob.seed, counts[k], batch=batch * world + rank,
                             problem_index=k) for k in range(n_geo)]

    tuned = None
    if args.autotune == 1 or (args.autotune < 0 and args.config == 4):
        tuned = ctx.autotune(problems(40_000), fraction=0.1, stream=stream)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for w in range(args.warmup):
        ctx.run_problems(problems(10_000 + w), stream)
    torch.cuda.synchronize()
    ctx.reset_tallies(stream)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            ctx.run_problems(problems(k), stream)
            ev[k][1].record(stream)
            stats.append(ctx.read_stats())   # synchronizes; outside the events
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = npart * args.steps * world / (tot_ms * 1e-3)
    lookups = sum(s["lookups"] for s in stats)
    micro = sum(s["micro_lookups"] for s in stats)
    iters = sum(s["iterations"] for s in stats)

    # replicas: one tally reduction after the timed region (domain replication)
    flux, counts_, weights = ctx.read_tallies(0)
    if world > 1:
        flux, counts_, weights = replicas.allreduce_tallies(flux, counts_, weights)

    # end to end through the C ABI with host buffers: run, then copy every
    # problem's tallies and every particle's outcome (collisions, fate) to
    # the host
    e2e_steps = max(1, args.e2e_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for k in range(e2e_steps):
        ctx.run_problems(problems(20_000 + k), stream)
        d2h = 0
        for slot in range(n_geo):
            fl, cn, wt = ctx.read_tallies(slot)
            o = ctx.read_outcomes(slot, 0, counts[slot])
            d2h += fl.nbytes + cn.nbytes + wt.nbytes + sum(o[f].nbytes for f in o)
    e2e_s = time.perf_counter() - t0
    h2d = ctypes.sizeof(gbmc.Problem) * n_geo

    # per-kernel device times (eager launches between CUDA events) on one
    # more batch of the same workload
    kt = ctx.profile_problems(problems(30_000), stream)
    pst = ctx.read_stats()
    top = max(kt, key=lambda k: kt[k][0])
    hbm, peak_src = peaks()
    lk_ms, lk_n = kt["lookup"]
    lk_bytes = pst["micro_lookups"] * BRACKET_BYTES[args.precision] + pst["lookups"] * LOOKUP_IO_BYTES
    lk_gbs = lk_bytes / (lk_ms * 1e-3) / 1e9
    roof = {"kernel": "lookup", "bound": "hbm", "achieved": lk_gbs, "peak": hbm, "unit": "GB/s",
            "frac": lk_gbs / hbm, "traffic": None, "peak_source": peak_src,
            "launches": lk_n, "avg_launch_ms": lk_ms / max(lk_n, 1),
            "algorithmic_bytes_per_launch": lk_bytes / max(lk_n, 1)}
    if args.precision == 0:
        slots = pst["micro_lookups"] * FP64_SLOTS_PER_MICRO / (lk_ms * 1e-3)
        alu_peak = FP64_NOMINAL_TFLOPS * 1e12 / 2
        if slots / alu_peak > roof["frac"]:
            roof.update({"bound": "alu", "achieved": slots / 1e9, "peak": alu_peak / 1e9,
                         "unit": "G FP64-slot/s", "frac": slots / alu_peak,
                         "peak_source": "nominal 1.25 TFLOP/s FP64 = 625 G DFMA slots/s",
                         "hbm_equiv_gbs": lk_gbs})

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = len(os.sched_getaffinity(0))
        rate, n, dt = oracle_rate(prob, args.cpu_budget_s, threads)
        cpu = {"value": rate, "unit": "particles/s", "cores": threads, "kind": "oracle",
               "sample": f"first {n} histories of batch 0 ({dt:.1f} s)"}

    launches = sum(1 + 9 * s["iterations"] for s in stats)
    if rank == 0:
        line = {
            "metric": "particles/s", "value": value, "unit": "particles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == 1 else "f64", "data": "synthetic",
            "config": config_of(args, prob),
            "lookups_per_s": lookups * world / (tot_ms * 1e-3),
            "micro_lookups_per_s": micro * world / (tot_ms * 1e-3),
            "iterations_per_step": iters / args.steps,
            "wall_s": wall,
            "e2e": {"value": npart * e2e_steps / e2e_s, "unit": "particles/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "autotune": tuned,
            "roofline": roof,
            "kernel_ms_per_batch": {k: v[0] for k, v in kt.items()},
            "top_kernel": top,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
