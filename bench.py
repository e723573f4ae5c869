"""Throughput of the event-based transport hot path on one GB300.

One step = one batch of the workload through the whole hot path (source,
sort, lookup, ray trace, collision, tallies) in one device-driven run of
libgbmc.  Default workload: the 17x17 pin lattice with 68 + 3 synthetic
nuclides of 10k-60k grid points, binary64 tables, 1e6 particles per batch.
--config 3 / 4: binary32 lattice, 64 lattices in one launch; --config 5:
learned weight windows against analog (figure of merit); --config 6: the
lookup-only stress set.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbmc|reference] [--config C]
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
BRACKET_BYTES = {0: 32, 1: 16}    # E_j, E_j+1, s_j, s_j+1
# binary64 operations a micro lookup must perform (the workload
# description's count: the two differences and the quotient of the
# interpolation factor, its multiply-add, and the multiply-add of the sum);
# the kernel issues fewer on the binary64 pipe: the interpolation's and the
# sum's fused multiply-adds, while E - E_k and the quotient run exactly on the
# integer units, so against the binary64 rate the algorithmic count can pass 1
ALGO_FP64_OPS_PER_MICRO = 6
ISSUED_FP64_PER_MICRO = 2         # binary64 instructions the kernel issues per micro lookup (Sigma_t)
LOOKUP_IO_BYTES = 28              # per macro lookup: E 8, material 4, sigma_t and sigma_a 16
# kernels an iteration launches: plan, source, 2 sort, lookup, ray trace, collision
ITER_KERNELS = {0: 7, 1: 7}
# DRAM (and L2) bytes of every lookup launch of one eager profiled batch, from
# ncu counters, written by `bench.py --record-traffic` and keyed by workload,
# table precision and window-load width; each entry carries a hash of the
# kernel sources it was measured on and is ignored once they change
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "lookup_traffic.json")
KERNEL_SOURCES = ("paper_2403_12345_gb300/csrc/device.cuh",
                  "paper_2403_12345_gb300/csrc/transport.cu")
E2E_REPEATS = 3                   # timed end-to-end calls; the median is reported
FP32_TALLY_L2_GATE = 1e-4         # binary32 tables against binary64, whole-batch flux

WORKLOADS = {
    1: "infinite medium, 4 nuclides x 2000 log-spaced points, 1e5 particles/batch",
    2: "17x17 pin lattice (r 0.4, p 1.26, H 100), pin 68 + moderator 3 nuclides x 10k-60k "
       "points, binary64 tables, 1e6 particles/batch",
    3: "17x17 pin lattice, binary32 tables, sorted, 1e7 particles/batch",
    4: "64 independent lattices (3x3..17x17, 4-68 pin nuclides, 1e4-1e6 particles each, "
       "log-uniform), binary32 tables, one device-driven graph launch, autotuned",
    5: "deep-penetration slab (10 cm scatterer + 100 cm absorber), far-face leakage; learned "
       "weight windows (4-64-64-1 BF16 MLP trained on analog estimates) against analog",
    6: "lookup-only stress set: 281 nuclides x 60k points, one 244-nuclide material, 1e7 "
       "energies log-uniform on [1e-5, 2e7] eV (unsorted; the library sorts)",
    7: "k-eigenvalue power iteration on the 17x17 lattice (40 fissile pin nuclides), binary64 "
       "tables, 1e6 particles per generation; steps are active generations after the inactive ones",
}


def bf16_peak():
    """The measured dense bf16 tensor rate (TFLOP/s, burst) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def mlp_forward_measure(ctx, stream, rows=1 << 24, reps=5):
    """The importance network's forward (gbmc_mlp_forward: the 64 x 64 layer
    on the tensor cores) over `rows` feature rows, timed with CUDA events
    after three warm-up calls: rows/s, the network's flops against the
    measured bf16 rate, and its 20 bytes a row against measured HBM."""
    import torch
    feat = torch.rand((rows, 4), dtype=torch.float32, device="cuda")
    out = torch.empty(rows, dtype=torch.float32, device="cuda")
    for _ in range(3):
        ctx.mlp_forward(feat, out, stream)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.mlp_forward(feat, out, stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    flops = 2 * (4 * 64 + 64 * 64 + 64 * 1) * rows
    tensor = 2 * 64 * 64 * rows
    peak, src = bf16_peak()
    hbm, hsrc = peaks()
    return {"rows": rows, "ms": ms, "rows_per_s": rows / (ms * 1e-3),
            "tflops_all_layers": flops / (ms * 1e-3) / 1e12,
            "tensor_tflops": tensor / (ms * 1e-3) / 1e12,
            "tensor_frac": tensor / (ms * 1e-3) / 1e12 / peak, "bf16_peak": peak,
            "bf16_peak_source": src,
            "hbm_gbs": 20 * rows / (ms * 1e-3) / 1e9, "hbm_frac": 20 * rows / (ms * 1e-3) / 1e9 / hbm,
            "timing": "CUDA events, median of 5 calls"}


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


def _eigen_of(prob):
    """Fission banking for the oracle when the workload is a k-eigenvalue one
    (a first generation from the box source)."""
    if getattr(prob, "nu", None) is None:
        return None
    return dict(nu=prob.nu, f_fis=prob.f_fis, k_norm=1.0, max_sites=255)


def oracle_rate(prob, budget_s, threads, batch=0, cap=None, geom_index=0):
    """Particles/s of the CPU oracle on a bounded sample (the first ids of a
    batch of problem `geom_index`); also returns the sample's result."""
    import oracle
    n = 2000
    kw = dict(seed=prob.seed, batch=batch, threads=threads, eigen=_eigen_of(prob),
              geom_index=geom_index, problem_index=geom_index)
    t = time.perf_counter()
    oracle.run(prob, n=n, **kw)
    dt = time.perf_counter() - t
    n = int(max(2000, min(budget_s / max(dt, 1e-6) * n, cap or prob.n_particles[geom_index])))
    t = time.perf_counter()
    res = oracle.run(prob, n=n, **kw)
    dt = time.perf_counter() - t
    return n / dt, n, dt, res


def kernel_source_sha():
    import hashlib
    h = hashlib.sha1()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_key(config, precision, sparse):
    return f"config{config}-{'fp32' if precision == 1 else 'fp64'}-w{int(sparse)}"


def recorded_traffic(config, precision, sparse):
    """The recorded lookup traffic of this workload, or None (no record, or
    one taken on other kernel sources)."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f).get(traffic_key(config, precision, sparse))
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sha") != kernel_source_sha():
        return None
    return rec


def record_traffic(csv_path, config, precision, sparse, command):
    """Sums the DRAM and L2 bytes of every lookup launch in an ncu CSV log
    (metrics dram__bytes_read.sum, dram__bytes_write.sum, lts__t_bytes.sum)
    into TRAFFIC_FILE under this workload's key."""
    import csv
    rows = []
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if "k_lookup" not in r.get("Kernel Name", ""):
            continue
        rows.append(r)
    if not rows:
        raise SystemExit(f"no lookup launches in {csv_path}")
    unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1024, "MB": 1 << 20,
            "GB": 1 << 30}
    tot = {}
    launches = set()
    for r in rows:
        launches.add(r["ID"])
        v = float(r["Metric Value"].replace(",", "")) * unit.get(r.get("Metric Unit", "byte"), 1)
        tot[r["Metric Name"]] = tot.get(r["Metric Name"], 0.0) + v
    dram = tot.get("dram__bytes_read.sum", 0.0) + tot.get("dram__bytes_write.sum", 0.0)
    data = {}
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            data = json.load(f)
    data[traffic_key(config, precision, sparse)] = {
        "dram_bytes_per_batch": dram, "l2_bytes_per_batch": tot.get("lts__t_bytes.sum"),
        "launches": len(launches), "kernel_sha": kernel_source_sha(), "command": command}
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(data[traffic_key(config, precision, sparse)]))


def compare_outcomes(gpu, ref):
    """Counts of identical per-particle outcomes (floats as bit patterns)."""
    n = len(ref["n_coll"])
    same = np.ones(n, dtype=bool)
    fields = {}
    for k in ("n_coll", "status", "n_flights", "n_draws", "E", "x", "y", "z"):
        a, b = np.asarray(gpu[k])[:n], np.asarray(ref[k])
        eq = a.view(np.int64) == b.view(np.int64) if a.dtype == np.float64 else a == b
        fields[k] = int(eq.sum())
        same &= eq
    return int(same.sum()), fields


def tally_error(gpu_flux, ref_flux):
    nz = ref_flux > 0
    rel = np.abs(gpu_flux[nz] - ref_flux[nz]) / ref_flux[nz]
    return {"max_rel": float(rel.max()) if rel.size else 0.0,
            "scored_where_oracle_zero": int(np.count_nonzero(gpu_flux[~nz])),
            "bins_compared": int(nz.sum())}


def parity_record(ctx, geom, prob, n, ref, precision, stream):
    """The GPU on the oracle sample's histories (batch 0, problem 0, ids
    [0, n)) against the oracle's result for them."""
    from paper_2403_12345_gb300 import gbmc
    ctx.reset_tallies(stream)
    ctx.run_problems([gbmc.problem(geom, prob.seed, n, batch=0, problem_index=0)], stream)
    flux, counts, _ = ctx.read_tallies(0)
    out = ctx.read_outcomes(0, 0, n)
    same, fields = compare_outcomes(out, ref)
    te = tally_error(flux, ref["flux"])
    return {"against": "oracle (history-based CPU definition), same histories",
            "precision": "fp32" if precision == 1 else "fp64", "batch": 0, "problem": 0,
            "ids": n, "outcomes_identical": same, "identical_per_field": fields,
            "flux_per_bin": te, "scalar_counts_equal": bool(np.array_equal(counts, ref["counts"])),
            "gate": "every outcome bit for bit; flux per bin within 1e-12 relative",
            "pass": bool(same == n and te["max_rel"] <= 1e-12
                         and te["scored_where_oracle_zero"] == 0
                         and np.array_equal(counts, ref["counts"]))}


def fp32_vs_fp64_record(stream, local, steps=3):
    """The 17x17 lattice at 1e7 particles per batch with binary32 tables
    against binary64 tables: throughput of each (autotuned, CUDA events, L2
    flushed between batches), and the binary32 tally error on the same
    histories against the binary64 path (whose outcomes are the oracle's bit
    for bit and tallies its to 1e-12: the parity record)."""
    import torch
    from paper_2403_12345_gb300 import gbmc
    prob = synth.make_config(3)
    n = prob.n_particles[0]
    geom = gbmc.geometry_from(prob.geom)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    with gbmc.Context(local) as ctx:
        ctx.load(prob, (gbmc.FP64, gbmc.FP32))
        for prec in (gbmc.FP64, gbmc.FP32):
            ctx.set_options(precision=prec)
            ctx.autotune([gbmc.problem(geom, prob.seed, n, batch=40_000)], fraction=0.1,
                         stream=stream)
            ctx.run_batch(gbmc.problem(geom, prob.seed, n, batch=10_000), stream)
            ms, clocks = _timed(lambda k: ctx.run_batch(gbmc.problem(geom, prob.seed, n,
                                                                     batch=1 + k), stream),
                                steps, flush, stream, local)
            ctx.reset_tallies(stream)
            ctx.run_batch(gbmc.problem(geom, prob.seed, n, batch=0), stream)
            flux, _, _ = ctx.read_tallies(0)
            o = ctx.read_outcomes(0, 0, n)
            res[prec] = dict(rate=n * steps / (sum(ms) * 1e-3), flux=flux,
                             n_coll=o["n_coll"].copy(), status=o["status"].copy(), clocks=clocks)
    f32, f64 = res[gbmc.FP32]["flux"], res[gbmc.FP64]["flux"]
    nz = f64 > 0
    per_bin = np.abs(f32[nz] - f64[nz]) / f64[nz]
    l2 = float(np.linalg.norm(f32 - f64) / np.linalg.norm(f64))
    div = float(np.mean((res[gbmc.FP32]["n_coll"] != res[gbmc.FP64]["n_coll"]) |
                        (res[gbmc.FP32]["status"] != res[gbmc.FP64]["status"])))
    r32, r64 = res[gbmc.FP32]["rate"], res[gbmc.FP64]["rate"]
    return {"workload": "17x17 lattice, 1e7 particles per batch, same histories in both",
            "fp64_particles_per_s": r64, "fp32_particles_per_s": r32, "ratio": r32 / r64,
            "tally": "flux [289 cells x 200 bins], batch 0",
            "l2_rel_err": l2, "per_bin_rel_err_p50": float(np.median(per_bin)),
            "per_bin_rel_err_p99": float(np.percentile(per_bin, 99)),
            "diverged_walk_fraction": div, "gate_l2": FP32_TALLY_L2_GATE,
            "pass": l2 <= FP32_TALLY_L2_GATE, "clocks_fp32": res[gbmc.FP32]["clocks"]}


def stress_measure(prec, nq, steps, warmup, stream, local, seed_offset=0, e2e_steps=3,
                   barrier=None, search=1, sparse=0):
    """Lookup-only stress set: lookups/s through gbmc_lookup_macro (the
    library's sort included), the lookup kernel alone on sorted queries
    (roofline), and end to end from pinned host memory."""
    import torch
    from paper_2403_12345_gb300 import gbmc
    prob, E, mat = synth.make_stress_lookup(n_queries=nq, seed_offset=seed_offset)
    micro_per = int(prob.mat_off[1] - prob.mat_off[0])
    ctx = gbmc.Context(local, precision=prec, search=search, sparse_windows=sparse)
    ctx.load(prob, (prec,))
    dE = torch.from_numpy(E).cuda()
    dm = torch.from_numpy(mat).cuda()
    st = torch.empty_like(dE)
    sa = torch.empty_like(dE)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        ctx.lookup_macro(dE, dm, st, sa, precision=prec, sort=True, stream=stream)
    if barrier:
        barrier()
    ms, clocks = _timed(lambda k: ctx.lookup_macro(dE, dm, st, sa, precision=prec, sort=True,
                                                   stream=stream), steps, flush, stream, local)
    # the lookup kernel alone: queries in sorted order, no library sort
    order = np.argsort(E, kind="stable")
    dEs = torch.from_numpy(E[order]).cuda()
    for _ in range(2):
        ctx.lookup_macro(dEs, dm, st, sa, precision=prec, sort=False, stream=stream)
    kms, _ = _timed(lambda k: ctx.lookup_macro(dEs, dm, st, sa, precision=prec, sort=False,
                                               stream=stream), steps, flush, stream, local)
    lk_ms = statistics.median(kms)
    alg = nq * (micro_per * BRACKET_BYTES[prec] + LOOKUP_IO_BYTES)
    hbm, peak_src = peaks()
    gbs = alg / (lk_ms * 1e-3) / 1e9
    if prec == 0:
        # binary64 tables: bound by the binary64 pipe; the algorithmic six
        # operations per micro lookup against the library's measured rate
        fp64_rate = ctx.measure_fp64_rate()
        ops = nq * micro_per * ALGO_FP64_OPS_PER_MICRO
        fp64_roof = {"bound": "alu", "achieved": ops / (lk_ms * 1e-3) / 1e9,
                     "peak": fp64_rate / 1e9, "unit": "G binary64 op/s",
                     "frac": ops / (lk_ms * 1e-3) / fp64_rate,
                     "peak_source": "measured: gbmc_measure_fp64_rate (binary64 fused "
                                    "multiply-add chains, CUDA events)",
                     "ops_per_micro_lookup": ALGO_FP64_OPS_PER_MICRO,
                     "issued_binary64_frac": nq * micro_per * ISSUED_FP64_PER_MICRO
                     / (lk_ms * 1e-3) / fp64_rate,
                     "issued_per_micro_lookup": ISSUED_FP64_PER_MICRO}
    else:
        fp64_roof = None
    hE = torch.from_numpy(E).pin_memory()
    hst = torch.empty(nq, dtype=torch.float64).pin_memory()
    hsa = torch.empty(nq, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dE.copy_(hE, non_blocking=True)
        ctx.lookup_macro(dE, dm, st, sa, precision=prec, sort=True, stream=stream)
        hst.copy_(st, non_blocking=True)
        hsa.copy_(sa, non_blocking=True)
        torch.cuda.synchronize()
    e2e = nq * e2e_steps / (time.perf_counter() - t0)
    ctx.close()
    roof = {"kernel": "lookup (sorted queries, no library sort)", "bound": "hbm",
            "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "traffic": None, "peak_source": peak_src, "launches": 1,
            "avg_launch_ms": lk_ms, "algorithmic_bytes_per_launch": alg,
            "table_bytes": int(prob.table_bytes(prec))}
    if fp64_roof:
        hbm_rec = {k: roof[k] for k in ("achieved", "peak", "unit", "frac", "peak_source",
                                         "algorithmic_bytes_per_launch")}
        roof.update(fp64_roof)
        roof["hbm"] = hbm_rec
        del roof["algorithmic_bytes_per_launch"]
    return {"prob": prob, "E": E, "micro_per": micro_per, "ms": ms, "clocks": clocks,
            "e2e": e2e, "roofline": roof}


def run_reference(args, prob, rank):
    if rank != 0:
        return
    threads = len(os.sched_getaffinity(0))
    import oracle
    # size a step to ~budget seconds of oracle work
    _, n, dt, _ = oracle_rate(prob, args.ref_step_s, threads)
    for w in range(args.warmup):
        oracle.run(prob, seed=prob.seed, batch=100 + w, n=min(n, 2000), threads=threads,
                   eigen=_eigen_of(prob))
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        oracle.run(prob, seed=prob.seed, batch=k, n=n, threads=threads, eigen=_eigen_of(prob))
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


def _timed(ctx_call, steps, flush, stream, clk_index):
    """CUDA-event times (ms) of `steps` calls of ctx_call(k), with an L2 flush
    before each, and the clocks sampled meanwhile."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    with Clocks(clk_index) as clk:
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            ctx_call(k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], clk.summary()


def _max_over_ranks(x, world):
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def run_stress(args, rank, world, local):
    """Lookup-only stress set: one step = the macroscopic lookup of every query
    (sorted by the library, then looked up) through gbmc_lookup_macro."""
    import torch
    from paper_2403_12345_gb300 import gbmc
    prec = 1 if args.precision < 0 else args.precision
    nq = args.particles or 10_000_000
    prob, E, mat = synth.make_stress_lookup(n_queries=nq, seed_offset=rank)
    micro_per = int(prob.mat_off[1] - prob.mat_off[0])
    bracket = BRACKET_BYTES[prec]
    cfg = {"workload": prob.name, "description": WORKLOADS[6], "queries_per_step": nq,
           "table_precision": "fp32" if prec == 1 else "fp64", "nuclides": int(prob.n_nuc),
           "grid_points": int(prob.grid_off[-1]), "nuclides_in_material": micro_per,
           "table_bytes": int(prob.table_bytes(prec)),
           "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas{args.gpus}"}
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        n = 2000
        t = time.perf_counter()
        oracle.macro(prob, 0, E[:n], precision=prec)
        dt = time.perf_counter() - t
        n = int(min(nq, max(2000, args.ref_step_s / max(dt, 1e-6) * n)))
        times = []
        for k in range(args.steps):
            t = time.perf_counter()
            oracle.macro(prob, 0, E[k * 7919 % max(1, nq - n):][:n], precision=prec)
            times.append(time.perf_counter() - t)
        value = n * args.steps / sum(times)
        print(json.dumps({
            "impl": "reference", "metric": "XS lookups/s", "value": value, "unit": "lookups/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == 1 else "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "lookups/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} queries per step"},
            "e2e": {"value": value, "unit": "lookups/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}), flush=True)
        return
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    m = stress_measure(prec, nq, args.steps, args.warmup, stream, local, seed_offset=rank,
                       e2e_steps=args.e2e_steps,
                       barrier=(lambda: dist.barrier()) if world > 1 else None,
                       sparse=max(args.sparse_windows, 0))
    tot_ms = _max_over_ranks(sum(m["ms"]), world)
    value = nq * args.steps * world / (tot_ms * 1e-3)
    # end to end, whole job: every rank's queries over the slowest rank's time
    e2e_steps = max(1, args.e2e_steps)
    e2e = nq * e2e_steps * world / _max_over_ranks(nq * e2e_steps / m["e2e"], world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        n = 2000
        t = time.perf_counter()
        oracle.macro(prob, 0, E[:n], precision=prec)
        n = int(min(nq, max(2000, args.cpu_budget_s / max(time.perf_counter() - t, 1e-6) * n)))
        t = time.perf_counter()
        oracle.macro(prob, 0, E[:n], precision=prec)
        dt = time.perf_counter() - t
        cpu = {"value": n / dt, "unit": "lookups/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n} queries ({dt:.1f} s, one thread)"}
    if rank == 0:
        print(json.dumps({
            "metric": "XS lookups/s", "value": value, "unit": "lookups/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == 1 else "f64", "data": "synthetic", "config": cfg,
            "micro_lookups_per_s": value * micro_per,
            "e2e": {"value": e2e, "unit": "lookups/s", "h2d_bytes_per_step": nq * 8,
                    "d2h_bytes_per_step": nq * 16},
            "roofline": m["roofline"],
            "cpu_baseline": cpu, "clocks": m["clocks"],
            "gpu_launches": 4 * args.steps}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_eigen(args, prob, rank, world, local):
    """k-eigenvalue power iteration: `warmup` inactive generations (the first
    from the box source), then `steps` timed active generations, each from the
    previous generation's fission bank (kept on the device) with the yield
    normalised by the previous estimate.  Replicas split each generation's
    ids and exchange their banks between generations."""
    import torch
    import torch.distributed as dist
    from paper_2403_12345_gb300 import gbmc, replicas
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    N = prob.n_particles[0]
    ctx = gbmc.Context(local, precision=args.precision, sort=args.sort)
    ctx.load(prob, (args.precision,))
    ctx.load_fission(prob.nu, prob.f_fis)
    g_box = gbmc.geometry_from(prob.geom)
    g_bank = gbmc.geometry_from(prob.geom)
    g_bank.source = gbmc.SRC_BANK
    first, n = replicas.id_range(0, N, rank, world)
    state = {"k": 1.0, "gen": 0}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def generation(_k=None):
        gen = state["gen"]
        ctx.set_eigen(state["k"], 64)
        g = g_box if gen == 0 else g_bank
        ctx.run_batch(gbmc.problem(g, prob.seed, n, batch=gen, first_id=first), stream)
        state["gen"] = gen + 1

    def next_source():
        if world > 1:
            bank = replicas.gather_bank(ctx.read_bank())
            ctx.set_source_bank(bank, N)
            size = len(bank)
        else:
            size = ctx.read_bank(sites=False)
            ctx.set_source_bank(None, N)
        k = size / N * state["k"]
        state["k"] = k
        return k

    for _ in range(max(args.warmup, 1)):
        generation()
        next_source()
    if world > 1:
        dist.barrier()
    ks, ms_all = [], []
    clocks = None
    for k_step in range(args.steps):
        ms, clocks = _timed(lambda _k: generation(), 1, flush, stream, local)
        ms_all.append(ms[0])
        ks.append(next_source())        # outside the timed region (bank exchange, k)
    tot_ms = _max_over_ranks(sum(ms_all), world)
    value = N * args.steps / (tot_ms * 1e-3)
    kk = np.array(ks)
    if rank == 0:
        cfg = {"workload": prob.name, "description": WORKLOADS[7], "particles_per_generation": N,
               "inactive_generations": max(args.warmup, 1), "active_generations": args.steps,
               "table_precision": "fp32" if args.precision == 1 else "fp64",
               "nuclides": int(prob.n_nuc), "l2": "flushed between timed generations (256 MiB write)",
               "parallelism": f"replicas{args.gpus}"}
        print(json.dumps({
            "metric": "particles/s", "value": value, "unit": "particles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if args.precision == 1 else "f64", "data": "synthetic", "config": cfg,
            "k_eff": {"mean": float(kk.mean()),
                      "std_err": float(kk.std(ddof=1) / np.sqrt(len(kk))) if len(kk) > 1 else None,
                      "per_generation": [float(x) for x in kk]},
            "e2e": None, "roofline": None, "cpu_baseline": None, "clocks": clocks,
            "gpu_launches": None}), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_windows(args, prob, rank, world, local):
    """Deep-penetration slab: learned weight windows against analog.  One step
    = one batch with the learned windows; the figure of merit FOM = 1/(R^2 T)
    of the far-face leakage is reported for both methods."""
    import torch
    import torch.distributed as dist
    from paper_2403_12345_gb300 import gbmc
    from paper_2403_12345_gb300 import importance as imp
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    g = gbmc.geometry_from(prob.geom)
    ctx = gbmc.Context(local)
    ctx.load(prob)
    n_an = 4_000_000
    n_ww = args.particles or 400_000
    off = 100_000 * rank
    analog = lambda b: gbmc.problem(g, prob.seed, n_an, batch=off + b)
    learned = lambda b: gbmc.problem(g, prob.seed, n_ww, batch=off + b)
    t0 = time.perf_counter()
    lw = imp.LearnedWindows(ctx, g, prob.edges, seed=5)
    lw.collect(analog, range(50_000, 50_004), capacity=16_000_000, stream=stream)
    loss = lw.train(steps=1500, lr=3e-3, stream=stream)
    lw.apply(stream=stream)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for w in range(args.warmup):
        ctx.run_batch(learned(60_000 + w), stream)
    if world > 1:
        dist.barrier()
    ms, clocks = _timed(lambda k: ctx.run_batch(learned(k), stream), args.steps, flush, stream,
                        local)
    tot_ms = _max_over_ranks(sum(ms), world)
    value = n_ww * args.steps * world / (tot_ms * 1e-3)
    fw = imp.figure_of_merit(ctx, learned, range(1000, 1020), n_ww, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.e2e_steps)
    for k in range(e2e_steps):
        ctx.run_batch(learned(2000 + k), stream)
        flux, _, _ = ctx.read_tallies(0)
    # whole job: every rank's batches over the slowest rank's time
    e2e = n_ww * e2e_steps * world / _max_over_ranks(time.perf_counter() - t0, world)
    ctx.clear_weight_windows()
    fa = imp.figure_of_merit(ctx, analog, range(3000, 3020), n_an, stream)
    mlp = mlp_forward_measure(ctx, stream)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = len(os.sched_getaffinity(0))
        rate, n, dt, _ = oracle_rate(prob, args.cpu_budget_s, threads)
        cpu = {"value": rate, "unit": "particles/s", "cores": threads, "kind": "oracle",
               "sample": f"first {n} analog histories of batch 0 ({dt:.1f} s)"}
    if rank == 0:
        se = float(np.hypot(fa["mean"] * fa["rel_err"], fw["mean"] * fw["rel_err"]))
        print(json.dumps({
            "metric": "particles/s", "value": value, "unit": "particles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": prob.name, "description": WORKLOADS[5],
                       "particles_per_batch": n_ww, "analog_particles_per_batch": n_an,
                       "table_precision": "fp64", "nuclides": int(prob.n_nuc),
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas{args.gpus}"},
            "fom": {"analog": fa["fom"], "learned": fw["fom"], "ratio": fw["fom"] / fa["fom"],
                    "analog_leak_far": [fa["mean"], fa["mean"] * fa["rel_err"]],
                    "learned_leak_far": [fw["mean"], fw["mean"] * fw["rel_err"]],
                    "z": (fw["mean"] - fa["mean"]) / se if se > 0 else None,
                    "batches": 20, "train_loss": loss, "setup_s": setup_s},
            "mlp_forward": mlp,
            "e2e": {"value": e2e, "unit": "particles/s",
                    "h2d_bytes_per_step": ctypes.sizeof(gbmc.Problem),
                    "d2h_bytes_per_step": int(flux.nbytes + 16 * gbmc.NSCAL)},
            "roofline": None,
            "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": None}), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


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
                    help="1: autotune launch settings before timing, 0: defaults "
                         "(default: autotune configs 2-4)")
    ap.add_argument("--search", type=int, default=1,
                    help="grid search: 1 coarse index (default), -1 plain binary search")
    ap.add_argument("--loops", type=int, default=0,
                    help="concurrent event loops over the steps' batches (gbmc_run_concurrent); "
                         "0: the fastest of 1-6 in a short trial after autotuning")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sub-records of the default run (binary32 against binary64 "
                         "at 1e7 particles, the lookup-only stress set)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="set up as the timed run does, then run one eager profiled batch at "
                         "the command line's options (no autotuning, no graph launches) and "
                         "exit: the command the lookup-traffic ncu capture wraps")
    ap.add_argument("--record-traffic", metavar="NCU_CSV",
                    help="sum the lookup launches' DRAM/L2 bytes of an ncu CSV log of "
                         "--profile-batch into the traffic file for this workload and exit")
    ap.add_argument("--sparse-windows", type=int, default=-1,
                    help="binary32 window form (0: 64-byte windows, 1: short windows) of the "
                         "lookup-only stress set (config 6), and with --profile-batch or "
                         "--record-traffic of the captured batch")
    ap.add_argument("--mlp-forward-only", action="store_true",
                    help="time the importance network's tensor-core forward alone (random "
                         "BF16 weights, 2^24 random feature rows) and exit: the command an ncu "
                         "capture of that kernel wraps")
    ap.add_argument("--ncu-command", default="",
                    help="with --record-traffic: the capture command, kept with the record")
    args = ap.parse_args()
    if args.record_traffic:
        prec = args.precision if args.precision >= 0 else (0 if args.config in (1, 2) else 1)
        record_traffic(args.record_traffic, args.config, prec, max(args.sparse_windows, 0),
                       args.ncu_command)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.mlp_forward_only:
        import torch
        from paper_2403_12345_gb300 import gbmc
        torch.cuda.set_device(local)
        ctx = gbmc.Context(local)
        g = torch.Generator().manual_seed(7)
        w = (torch.randn(gbmc.MLP_NPARAM, generator=g) * 0.2).to(torch.bfloat16)
        ctx.set_importance_net(w.view(torch.int16).numpy().view(np.uint16), np.zeros(4), np.ones(4))
        print(json.dumps({"mlp_forward": mlp_forward_measure(ctx, torch.cuda.current_stream())}),
              flush=True)
        ctx.close()
        return
    if args.config == 6:
        run_stress(args, rank, world, local)
        return
    if args.config == 7:
        prob = synth.make_eigen_lattice(n_particles=args.particles or 1_000_000)
        if args.precision < 0:
            args.precision = prob.precision
        if args.impl == "reference":
            run_reference(args, prob, rank)
        else:
            run_eigen(args, prob, rank, world, local)
        return
    prob = synth.make_config(args.config, n_particles=args.particles or None)
    if args.precision < 0:
        args.precision = prob.precision
    npart = prob.n_particles[0]

    if args.impl == "reference":
        run_reference(args, prob, rank)
        return
    if args.config == 5:
        run_windows(args, prob, rank, world, local)
        return

    import torch
    import torch.distributed as dist
    from paper_2403_12345_gb300 import gbmc, replicas

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()

    opts = dict(precision=args.precision, sort=args.sort, search=args.search)
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

    if args.profile_batch:
        # the command an ncu capture wraps: one eager profiled batch at the
        # options given on the command line, no graph launches
        if args.sparse_windows >= 0:
            ctx.set_options(sparse_windows=args.sparse_windows)
        kt = ctx.profile_problems(problems(30_000), stream)
        print(json.dumps({"profiled_batch": {k: v[0] for k, v in kt.items()},
                          "sparse_windows": int(ctx.options.sparse_windows)}), flush=True)
        ctx.close()
        return

    tuned = None
    if args.autotune == 1 or (args.autotune < 0 and args.config in (2, 3, 4)):
        tuned = ctx.autotune(problems(40_000), fraction=0.1 if n_geo > 1 else 0.3, stream=stream)
    # the settings of one event loop (the autotuner's): the per-kernel profile
    # and the lookup roofline below run at them
    o = ctx.options
    single_opts = {"blocks_per_sm": int(o.blocks_per_sm), "tail_max": int(o.tail_max),
                   "group_lookup_max": int(o.group_lookup_max)}

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for w in range(args.warmup):
        ctx.run_problems(problems(10_000 + w), stream)
    torch.cuda.synchronize()
    # concurrent event loops (Sec. 2, "GPU Streams"): a short trial of 1-6
    # loops, each also at 4 blocks per SM, measures the rate of each with two
    # runs per loop; the timed steps then take ceil(steps / L) rounds of L
    # concurrent runs (a run costs its late iterations' latency whatever its
    # size, so a last partial round is not split), and the L with the
    # shortest predicted time wins (more loops must gain 2%)
    loops, loop_trials = max(args.loops, 1), None
    if args.loops == 0 and args.config in (1, 2, 3, 4):
        loop_trials = {}
        tuned_bps = ctx.options.blocks_per_sm
        best = None
        for L in (1, 2, 3, 4, 5, 6):
            for bps in sorted({tuned_bps, 4}):
                ctx.set_options(blocks_per_sm=bps)
                nb = 2 * L
                for rep in range(2):   # the first builds the loops' graphs
                    batch = [pr for b in range(nb) for pr in problems(50_000 + 10 * rep + b)]
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    ctx.run_concurrent(batch, n_loops=L, per_run=n_geo, stream=stream)
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t
                rate = nb * npart / dt
                loop_trials[f"{L}x{bps}"] = rate
                t_steps = -(-args.steps // L) * L * npart / rate
                if best is None or (t_steps < best[0] / 1.02 if L > best[1] else t_steps < best[0]):
                    best = (t_steps, L, bps)
        _, loops, bps = best
        ctx.set_options(blocks_per_sm=bps)
    conc_tune = None
    if loops > 1:
        def full_call(base):
            ctx.run_concurrent([pr for b in range(args.steps) for pr in problems(base + b)],
                               n_loops=loops, per_run=n_geo, stream=stream)
            torch.cuda.synchronize()

        # one untimed call of the timed configuration (as many batches on as
        # many loops): the context sizes its outcome and tally buffers for
        # the call, and each loop builds its graph on them, outside the timed
        # region
        full_call(60_000)
        if args.loops == 0:
            # the single-loop autotuner's settings, tuned again for concurrent
            # loops (their late iterations overlap, which shifts the best
            # thresholds): coordinate descent over blocks per SM, the tail
            # threshold and (binary64) the group-lookup threshold, each
            # candidate timed on one round of runs (a 1% gain to switch)
            def round_rate(opts, rep, n_loops=None):
                n_loops = n_loops or loops
                ctx.set_options(**opts)
                batch = [pr for b in range(n_loops) for pr in problems(70_000 + 20 * rep + b)]
                ctx.run_concurrent(batch, n_loops=n_loops, per_run=n_geo, stream=stream)   # graphs
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                batch = [pr for b in range(n_loops) for pr in problems(80_000 + 20 * rep + b)]
                a.record(stream)
                ctx.run_concurrent(batch, n_loops=n_loops, per_run=n_geo, stream=stream)
                e.record(stream)
                e.synchronize()
                return n_loops * npart / (a.elapsed_time(e) * 1e-3)
            o = ctx.options
            cur = {"blocks_per_sm": o.blocks_per_sm, "tail_max": o.tail_max,
                   "group_lookup_max": o.group_lookup_max}
            cands = [("blocks_per_sm", (1, 2, 3, 4)), ("tail_max", (1024, 4096, 16384))]
            if args.precision == 0:
                cands.append(("group_lookup_max", (60_000, 160_000)))
            best_rate, trials, rep = round_rate(cur, 0), {}, 1
            for key, vals in cands:
                for v in vals:
                    if v == cur[key]:
                        continue
                    trial = dict(cur, **{key: v})
                    r = round_rate(trial, rep)
                    rep += 1
                    trials[f"{key}={v}"] = r
                    if r > best_rate * 1.01:
                        best_rate, cur = r, trial
            # the loop count again at these settings (fewer blocks per loop
            # leave room for more loops): ceil(steps / L) rounds of one
            # round's time, more loops to gain 2%
            best_t = -(-args.steps // loops) * npart * loops / best_rate
            for L in (2, 3, 4, 5, 6, 7, 8, 10, 12):
                if L == loops or L > args.steps:
                    continue
                r = round_rate(cur, rep, L)
                rep += 1
                trials[f"loops={L}"] = r
                t_steps = -(-args.steps // L) * L * npart / r
                if t_steps < best_t / (1.02 if L > loops else 1.0):
                    best_t, loops = t_steps, L
            ctx.set_options(**cur)
            conc_tune = {"options": cur, "loops": loops, "round_particles_per_s": best_rate,
                         "trials": trials}
            full_call(90_000)   # the graphs at the chosen settings, outside the timed region
    ctx.reset_tallies(stream)

    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if loops > 1:
        # every step's batch in one concurrent call (batch k in tally slots
        # k n_geo ..): the steps overlap, so the time is the call's
        all_probs = [pr for k in range(args.steps) for pr in problems(k)]
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            t0 = time.perf_counter()
            e0.record(stream)
            ctx.run_concurrent(all_probs, n_loops=loops, per_run=n_geo, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        stats.append(ctx.read_stats())
        tot_ms = e0.elapsed_time(e1)
    else:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
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
        tot_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        dist.barrier()
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
    # the host; at least one batch per loop, so the loops run as concurrently
    # as in the timed region
    e2e_steps = max(1, args.e2e_steps, min(loops, args.steps))

    # result buffers in page-locked host memory from the library's allocator
    # (gbmc_host_alloc), one set per e2e batch and problem (the copies of all
    # batches are in flight together), allocated before the timed region
    def batch_dests():
        # one array per result field for the whole batch, each problem's
        # destination a contiguous slice of it (the library then copies a
        # run's results in one piece per field)
        ncs = [gbmc._n_cells(geoms[k]) * prob.n_bins for k in range(n_geo)]
        spec = {"flux": (np.float64, ncs), "counts": (np.int64, [gbmc.NSCAL] * n_geo),
                "weights": (np.float64, [gbmc.NSCAL] * n_geo),
                "n_coll": (np.int32, counts), "status": (np.int8, counts),
                "n_flights": (np.int32, counts), "n_draws": (np.uint32, counts),
                "E": (np.float64, counts), "x": (np.float64, counts),
                "y": (np.float64, counts), "z": (np.float64, counts)}
        out = [dict() for _ in range(n_geo)]
        for name, (dt, sizes) in spec.items():
            whole = gbmc.host_array(int(sum(sizes)), dt)
            at = 0
            for k in range(n_geo):
                out[k][name] = whole[at:at + sizes[k]]
                at += sizes[k]
        return out
    dests = [d for _ in range(e2e_steps) for d in batch_dests()]
    d2h = sum(a.nbytes for d in dests for a in d.values()) // e2e_steps
    # three timed repetitions on new batches each (one call of e2e_steps
    # batches lasts tens of milliseconds, where host jitter and the last
    # run's exposed copy weigh): the median is the e2e figure
    e2e_runs = []
    for rep in range(E2E_REPEATS):
        e2e_probs = [pr for k in range(e2e_steps)
                     for pr in problems(20_000 + rep * e2e_steps + k)]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        # the e2e batches through the C ABI with host destinations: each
        # run's tallies and outcomes are copied to pinned host memory as soon
        # as it ends, overlapping the runs still going (one loop: the next
        # batch)
        ctx.run_concurrent_to_host(e2e_probs, n_loops=loops, dests=dests, per_run=n_geo,
                                   stream=stream)
        stream.synchronize()
        # whole job: every rank's batches over the slowest rank's time
        e2e_runs.append(_max_over_ranks(time.perf_counter() - t0, world))
    e2e_s = sorted(e2e_runs)[len(e2e_runs) // 2]
    h2d = ctypes.sizeof(gbmc.Problem) * n_geo

    # per-kernel device times (eager launches between CUDA events) on one
    # more batch of the same workload, at one event loop's settings
    timed_opts = {k: int(getattr(ctx.options, k)) for k in single_opts}
    ctx.set_options(**single_opts)
    kt = ctx.profile_problems(problems(30_000), stream)
    pst = ctx.read_stats()
    top = max(kt, key=lambda k: kt[k][0])
    hbm, peak_src = peaks()
    lk_ms, lk_n = kt["lookup"]
    lk_bytes = pst["micro_lookups"] * BRACKET_BYTES[args.precision] + pst["lookups"] * LOOKUP_IO_BYTES
    lk_gbs = lk_bytes / (lk_ms * 1e-3) / 1e9
    stock = (args.particles == 0 and args.max_in_flight == 0 and args.blocks_per_sm == 0
             and args.sort == 1 and args.search == 1)
    tr = recorded_traffic(args.config, args.precision, ctx.options.sparse_windows) if stock else None
    l2_size = torch.cuda.get_device_properties(local).L2_cache_size
    roof = {"kernel": "lookup", "bound": "hbm", "achieved": lk_gbs, "peak": hbm, "unit": "GB/s",
            "frac": lk_gbs / hbm, "peak_source": peak_src,
            # per lookup event (one launch) of the batch, as `achieved`
            "traffic": tr["dram_bytes_per_batch"] / max(lk_n, 1) if tr else None,
            "l2_bytes": (tr["l2_bytes_per_batch"] / max(lk_n, 1)
                         if tr and tr.get("l2_bytes_per_batch") else None),
            "launches": lk_n, "avg_launch_ms": lk_ms / max(lk_n, 1),
            "algorithmic_bytes_per_launch": lk_bytes / max(lk_n, 1),
            "timing": "CUDA events around each lookup launch of one eager batch of this workload, "
                      "at the single-loop autotuned settings",
            "table_bytes": int(prob.table_bytes(args.precision)), "l2_capacity": int(l2_size)}
    if args.precision == 0:
        # binary64 tables: the algorithmic operations against the rate the
        # library's own probe measures (ncu on a full queue: DRAM under 10%,
        # binary64 pipe 41%, integer ALU 74%, issue 71%), and the binary64
        # instructions the kernel issues against the same rate
        fp64_rate = ctx.measure_fp64_rate()
        ops = pst["micro_lookups"] * ALGO_FP64_OPS_PER_MICRO
        hbm_rec = {k: roof[k] for k in ("achieved", "peak", "unit", "frac", "peak_source",
                                         "algorithmic_bytes_per_launch")}
        roof.update({"bound": "alu", "achieved": ops / (lk_ms * 1e-3) / 1e9,
                     "peak": fp64_rate / 1e9, "unit": "G binary64 op/s",
                     "frac": ops / (lk_ms * 1e-3) / fp64_rate,
                     "peak_source": "measured: gbmc_measure_fp64_rate (binary64 fused "
                                    "multiply-add chains, CUDA events)",
                     "algorithmic_ops_per_launch": ops / max(lk_n, 1),
                     "ops_per_micro_lookup": ALGO_FP64_OPS_PER_MICRO,
                     "issued_binary64_frac": pst["micro_lookups"] * ISSUED_FP64_PER_MICRO
                     / (lk_ms * 1e-3) / fp64_rate,
                     "issued_per_micro_lookup": ISSUED_FP64_PER_MICRO, "hbm": hbm_rec})
        del roof["algorithmic_bytes_per_launch"]
    if timed_opts != single_opts:
        # the same batch at the settings the concurrent loops were timed at
        # (tuned for several loops whose late iterations overlap; one loop
        # alone runs its lookups at them less efficiently)
        ctx.set_options(**timed_opts)
        kt2 = ctx.profile_problems(problems(30_000), stream)
        ms2 = kt2["lookup"][0]
        roof["at_timed_settings"] = {"settings": timed_opts, "lookup_ms_per_batch": ms2,
                                     "frac": roof["frac"] * lk_ms / ms2}
    ctx.set_options(**timed_opts)

    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = len(os.sched_getaffinity(0))
        rate, n, dt, ref = oracle_rate(prob, args.cpu_budget_s, threads)
        cpu = {"value": rate, "unit": "particles/s", "cores": threads, "kind": "oracle",
               "sample": f"first {n} histories of batch 0 of problem 0 ({dt:.1f} s)"}
        parity = parity_record(ctx, geoms[0], prob, n, ref, args.precision, stream)

    run_bps = int(ctx.options.blocks_per_sm)
    extras = {}
    if rank == 0 and args.config == 2 and stock and not args.no_extras:
        # the coarse index against a plain binary search of each grid, on the
        # lookup kernel of one eager batch each (same histories, same results),
        # at one event loop's autotuned settings as the roofline
        ctx.set_options(search=-1, **single_opts)
        kp = ctx.profile_problems(problems(30_000), stream)
        ctx.set_options(search=1)
        ki = ctx.profile_problems(problems(30_000), stream)
        search_cmp = {"lattice17_fp64_lookup_ms_per_batch": {"index": ki["lookup"][0],
                                                             "plain": kp["lookup"][0]},
                      "settings": dict(single_opts)}
        ctx.close()
        ctx = None
        extras["fp32_vs_fp64"] = fp32_vs_fp64_record(stream, local)
        m = stress_measure(1, 10_000_000, args.steps, args.warmup, stream, local)
        mp = stress_measure(1, 10_000_000, 3, 1, stream, local, e2e_steps=1, search=-1)
        search_cmp["stress_fp32_lookup_kernel_ms"] = {
            "index": m["roofline"]["avg_launch_ms"], "plain": mp["roofline"]["avg_launch_ms"]}
        extras["search_comparison"] = search_cmp
        extras["lookup_stress_fp32"] = {
            "workload": m["prob"].name, "description": WORKLOADS[6],
            "lookups_per_s": 10_000_000 * args.steps / (sum(m["ms"]) * 1e-3),
            "micro_lookups_per_s": 10_000_000 * m["micro_per"] * args.steps / (sum(m["ms"]) * 1e-3),
            "roofline": m["roofline"], "clocks": m["clocks"]}

    runs = args.steps if loops > 1 else 1   # graph launches per entry of stats
    launches = sum(2 * runs + ITER_KERNELS[args.precision] * s["iterations"]
                   for s in stats)   # + init and tail per run
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
            "e2e": {"value": npart * e2e_steps * world / e2e_s, "unit": "particles/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "batches_per_run": e2e_steps,
                    "runs_particles_per_s": [npart * e2e_steps * world / t for t in e2e_runs],
                    "statistic": f"median of {E2E_REPEATS} timed calls"},
            "autotune": tuned,
            "concurrent_loops": {"loops": loops, "blocks_per_sm": run_bps,
                                 "trial_particles_per_s": loop_trials,
                                 "concurrent_tuning": conc_tune,
                                 "how": "gbmc_run_concurrent: the steps' batches spread over this "
                                        "many event loops on their own streams (Sec. 2 'GPU "
                                        "Streams'); one loop: one graph launch per step"},
            "roofline": roof,
            "kernel_ms_per_batch": {k: v[0] for k, v in kt.items()},
            "events_per_batch": {k: pst[k] for k in ("lookups", "micro_lookups", "flights",
                                                     "crossings", "collisions", "histories",
                                                     "handoffs")},
            "top_kernel": top,
            "cpu_baseline": cpu,
            "parity": parity,
            "clocks": clk.summary(),
            "gpu_launches": launches,
        }
        if loops > 1:
            line["config"]["l2"] = ("flushed once before the timed call (256 MiB write); the "
                                    "steps' batches overlap on the loops, each with a working set "
                                    "(tables, particle bank, running sums) beyond the L2")
            line["config"]["parallelism"] += f" x {loops} concurrent event loops"
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
