#!/usr/bin/env python
"""Benchmark: pairwise interactions/s of direct-sum N-body + velocity Verlet.

Workload (the paper's 10,425-body Solar-System model, Section 2, as seeded
synthetic stand-in): N = 10,425 bodies (Sun, 30 major bodies, 100 moons,
10,294 main-belt asteroids), dt = 0.1 day.  One benchmark "step" is one
``nbody_step(S)`` call advancing the system by S velocity-Verlet steps
(FP64: S = 10, i.e. one day; mixed: S = 100); each Verlet step is an Eq. 1
force launch and a per-body Verlet launch (kick, drift, staging), chained
with programmatic dependent launch and replayed from CUDA graphs.  The
headline ``value`` is the FP64 path (the paper's arithmetic); the mixed path
is measured the same way and reported under "mixed" with its speed-up.  Each
roofline object describes that path's force kernel: its flops per launch
over its mean event-timed duration (the same workload, each kernel launched
alone by ``nbody_kernel_times``).

    interactions/s = N (N - 1) * S * K / (timed seconds)

Timing: W untimed warm-up steps, then K timed steps, each bracketed by CUDA
events on the stream the library launches on; L2 is flushed (256 MB write)
between timed steps, outside the events.  Multi-GPU (torchrun): every rank
runs an independent replica (no collective on the data path, weak scaling);
the barrier-bracketed elapsed time is the max over ranks.

``--impl reference`` times the FP64 C oracle (OpenMP build, all host cores)
on the same workload and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pairwise interactions/s"
UNIT = "interactions/s"
FLOPS_PER_INTERACTION = 20  # 3 sub, 5 for |d|^2, 1 rsqrt, 2 cube, 1 mu*s, 6 for the 3 FMAs
# Derived CUDA-core peaks of one GB300 (152 SMs at the 2070 MHz maximum clock):
# FP32 128 FMA lanes/SM/clk -> 80.5 TFLOP/s; FP64 2 FMA lanes/SM/clk -> 1.26 TFLOP/s.
SMS, MAX_MHZ = 152, 2070.0
PEAK_TFLOPS = {"mixed": SMS * 128 * 2 * MAX_MHZ * 1e6 * 1e-12, "fp64": SMS * 2 * 2 * MAX_MHZ * 1e6 * 1e-12}
# The paper's production run (Section 4): 1e4-body model, 1000 steps in about
# 23 minutes on 176 CPU processors -> 10,425 * 10,424 * 1000 / 1380 s.
PAPER_INTERACTIONS_PER_S = 7.9e7
# DRAM bytes per launch of the force kernel from one ncu capture (ncu flushes
# the caches before each replay, so these are cold-L2 figures; in the timed
# loop the state is L2-resident), keyed by a hash of the kernel sources they
# were taken on (null once the sources change).
NCU_TRAFFIC = {("f543b52654f59900", "mixed"): 1070592, ("f543b52654f59900", "fp64"): 606208}


def kernel_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2112_15079_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.startswith(("step_", "nbody_dev", "sym")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=10425, help="bodies (10425 = the paper's model)")
    ap.add_argument("--inner", type=int, default=100, help="Verlet steps per benchmark step (mixed)")
    ap.add_argument("--inner-fp64", type=int, default=10, help="Verlet steps per benchmark step (FP64)")
    ap.add_argument("--no-mixed", action="store_true", help="time the FP64 path only (the headline)")
    ap.add_argument("--only", choices=["mixed", "fp64"], default=None, help="time one precision only")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tiles", default=None,
                    help='JSON work decomposition for both precisions, e.g. {"threads":1024,"ipt":1,"tj":512,'
                         '"jsplit":4,"ctas_per_sm":1}; skips the autotuner')
    ap.add_argument("--tiles-fp64", default=None, help="JSON work decomposition for the FP64 path only")
    ap.add_argument("--no-pair-once", action="store_true",
                    help="the force kernel that evaluates every ordered pair, in both precisions (NBODY_FLAG_NO_SYM)")
    ap.add_argument("--pair-once-block", type=int, default=0,
                    help="bodies (FP64) or stage entries (mixed) per block of the pair-once kernels; 0 = automatic")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint, 31-body and ensemble measurements")
    ap.add_argument("--adjoint-steps", type=int, default=1000,
                    help="trajectory length of the adjoint timing (mixed; FP64 runs a fifth of it)")
    ap.add_argument("--ensemble-systems", type=int, default=256)
    ap.add_argument("--sweep", action="store_true", help="also time N = 16,384 / 65,536 / 262,144 / 1,048,576")
    ap.add_argument("--dt-sweep", action="store_true",
                    help="also report the maximum energy drift against dt (FP64 and mixed, no moons)")
    ap.add_argument("--close", type=float, default=0.0, metavar="THETA_C",
                    help="with --only: time the path with close-encounter handling (close_omega_dt = THETA_C, "
                         "substep_omega_dt = 0.05); no roofline (nbody_kernel_times covers plain Verlet)")
    ap.add_argument("--shard", action="store_true",
                    help="row shards instead of replicas: under torchrun every rank steps its own bodies of ONE "
                         "system (FP64, or --only mixed) and an all-gather per Verlet step exchanges the staged "
                         "positions (strong scaling)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (timing only; no collective touches the data path)
# ---------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def max_over_ranks(value: float, dist, device=None) -> float:
    """Max of a per-rank float over all ranks (identity without a group)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
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

    def summary(self) -> dict:
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        load = [v for v in sm if mx and v >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(num(r[3]) or 0 for r in rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def time_oracle(system, seconds: float, max_steps: int = 1000):
    """Velocity-Verlet steps of the oracle (OpenMP build) for about `seconds`."""
    import oracle

    t0 = time.perf_counter()
    r, v, a = oracle.verlet(system.G, system.dt, 1, system.r, system.v, system.m, openmp=True)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(max_steps, seconds / max(t1, 1e-9))))
    t0 = time.perf_counter()
    oracle.verlet(system.G, system.dt, n, r, v, system.m, a, openmp=True)
    dt = time.perf_counter() - t0
    N = system.n
    return {"value": N * (N - 1) * n / dt, "unit": UNIT, "cores": oracle.threads(True), "kind": "oracle",
            "sample": f"{n} velocity-Verlet steps of the N={N} system (FP64 C oracle, OpenMP build)",
            "seconds": dt, "verlet_steps_per_s": n / dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2112_15079_gb300 import inputs

    oracle.build()
    s = inputs.solar_system(args.n)
    N = s.n
    per_step = N * (N - 1)
    import oracle as o

    # One benchmark step = inner_fp64 Verlet steps, as the GPU arm's headline.
    inner = args.inner_fp64
    r, v, a = s.r, s.v, None
    for _ in range(args.warmup):
        r, v, a = o.verlet(s.G, s.dt, inner, r, v, s.m, a, openmp=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, v, a = o.verlet(s.G, s.dt, inner, r, v, s.m, a, openmp=True)
    el = time.perf_counter() - t0
    value = per_step * inner * args.steps / el
    cores = oracle.threads(True)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_INTERACTIONS_PER_S,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"solar_system_n{N}", "n_bodies": N, "dt_day": s.dt,
                   "verlet_steps_per_step": inner, "precision": "fp64",
                   "parallelism": "host cores (OpenMP over target bodies)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{inner} velocity-Verlet steps of the N={N} system per benchmark step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "verlet_steps_per_s": inner * args.steps / el,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def timed_region(torch, b, stream, inner, steps, flush, dist, device):
    """K timed benchmark steps; returns (summed event ms, barrier-bracketed wall s)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(dist, device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for e0, e1 in evs:
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            b.step(inner)
            e1.record(stream)
    torch.cuda.synchronize(device)
    barrier(dist, device)
    wall = time.perf_counter() - t0
    b.sync()
    return sum(e0.elapsed_time(e1) for e0, e1 in evs), wall


def force_kernel_name(prec: str, block: int) -> str:
    """The force kernel a context launches: block = its pair-once block size
    (nbody_pair_once), 0 for the every-ordered-pair kernel."""
    if not block:
        return f"force_kernel<{prec}>"
    if prec == "mixed":
        return f"force_msym_kernel (mixed, each pair once, {block}-entry blocks)"
    if block == 64:
        return "force_sym_kernel (FP64, each pair once, 64-body blocks)"
    return f"force_sym_wide_kernel (FP64, each pair once, {block}-body blocks)"


def roofline(r, prec, traffic, peaks=None):
    """ALU roofline of the force kernel (Eq. 1): FLOPS_PER_INTERACTION x
    N(N-1) per launch over its mean event-timed duration, against the derived
    FP32 (mixed) or FP64 peak (and, with `peaks`, the FFMA / DFMA rates the
    library's microbenchmark measured in the same run).  frac_step is the same
    flop count over the whole timed step (force + Verlet kernels + launch
    gaps)."""
    lanes = 128 if prec == "mixed" else 2
    kt = r["kernel_ms"]
    pair_once = bool(r.get("pair_once"))
    out = {"bound": "alu", "achieved": r["force_tflops"], "peak": PEAK_TFLOPS[prec], "unit": "TFLOP/s",
           "frac": r["force_tflops"] / PEAK_TFLOPS[prec], "traffic": traffic,
           "kernel": force_kernel_name(prec, r.get("pair_once_block") if pair_once else 0),
           "force_ms": kt["force_ms"], "verlet_ms": kt["verlet_ms"],
           "force_share": kt["force_ms"] / (kt["force_ms"] + kt["verlet_ms"]),
           "frac_step": r["achieved_tflops"] / PEAK_TFLOPS[prec],
           "peak_note": f"derived: 152 SMs x {lanes} {'FP32' if prec == 'mixed' else 'FP64'} FMA lanes x 2 flop "
                        f"x 2070 MHz; {FLOPS_PER_INTERACTION} flop per interaction; achieved over the force "
                        "kernel's mean event-timed launch duration"}
    if pair_once and prec == "fp64":
        # Each unordered pair is evaluated once and applied to both bodies:
        # 20 FP64 operations per two interactions, so the 20-flop-per-
        # interaction convention counts 2x the FMA-equivalent work issued.
        # The FP64 pipe's own load is the convention's figure / 2 over the
        # pipe's peak (both counted as FMA = 2 flop).
        out["executed_fp64_ops_per_interaction"] = 10
        out["note"] = ("achieved counts 20 flop per ordered interaction (the metric's convention); the kernel "
                       "issues 10 FP64 operations per interaction (Newton's third law), so frac can exceed 1")
        out["fp64_pipe_frac_of_derived"] = r["force_tflops"] / 2 / PEAK_TFLOPS[prec]
    elif pair_once:
        # Mixed, each pair once: 16 FP32 lane operations per far pair and 22
        # per near pair, i.e. 8 and 11 per interaction, against 12 and 18 on
        # the every-ordered-pair kernel.
        out["executed_fp32_ops_per_interaction"] = {"far": 8, "near": 11}
        out["note"] = ("achieved counts 20 flop per ordered interaction (the metric's convention); the kernel "
                       "evaluates each pair once for both bodies (Newton's third law)")
    if peaks:
        measured = peaks["fp32_tflops"] if prec == "mixed" else peaks["fp64_tflops"]
        out["peak_measured_tflops"] = measured
        out["frac_of_measured"] = r["force_tflops"] / measured
    return out


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = dist_init(world, True)
    from paper_2112_15079_gb300 import build as libbuild

    libbuild.build()
    from paper_2112_15079_gb300 import inputs, nbody

    s = inputs.solar_system(args.n, seed=inputs.BASE_SEED + rank)
    N = s.n
    per_step = N * (N - 1)
    stream = torch.cuda.Stream(device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    results = {}
    tiles = {}
    # FP64 first: the paper's arithmetic and the headline; the mixed path is
    # reported beside it.
    for prec, inner in (("fp64", args.inner_fp64), ("mixed", args.inner)):
        if (prec == "mixed" and args.no_mixed) or (args.only and prec != args.only):
            continue
        with torch.cuda.stream(stream):
            b = nbody.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=prec, device=device,
                            close_omega_dt=args.close if args.only else 0.0, substep_omega_dt=0.05,
                            pair_once=not args.no_pair_once, pair_once_block=args.pair_once_block)
            forced = args.tiles_fp64 if (prec == "fp64" and args.tiles_fp64) else args.tiles
            if forced:
                b.tiles = json.loads(forced)
                b.reset()
            elif not args.no_autotune:
                b.autotune(probe_steps=16 if prec == "mixed" else 2)
            tiles[prec] = b.tiles
            for _ in range(args.warmup):
                b.step(inner)
            b.sync()
        clk = ClockSampler(local)
        clk.__enter__()
        ev_ms, wall = timed_region(torch, b, stream, inner, args.steps, flush, dist, device)
        clk.__exit__(None, None, None)
        ev_s = max_over_ranks(ev_ms * 1e-3, dist, device)
        total = per_step * inner * args.steps * world
        results[prec] = {
            "pair_once": b.pair_once,
            "pair_once_block": b.pair_once_block,
            "value": total / ev_s, "ms_per_step": ev_s / args.steps * 1e3,
            "verlet_steps_per_s": inner * args.steps / ev_s, "wall_s": wall,
            "achieved_tflops": FLOPS_PER_INTERACTION * per_step * inner * args.steps / ev_s * 1e-12,
            "inner": inner, "clocks": clk.summary(),
            # one staging launch per nbody_step call, then per Verlet step the
            # force and Verlet launches (mixed: and the source-box launch first)
            "gpu_launches": args.steps * (1 + (3 if prec == "mixed" else 2) * inner),
        }
        # Roofline of the dominant kernel: the same workload, each kernel of
        # `inner` Verlet steps bracketed alone by events on this stream.
        if args.only and args.close > 0:
            results[prec]["close"] = b.close_info()
            b.close()
            continue
        with torch.cuda.stream(stream):
            kt = b.kernel_times(inner)
        results[prec]["kernel_ms"] = kt
        results[prec]["force_tflops"] = FLOPS_PER_INTERACTION * per_step / (kt["force_ms"] * 1e-3) * 1e-12
        if not args.no_e2e:
            results[prec]["e2e"] = e2e(torch, b, s, stream, inner, args, dist, device, world)
        b.close()
    peaks = None
    if rank == 0:
        p = nbody.peaks()  # measured instruction rates (1e9 lane-ops/s) on this GPU
        peaks = {"fp32_tflops": 2 * p["ffma"] * 1e-3, "fp64_tflops": 2 * p["dfma"] * 1e-3,
                 "mufu_rsqrt_f32_gops": p["rsqrt_f32"], "mufu_rsqrt_f64_gops": p["rsqrt_f64"],
                 "cvt_f32_f64_gops": p["cvt_f32_f64"], "ffma2_tflops": 2 * p["ffma2_lanes"] * 1e-3,
                 "sm_mhz_during_ffma": p["sm_mhz"]}
    extra = None
    if rank == 0 and world == 1 and not args.no_extras and not args.only:
        extra = extras(torch, nbody, inputs, stream, device, args, peaks)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(s, args.cpu_seconds)
    if rank == 0 and args.only:
        r = results[args.only]
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                "precision": args.only, "tiles": tiles.get(args.only)}
        if "close" in r:
            line["close_encounters"] = dict(r["close"], close_omega_dt=args.close, substep_omega_dt=0.05)
        else:
            line["roofline"] = roofline(r, args.only, None, peaks)
        print(json.dumps(line), flush=True)
        return 0
    if rank == 0:
        f = results["fp64"]
        khash = kernel_hash()
        line = {
            "metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": f["value"] / PAPER_INTERACTIONS_PER_S,
            "baseline_note": "vs the paper's production run (1e4-body model, 176 CPU processors, ~23 min for "
                             "1000 steps) = 7.9e7 interactions/s: context on other hardware",
            "dtype": "f64",
            "data": "synthetic (seeded Solar-System-shaped initial conditions)",
            "config": {"workload": f"solar_system_n{N}", "n_bodies": N, "dt_day": s.dt,
                       "verlet_steps_per_step": f["inner"], "precision": "fp64",
                       "force_kernel": "each pair once" if f.get("pair_once") else "stream-K, every ordered pair",
                       "tiles": tiles.get("fp64"),
                       "l2": "flushed between timed steps (256 MB write outside the events); the 1.3 MB state "
                             "stays L2-resident within a step by design",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "verlet_steps_per_s": f["verlet_steps_per_s"],
            "roofline": roofline(f, "fp64", NCU_TRAFFIC.get((khash, "fp64")), peaks),
            "gpu_launches": f["gpu_launches"],
            "clocks": f["clocks"],
        }
        if "e2e" in f:
            line["e2e"] = f["e2e"]
        if "mixed" in results:
            m = results["mixed"]
            line["mixed"] = {"value": m["value"], "unit": UNIT, "ms_per_step": m["ms_per_step"],
                             "dtype": "f32+f64 (FP64 state and Verlet update, FP32 pair arithmetic)",
                             "verlet_steps_per_step": m["inner"], "verlet_steps_per_s": m["verlet_steps_per_s"],
                             "tiles": tiles.get("mixed"),
                             "roofline": roofline(m, "mixed", NCU_TRAFFIC.get((khash, "mixed")), peaks),
                             "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
                             "mixed_speedup": m["value"] / f["value"]}
            if "e2e" in m:
                line["mixed"]["e2e"] = m["e2e"]
        if peaks:
            line["measured_peaks"] = peaks
        if extra:
            line.update(extra)
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_shard(args):
    """Row shards of one system over the ranks (Section 3's distributed
    method): the same metric over the whole system, all ranks' work counted
    once (strong scaling)."""
    import torch

    rank, world, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = dist_init(world, True)
    from paper_2112_15079_gb300 import build as libbuild

    libbuild.build()
    from paper_2112_15079_gb300 import inputs, shard

    s = inputs.solar_system(args.n)  # the same system on every rank
    N = s.n
    prec = args.only or "fp64"
    inner = args.inner_fp64 if prec == "fp64" else args.inner
    stream = torch.cuda.Stream(device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    exchange = shard.allgather_exchange if world > 1 else (lambda sh: None)
    with torch.cuda.stream(stream):
        sh = shard.ShardedNBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=prec, rank=rank, world=world,
                                exchange=exchange, device=device, stream=stream)
        for _ in range(args.warmup):
            sh.step(inner)
    sh.sync()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.__enter__()
    barrier(dist, device)
    torch.cuda.synchronize(device)
    for e0, e1 in evs:
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            sh.step(inner)
            e1.record(stream)
    torch.cuda.synchronize(device)
    barrier(dist, device)
    clk.__exit__(None, None, None)
    sh.sync()
    ev_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) * 1e-3, dist, device)
    if rank == 0:
        per_launch = 3 if prec == "mixed" else 2  # (box,) force and Verlet kernels per Verlet step
        print(json.dumps({
            "metric": METRIC, "value": N * (N - 1) * inner * args.steps / ev_s, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ev_s / args.steps * 1e3,
            "higher_is_better": True, "scaling": "strong",
            "vs_baseline": N * (N - 1) * inner * args.steps / ev_s / PAPER_INTERACTIONS_PER_S,
            "dtype": "f64" if prec == "fp64" else "f32+f64", "data": "synthetic (seeded Solar-System-shaped "
            "initial conditions)",
            "config": {"workload": f"solar_system_n{N}", "n_bodies": N, "dt_day": s.dt, "verlet_steps_per_step": inner,
                       "precision": prec, "parallelism": f"row shards x{world} (one all-gather per Verlet step)",
                       "chunk_bodies": sh.chunk,
                       "l2": "flushed between timed steps (256 MB write outside the events)"},
            "gpu_launches": args.steps * inner * per_launch, "clocks": clk.summary()}), flush=True)
    sh.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def e2e(torch, b, s, stream, inner, args, dist, device, world):
    """Same metric through the public API from pinned host buffers: per step,
    H2D of the full state and masses, re-bind (nbody_reset: Eq. 1 at the new
    positions), S Verlet steps, D2H of the state."""
    N = s.n
    h_state = torch.empty((6, N), dtype=torch.float64).pin_memory()
    h_state[0:3].copy_(torch.from_numpy(s.r))
    h_state[3:6].copy_(torch.from_numpy(s.v))
    h_m = torch.from_numpy(s.m.copy()).pin_memory()
    h_out = torch.empty((6, N), dtype=torch.float64).pin_memory()

    def one():
        with torch.cuda.stream(stream):
            b.state.copy_(h_state, non_blocking=True)
            b.m.copy_(h_m, non_blocking=True)
            b.reset()
            b.step(inner)
            h_out.copy_(b.state, non_blocking=True)
        stream.synchronize()

    for _ in range(args.warmup):
        one()
    barrier(dist, device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = max_over_ranks(time.perf_counter() - t0, dist, device)
    return {"value": N * (N - 1) * inner * args.steps * world / el, "unit": UNIT,
            "h2d_bytes_per_step": int(h_state.numel() * 8 + h_m.numel() * 8),
            "d2h_bytes_per_step": int(h_out.numel() * 8), "ms_per_step": el / args.steps * 1e3}


def timed(torch, stream, fn, reps=1):
    """Event-timed seconds of fn() on `stream` (after a synchronize)."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def extras(torch, nbody, inputs, stream, device, args, peaks=None):
    """Adjoint cost, the 31-body model, a 521-body FP64 system, RK4, the uneven
    ensemble, N = 1M in both precisions, and (optionally) the full N sweep and
    the dt sweep."""
    out = {}
    # adjoint on the 10,425-body model: backward wall / (T x forward step)
    s = inputs.solar_system(args.n)
    idx, tgt = inputs.loss_targets(s)
    T = args.adjoint_steps
    for prec in ("mixed", "fp64"):
        TT = T if prec == "mixed" else max(1, T // 5)  # FP64: ~11 ms per step and reverse step
        with torch.cuda.stream(stream):
            b = nbody.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=prec, ckpt_every=100, device=device)
            fwd = timed(torch, stream, lambda: b.step(TT)) / TT
            gr = torch.zeros((3, s.n), dtype=torch.float64, device=device)
            gr[:, torch.as_tensor(idx, device=device)] = 1.0
            b.grad(TT, gr)  # allocate the workspace
            bwd = timed(torch, stream, lambda: b.grad(TT, gr))
        out.setdefault("adjoint", {})[prec] = {"steps": TT, "backward_s": bwd, "forward_step_ms": fwd * 1e3,
                                               "cost_per_forward_step": bwd / (TT * fwd), "ckpt_every": 100}
        b.close()
        if prec == "mixed":  # one segment: every staged position kept, (T+1) x 32 B x N, no recomputation
            with torch.cuda.stream(stream):
                b = nbody.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=prec, ckpt_every=TT, device=device)
                b.grad(TT, gr)
                bwd1 = timed(torch, stream, lambda: b.grad(TT, gr))
            out["adjoint"][prec]["cost_per_forward_step_ckpt_every_T"] = bwd1 / (TT * fwd)
            b.close()
    # the 31-body model (one FP64 system: single-launch cluster kernel), 3650 steps
    s31 = inputs.solar_system(31)
    with torch.cuda.stream(stream):
        b = nbody.NBody(s31.r, s31.v, s31.m, G=s31.G, dt=s31.dt, precision="fp64", device=device)
        b.step(10)
        t = timed(torch, stream, lambda: b.step(3650))
        b2 = nbody.NBody(s31.r, s31.v, s31.m, G=s31.G, dt=s31.dt, precision="fp64", small=False, device=device)
        b2.step(10)
        t2 = timed(torch, stream, lambda: b2.step(3650))
    out["solar_system_n31"] = {"steps": 3650, "seconds": t, "verlet_steps_per_s": 3650 / t,
                               "interactions_per_s": 31 * 30 * 3650 / t, "precision": "fp64",
                               "general_path_verlet_steps_per_s": 3650 / t2}
    b.close()
    b2.close()
    # a mid-size FP64 system (521 bodies): the single-launch cooperative grid kernel against the general path
    s521 = inputs.solar_system(521, n_moons=0)
    with torch.cuda.stream(stream):
        b = nbody.NBody(s521.r, s521.v, s521.m, G=s521.G, dt=s521.dt, precision="fp64", device=device)
        b.step(10)
        t = timed(torch, stream, lambda: b.step(1000))
        b2 = nbody.NBody(s521.r, s521.v, s521.m, G=s521.G, dt=s521.dt, precision="fp64", small=False, device=device)
        b2.step(10)
        t2 = timed(torch, stream, lambda: b2.step(1000))
    out["fp64_n521"] = {"steps": 1000, "verlet_steps_per_s": 1000 / t, "interactions_per_s": 521 * 520 * 1000 / t,
                        "path": "cooperative grid kernel", "general_path_verlet_steps_per_s": 1000 / t2}
    b.close()
    b2.close()
    # RK4 (Section 2's higher-order method): four Eq. 1 evaluations per step
    for prec, k in (("mixed", 50), ("fp64", 5)):
        with torch.cuda.stream(stream):
            b = nbody.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=prec, integrator="rk4", device=device)
            b.step(k)
            t = timed(torch, stream, lambda: b.step(k))
        out.setdefault("rk4", {})[prec] = {"steps": k, "ms_per_step": t / k * 1e3,
                                           "interactions_per_s": 4 * s.n * (s.n - 1) * k / t,
                                           "force_evaluations_per_step": 4}
        b.close()
    # Close-encounter handling on the 10,425-body model (its moons as drawn:
    # 13 have w dt > 2): cost per step, and how far the fast moons' distances
    # to their hosts move over 365 steps, with and without it.
    G, dt = s.G, s.dt
    fast = []
    for p in range(31, 131):  # the moons: each against the major bodies
        for j in range(31):
            d = np.linalg.norm(s.r[:, p] - s.r[:, j])
            if math.sqrt(G * (s.m[p] + s.m[j]) / d ** 3) * dt > 2.0:
                fast.append((j, p, d))
    for prec, k in (("fp64", 20), ("mixed", 200)):
        row = {}
        for tc in (0.5, 0.0):
            with torch.cuda.stream(stream):
                b = nbody.NBody(s.r, s.v, s.m, G=G, dt=dt, precision=prec, close_omega_dt=tc, substep_omega_dt=0.05,
                                device=device)
                info = b.close_info()
                b.step(2)
                t = timed(torch, stream, lambda: b.step(k))
                b.step(365 - 2 - k)
                b.sync()
                rr = b.state[0:3].cpu().numpy()
            dev = max(abs(np.linalg.norm(rr[:, p] - rr[:, j]) / d0 - 1.0) for j, p, d0 in fast)
            key = "close" if tc > 0 else "plain_verlet"
            row[key] = {"ms_per_step": t / k * 1e3, "fast_moons_max_rel_distance_change_365_steps": dev}
            if tc > 0:
                row[key].update(close_pairs=info["pairs"], clusters=info["clusters"], k_max=info["k_max"],
                                close_omega_dt=tc, substep_omega_dt=0.05)
            b.close()
        out.setdefault("close_encounters", {"fast_moons": len(fast)})[prec] = row
    # uneven ensemble, mixed, one context
    ens = inputs.ensemble(args.ensemble_systems)
    off, r, v, m = inputs.concat(ens)
    pairs = sum(e.n * (e.n - 1) for e in ens)
    with torch.cuda.stream(stream):
        b = nbody.NBody(r, v, m, off, G=inputs.G_AU_DAY, dt=inputs.DT_DAY, precision="mixed", device=device)
        if not args.no_autotune:
            b.autotune(probe_steps=1)  # the work line of uneven systems has its own best tiles
        b.step(2)
        n_ens = 5
        t = timed(torch, stream, lambda: b.step(n_ens))
    out["ensemble"] = {"systems": len(ens), "bodies": int(off[-1]), "steps": n_ens,
                       "interactions_per_s": pairs * n_ens / t, "verlet_steps_per_s": n_ens / t,
                       "ms_per_step": t / n_ens * 1e3, "precision": "mixed", "tiles": b.tiles}
    b.close()
    if args.dt_sweep:
        # Energy accuracy against dt (Section 4's criterion): the 10,425-body
        # construction without moons (their periods fall below dt), 73 days,
        # maximum |E - E0|/|E0| over 20 samples per run.
        sd = inputs.solar_system(args.n, n_moons=0)
        rows = []
        for dt in (0.8, 0.4, 0.2, 0.1, 0.05):
            row = {"dt_day": dt}
            n_steps = int(round(73.0 / dt))
            every = max(1, n_steps // 20)
            for prec, integ in (("fp64", "verlet"), ("mixed", "verlet"), ("fp64", "rk4"), ("mixed", "rk4"),
                                ("fp64", "leapfrog"), ("mixed", "leapfrog")):
                with torch.cuda.stream(stream):
                    b = nbody.NBody(sd.r, sd.v, sd.m, G=sd.G, dt=dt, precision=prec, integrator=integ,
                                    device=device)
                    e0 = b.energy()[0]
                    worst = 0.0
                    for _ in range(n_steps // every):
                        b.step(every)
                        worst = max(worst, abs(b.energy()[0] - e0) / abs(e0))
                    b.close()
                row[prec if integ == "verlet" else prec + "_" + integ] = worst
            rows.append(row)
        for a, b2 in zip(rows, rows[1:]):
            for key in ("fp64", "mixed", "fp64_rk4", "mixed_rk4", "fp64_leapfrog", "mixed_leapfrog"):
                b2[key + "_order"] = float(np.log2(a[key] / b2[key]))
        out["dt_sweep"] = {"bodies": sd.n, "days": 73.0, "max_rel_energy_drift": rows}
    # N sweep.  By default N = 65,536 and 1,048,576 (the metric's second size),
    # mixed and FP64, the library's default tiles (tuning at 1M would cost
    # minutes); --sweep adds 16,384 and 65,536 autotuned, and 262,144 with
    # their winner.  FP64 above 65,536 bodies runs the wide-block pair-once
    # kernel (one step each: about 1.3 s at 262,144 and 20 s at 1M bodies).
    if not args.no_extras:
        tuned = {}
        for n in ((16384, 65536, 262144, 1048576) if args.sweep else (65536, 1048576)):
            sn = inputs.solar_system(n)
            row = {}
            for prec in ("mixed", "fp64"):
                with torch.cuda.stream(stream):
                    b = nbody.NBody(sn.r, sn.v, sn.m, G=sn.G, dt=sn.dt, precision=prec, device=device)
                    if n <= 65536 and args.sweep:
                        tuned[prec] = b.autotune(probe_steps=4 if prec == "mixed" else 1)[0]
                    elif prec in tuned:
                        b.tiles = tuned[prec]
                        b.reset()
                    k = 1 if prec == "fp64" and n > 65536 else 2 if n >= 262144 else 5
                    if k > 1:
                        b.step(1)  # warm-up (the FP64 1M step is long enough without one)
                    t = timed(torch, stream, lambda: b.step(k))
                per = n * (n - 1) * k / t
                row[prec] = {"interactions_per_s": per, "ms_per_step": t / k * 1e3,
                             "roofline_frac": per * FLOPS_PER_INTERACTION * 1e-12 / PEAK_TFLOPS[prec],
                             "force_kernel": force_kernel_name(prec, b.pair_once_block),
                             "tiles": None if b.pair_once_block else b.tiles}
                if peaks:  # the whole step (force, Verlet, boxes) against the measured peak
                    measured = peaks["fp32_tflops"] if prec == "mixed" else peaks["fp64_tflops"]
                    row[prec]["frac_of_measured"] = per * FLOPS_PER_INTERACTION * 1e-12 / measured
                b.close()
            out.setdefault("sweep", {})[str(n)] = row
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.shard:
        return run_shard(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
