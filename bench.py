#!/usr/bin/env python3
"""Throughput of the WCSPH time step (NL + PI + SU) on GB300.

Default workload: the 3D dam break at dp = 0.005 m (643,200 fluid + 232,727
boundary particles, the "1M" point), FP32 split-precision PI, neighbour list
rebuilt every step, variable dt.  One JSON line on stdout (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: each timed step is bracketed by CUDA events on the stream the library
launches on; L2 is flushed (a 512 MB write) between timed steps, outside the
events.  Under torchrun (N > 1) every rank runs an independent replica (the
dam break does not shard across GPUs here: "replicas only"), the time is the
max over ranks and the value counts the steps of all ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from sphcases import dam_break  # noqa: E402

# FLOPs of the method per unit of work, counted from the formulas (every add,
# sub, mul, div, sqrt, compare, abs and max is one FLOP, so a multiply-add is
# two, as in the FMA peak the fraction is taken against).
FLOP_PER_CANDIDATE = 9        # r_ab (3), |r_ab|^2 (5), test (1)
FLOP_PER_PAIR_FLUID = 45      # kernel gradient, viscosity, momentum, continuity, dt term
FLOP_PER_PAIR_BOUNDARY = 24   # kernel gradient, continuity, dt term
GB300_SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0

WORKLOADS = {
    "dam1m": dict(dp=0.005, label="3D dam break dp=0.005 m (643,200 fluid + 232,727 boundary)"),
    "dam5m": dict(dp=0.0025, label="3D dam break dp=0.0025 m (5,145,600 fluid + 927,529 boundary)"),
    "dam10k": dict(dp=0.02, label="3D dam break dp=0.02 m (9,900 fluid + 14,744 boundary)"),
    "dam20m": dict(dp=0.0016, label="3D dam break dp=0.0016 m (19,541,500 fluid + 2,259,259 boundary)"),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def fp32_peak_tflops(mhz=SM_MAX_MHZ_NOMINAL):
    """FP32 FMA peak: SMs x FP32 lanes x 2 FLOP x clock."""
    return GB300_SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons in a thread."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- dist utils --

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(torch, value, world):
    """Largest value over the ranks (the slowest rank's time)."""
    if world <= 1:
        return value
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_steps_per_s(world, steps, max_ms):
    """Whole-job throughput of independent replicas: every rank's steps over
    the slowest rank's time."""
    return world * steps / (max_ms / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------- GPU timing --

def fine_cells(case):
    """The same case on cells of edge h (half the support), the paper's finer
    cells (Section 4.6, optimisation F; Section 3.2 on the CPU)."""
    p = dataclasses.replace(case.params, cell_size=case.params.h)
    return type(case)(**{**case.__dict__, "params": p})


def pi_flops(counts):
    """Algorithmic FLOPs of one PI call for the exact candidate and pair counts."""
    c = np.asarray(counts, dtype=np.float64)
    return (FLOP_PER_CANDIDATE * (c[0] + c[2]) + FLOP_PER_PAIR_FLUID * c[1]
            + FLOP_PER_PAIR_BOUNDARY * c[3])


def counts_now(sim):
    """Exact work counts of the current state (a full NL -> count -> PI -> SU step)."""
    sim.neighbour_list()
    c = sim.count_work()
    sim.interact()
    sim.update()
    return c


def time_steps(torch, sim, steps, flush):
    """Per-step CUDA-event timing with an L2 flush between steps."""
    st = sim.stream
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        e = ev[k]
        e[0].record(st)
        sim.neighbour_list()
        e[1].record(st)
        sim.interact()
        e[2].record(st)
        sim.update()
        e[3].record(st)
    torch.cuda.synchronize()
    nl = sum(e[0].elapsed_time(e[1]) for e in ev)
    pi = sum(e[1].elapsed_time(e[2]) for e in ev)
    su = sum(e[2].elapsed_time(e[3]) for e in ev)
    tot = sum(e[0].elapsed_time(e[3]) for e in ev)
    return dict(total_ms=tot, nl_ms=nl, pi_ms=pi, su_ms=su)


def time_steps_graph(torch, sim, steps, flush):
    """Steps replayed from the library's captured CUDA graph (two steps per
    replay), CUDA events around each replay, L2 flushed between replays."""
    st = sim.stream
    pairs = steps // 2
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(pairs)]
    for k in range(pairs):
        flush.zero_()
        ev[k][0].record(st)
        sim.run_graph(2)
        ev[k][1].record(st)
    torch.cuda.synchronize()
    return sum(e[0].elapsed_time(e[1]) for e in ev), 2 * pairs


def run_form(torch, case, precision, steps, warmup, flush, world, clocks=False, rank=0, local=0,
             pi_kernel="warp", graph=False):
    from paper_1110_3711_gb300.sph import Simulation
    sim = Simulation.from_case(case, precision=precision, pi_kernel=pi_kernel,
                               stream=torch.cuda.current_stream())
    for _ in range(warmup):
        sim.step()
    ckpt = None
    if graph:
        # the graph replays the same steps as the ordinary launches: the state
        # after the warm-up is kept and restored before the graph is timed
        ckpt = torch.empty(sim.checkpoint_bytes(), dtype=torch.uint8, device="cuda")
        sim.save_state(ckpt)
    c0 = counts_now(sim)
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    l0 = sim.launches
    t = time_steps(torch, sim, steps, flush)
    launches = sim.launches - l0
    graph_res = None
    if graph:
        sim.run_graph(2)   # capture outside the timed region
        sim.load_state(ckpt)
        torch.cuda.synchronize()
        barrier(world)
        g0 = sim.launches
        g_ms, g_steps = time_steps_graph(torch, sim, steps, flush)
        g_launches = sim.launches - g0
        g_ms = max_over_ranks(torch, g_ms, world)
        graph_res = dict(steps_per_s=replica_steps_per_s(world, g_steps, g_ms),
                         ms_per_step=g_ms / g_steps, steps=g_steps, launches=g_launches)
    torch.cuda.synchronize()
    barrier(world)
    clk = sampler.stop() if sampler else None
    c1 = counts_now(sim)
    flags = sim.status()
    tot = max_over_ranks(torch, t["total_ms"], world)
    counts = (np.asarray(c0, np.float64) + np.asarray(c1, np.float64)) / 2
    pairs = counts[1] + counts[3]
    sps = replica_steps_per_s(world, steps, tot)
    res = dict(steps_per_s=sps, ms_per_step=tot / steps,
               interactions_per_s=pairs * sps,
               stage_ms=dict(nl=t["nl_ms"] / steps, pi=t["pi_ms"] / steps, su=t["su_ms"] / steps),
               pi_ms=t["pi_ms"] / steps, counts=counts.tolist(), launches=launches,
               status_flags=flags)
    if graph_res is not None:
        res["graph"] = graph_res
    simtime = sim.time()
    res["sim_time_s"] = simtime[0]
    res["last_dt_s"] = simtime[1]
    if clk is not None:
        res["clocks"] = clk
    return sim, res


def e2e_form(torch, sim, steps):
    """Steps/s through the C ABI with host buffers: every step uploads the full
    state from pinned host memory (sph_set_state), runs NL, PI, SU and reads the
    state back (sph_get_state)."""
    n = sim.n
    pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    pos, vel, rho, vp, rp = pin((n, 3)), pin((n, 3)), pin(n), pin((n, 3)), pin(n)
    from paper_1110_3711_gb300 import sph as S
    S.sph_get_state(sim.ctx, n, pos, vel, rho, vp, rp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        S.sph_set_state(sim.ctx, n, pos, vel, rho, vp, rp)
        sim.step()
        S.sph_get_state(sim.ctx, n, pos, vel, rho, vp, rp)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nbytes = 8 * (3 + 3 + 1 + 3 + 1) * n
    return dict(value=steps / dt, unit="steps/s", h2d_bytes_per_step=nbytes,
                d2h_bytes_per_step=nbytes, steps=steps,
                note="state uploaded from and read back to pinned host memory every step")


def code_hash(paths):
    """sha256 (16 hex digits) of C/CUDA sources with their comments and
    whitespace removed: edits of comments do not change it, edits of code do."""
    import re
    src = ""
    for path in paths:
        s = open(path, encoding="utf-8").read()
        s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
        s = re.sub(r"//[^\n]*", "", s)
        src += re.sub(r"\s+", "", s)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


# the sources of the FP32 PI kernel k_pi32
PI32_SOURCES = [os.path.join(ROOT, "paper_1110_3711_gb300", "csrc", f)
                for f in ("pi32.cu", "warp_items.cuh", "pair32.cuh")]


def traffic_from_profiles(kernel_srcs):
    """DRAM bytes per PI call from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "pi_dram_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = code_hash(kernel_srcs)
    vals = {}
    for ln in open(path):
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.split("=", 1)
            vals[k.strip()] = v.strip()
    if vals.get("pi_cu_code_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_pi_call"])
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------- CPU legs --

def measured_fma(torch):
    """Float32 and float64 FMA rates of this GPU (sph_fma_rate: independent FMA
    chains, CUDA events), in TFLOP/s at 2 FLOP per FMA."""
    from paper_1110_3711_gb300 import sph
    scratch = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    out = {}
    for name in ("fp32", "fp64"):
        out[name + "_tflops"] = sph.sph_fma_rate(name, scratch, st) / 1e12
    return out


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: the
    implementer and part numbers), else what platform reports."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k, _, v = ln.partition(":")
                k, v = k.strip(), v.strip()
                if k and v and k not in fields:
                    fields[k] = v
    except OSError:
        pass
    if "model name" in fields:
        return fields["model name"]
    if "CPU part" in fields:
        return f"Arm implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    import platform
    return platform.processor() or platform.machine()


def oracle_step_seconds(O, case, stride, cores):
    """Time one oracle step on the host: list build and PI on every stride-th
    target (scaled by stride), the time step and SU on all particles."""
    p = case.params
    ace, ar, vm, counts, nout, secs = O.interact_sampled(p, case.n_f, case.n_b, case.pos,
                                                         case.vel, case.rho, stride, cores)
    pos, vel, rho = case.pos.copy(), case.vel.copy(), case.rho.copy()
    velm, rhom = vel.copy(), rho.copy()
    t0 = time.perf_counter()
    dt = O.time_step(p, case.n_f, case.n_b, pos, ace, rho, vm)
    O.update(p, case.n_f, case.n_b, 0, dt if math.isfinite(dt) and dt > 0 else 1e-5,
             pos, vel, velm, rho, rhom, ace, ar)
    t_su = time.perf_counter() - t0
    return secs[0] + secs[1] * stride + t_su, dict(nl=secs[0], pi=secs[1] * stride, su=t_su)


def cpu_baseline(case, budget_s=15.0):
    """The FP64 oracle as it stands on the host cores: full steps (NL, PI, SU on
    every particle) until about budget_s of wall time."""
    from oracle import oracle as O
    O.lib()
    cores = cpu_cores()
    st = O.State(case)
    n = 0
    t0 = time.perf_counter()
    while True:
        st.step(nthreads=cores)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 50:
            break
    pairs = st.last_counts[1] + st.last_counts[3]
    return {"value": n / el, "unit": "steps/s", "cores": cores, "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"{n} full oracle steps (NL+PI+SU, all {case.n} particles, FP64) "
                      f"from the initial state, {el:.1f} s wall",
            "interactions_per_s": float(pairs) * n / el}


def run_reference(args, workload):
    """--impl reference: the FP64 oracle on the host cores, same workload and
    metric; each step times NL, PI on a uniform sample of targets (scaled to all
    targets), dt and SU on all particles."""
    from oracle import oracle as O
    O.lib()
    case = dam_break(WORKLOADS[workload]["dp"])
    cores = cpu_cores()
    total_budget = float(os.environ.get("SPH_REFERENCE_BUDGET_S", "150"))
    # calibrate the PI cost on a 1/64 sample
    t_cal, parts = oracle_step_seconds(O, case, 64, cores)
    per_step = total_budget / max(1, args.steps + args.warmup)
    t_fixed = parts["nl"] + parts["su"]
    pi_full = parts["pi"]
    frac = min(1.0, max(1e-4, (per_step - t_fixed) / max(pi_full, 1e-9)))
    stride = max(1, int(math.ceil(1.0 / frac)))
    for _ in range(args.warmup):
        oracle_step_seconds(O, case, stride, cores)
    tot = 0.0
    for _ in range(args.steps):
        s, _ = oracle_step_seconds(O, case, stride, cores)
        tot += s
    value = args.steps / tot
    sample = (f"per step: oracle list build, PI on every {stride}-th of {case.n} targets "
              f"scaled by {stride}, dt and SU on all particles; FP64, {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(workload, case),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores,
                             "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "steps/s and particle-interactions/s at 1M and 5M particles, FP32 vs FP64, 1xGB300"


def config_block(workload, case):
    return {"workload": WORKLOADS[workload]["label"] + ", NL rebuilt every step, "
            "variable dt (CFL 0.2), Verlet with an Euler step every 40 steps",
            "particles": case.n, "fluid": case.n_f, "boundary": case.n_b,
            "l2": "flushed between timed steps (512 MB write)",
            "parallelism": "replicas only (one independent dam break per GPU)"}


# ------------------------------------------------------------------- main --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="dam1m")
    ap.add_argument("--fp64-steps", type=int, default=-1,
                    help="FP64 steps at the benchmark size (default: the same window as --steps)")
    ap.add_argument("--late-advance", type=int, default=5000,
                    help="untimed steps before the late-state timing (0: skip the late state)")
    ap.add_argument("--late-steps", type=int, default=200)
    ap.add_argument("--no-20m", action="store_true", help="skip the 21.8M-particle line")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-5m", action="store_true", help="skip the 5M-particle lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ablation-steps", type=int, default=100,
                    help="steps for each of the paper-design PI kernels (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.fp64_steps < 0:
        args.fp64_steps = args.steps
    world, rank, local = dist_env()

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, args.workload)
        return

    import torch
    torch.cuda.set_device(local)
    # a stream of our own: the library's CUDA-graph replay cannot capture the
    # legacy default stream
    bench_stream = torch.cuda.Stream()
    torch.cuda.set_stream(bench_stream)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1110_3711_gb300 import build as B
    if rank == 0 or not B.up_to_date():
        B.build()
    barrier(world)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    case = dam_break(WORKLOADS[args.workload]["dp"])
    sim, r32 = run_form(torch, case, "fp32", args.steps, args.warmup, flush, world,
                        clocks=True, rank=rank, local=local, graph=True)
    e2e = None
    if args.e2e_steps > 0:
        e2e = e2e_form(torch, sim, args.e2e_steps)
        e2e["value"] = e2e["value"] * world  # replicas: all ranks' steps
    del sim
    r64 = None
    if args.fp64_steps > 0:
        # same warm-up as the FP32 run, so that with fp64_steps == steps both
        # forms are timed over the same window of the flow
        sim64, r64 = run_form(torch, case, "fp64", args.fp64_steps, args.warmup, flush, world)
        del sim64

    extra = {}
    if args.ablation_steps > 0:
        # the paper's GPU design on the same workload (Section 4, Fig. 11): one
        # thread per particle, ranges from CellBeginEnd or precomputed per cell,
        # and the same on cells of edge h (Section 4.6, optimisation F: 125-cell search);
        # all designs over the same steps from the initial state
        abl = {"steps": args.ablation_steps}
        fine = fine_cells(case)
        for name, kname, cs in (("warp", "warp", case), ("warp_sym", "warp_sym", case),
                                ("thread", "thread", case),
                                ("thread_fastcells", "thread_fastcells", case),
                                ("thread_hcells", "thread", fine)):
            s_a, r_a = run_form(torch, cs, "fp32", args.ablation_steps, 3, flush, world,
                                pi_kernel=kname)
            del s_a
            abl[name] = {"steps_per_s": r_a["steps_per_s"], "pi_ms": r_a["pi_ms"],
                         "stage_ms": r_a["stage_ms"],
                         "candidates_per_step": r_a["counts"][0] + r_a["counts"][2]}
        if args.fp64_steps > 0:
            abl["fp64"] = {"steps_per_s": r64["steps_per_s"], "pi_ms": r64["pi_ms"],
                           "candidates_per_step": r64["counts"][0] + r64["counts"][2]}
            for name, kname, cs in (("fp64_thread", "thread", case),
                                    ("fp64_hcells", "warp", fine)):
                s_a, r_a = run_form(torch, cs, "fp64", min(args.fp64_steps, 50), 3, flush, world,
                                    pi_kernel=kname)
                del s_a
                abl[name] = {"steps_per_s": r_a["steps_per_s"], "pi_ms": r_a["pi_ms"],
                             "candidates_per_step": r_a["counts"][0] + r_a["counts"][2]}
        extra["pi_kernel_ablation"] = abl
    if args.late_advance > 0 and args.late_steps > 0:
        # the same workload after the column has collapsed: the untimed
        # advance runs as the warm-up, then steps are timed as above
        s_l, r_l = run_form(torch, case, "fp32", args.late_steps, args.late_advance, flush, world)
        del s_l
        fl = pi_flops(r_l["counts"])
        ach = fl / (r_l["pi_ms"] / 1e3) / 1e12
        extra["late_state"] = {
            "advance_steps": args.late_advance, "steps": args.late_steps,
            "sim_time_s": r_l["sim_time_s"], "steps_per_s": r_l["steps_per_s"],
            "ms_per_step": r_l["ms_per_step"], "interactions_per_s": r_l["interactions_per_s"],
            "stage_ms": r_l["stage_ms"], "counts": r_l["counts"],
            "roofline": {"bound": "alu", "achieved": ach, "peak": fp32_peak_tflops(),
                         "unit": "TFLOP/s", "frac": ach / fp32_peak_tflops(),
                         "flops_per_call": fl},
            "status_flags": r_l["status_flags"]}
    if not args.no_5m and args.workload != "dam5m":
        case5 = dam_break(WORKLOADS["dam5m"]["dp"])
        n5 = 100
        s5, r5 = run_form(torch, case5, "fp32", n5, 5, flush, world)
        del s5
        s5d, r5d = run_form(torch, case5, "fp64", n5, 5, flush, world)
        del s5d
        extra["dam5m"] = {"particles": case5.n, "steps": n5, "warmup": 5,
                          "fp32_steps_per_s": r5["steps_per_s"],
                          "fp32_interactions_per_s": r5["interactions_per_s"],
                          "fp32_stage_ms": r5["stage_ms"],
                          "fp64_steps_per_s": r5d["steps_per_s"],
                          "fp64_interactions_per_s": r5d["interactions_per_s"],
                          "fp64_stage_ms": r5d["stage_ms"],
                          "fp32_over_fp64": r5["steps_per_s"] / r5d["steps_per_s"],
                          "window": "both forms timed over the same steps 6-105 from rest"}
        del case5
    if not args.no_20m and args.workload != "dam20m":
        # configuration of the large dam break: 500 steps, NL / PI / SU shares
        case20 = dam_break(WORKLOADS["dam20m"]["dp"])
        s20, r20 = run_form(torch, case20, "fp32", 500, 5, flush, world)
        del s20
        st_ms = r20["stage_ms"]
        tot_ms = sum(st_ms.values())
        fl = pi_flops(r20["counts"])
        extra["dam20m"] = {"particles": case20.n, "steps": 500, "warmup": 5,
                           "steps_per_s": r20["steps_per_s"],
                           "interactions_per_s": r20["interactions_per_s"],
                           "stage_ms": st_ms,
                           "stage_share": {k: v / tot_ms for k, v in st_ms.items()},
                           "pi_roofline_frac": fl / (r20["pi_ms"] / 1e3) / 1e12 / fp32_peak_tflops(),
                           "sim_time_s": r20["sim_time_s"], "status_flags": r20["status_flags"]}
        del case20

    pk = peaks()
    fma = measured_fma(torch)
    clk = r32.get("clocks", {})
    flops = pi_flops(r32["counts"])
    achieved = flops / (r32["pi_ms"] / 1e3) / 1e12
    peak = fp32_peak_tflops()
    traffic = traffic_from_profiles(PI32_SOURCES)

    g = r32.get("graph")
    sps = g["steps_per_s"] if g else r32["steps_per_s"]
    line = {
        "metric": METRIC,
        "value": sps, "unit": "steps/s",
        "n_gpus": world, "steps": g["steps"] if g else args.steps, "warmup": args.warmup,
        "ms_per_step": g["ms_per_step"] if g else r32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 PI, f64 positions and dt", "data": "synthetic",
        "config": config_block(args.workload, case),
        "interactions_per_s": r32["interactions_per_s"] * sps / r32["steps_per_s"],
        "timing": ("steps replayed from the library's CUDA graph (sph_run_graph, two steps per "
                   "replay, CUDA events around each replay); stage_ms and the PI roofline from a "
                   "run of ordinary launches with events around each stage over the same steps "
                   "(state after the warm-up restored between the two runs)"),
        "plain_launches": {"steps_per_s": r32["steps_per_s"], "ms_per_step": r32["ms_per_step"]},
        "stage_ms": r32["stage_ms"],
        "fp64": (None if r64 is None else
                 {"steps_per_s": r64["steps_per_s"], "ms_per_step": r64["ms_per_step"],
                  "interactions_per_s": r64["interactions_per_s"], "steps": args.fp64_steps,
                  "stage_ms": r64["stage_ms"],
                  # the same FLOP count in float64 over the measured float64 FMA rate
                  "pi_tflops": pi_flops(r64["counts"]) / (r64["pi_ms"] / 1e3) / 1e12,
                  "pi_frac_of_measured_fp64_fma": (
                      pi_flops(r64["counts"]) / (r64["pi_ms"] / 1e3) / 1e12 / fma["fp64_tflops"]
                      if fma.get("fp64_tflops") else None)}),
        "fp32_over_fp64": None if r64 is None else r32["steps_per_s"] / r64["steps_per_s"],
        "roofline": {"bound": "alu",
                     "kernel": "PI (sph_interact: k_pi32, fluid and boundary work items)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (derived)",
                     "flops_per_call": flops,
                     "frac_at_measured_clock": (achieved / fp32_peak_tflops(clk["sm_mhz"])
                                                if clk.get("sm_mhz") else None),
                     "frac_of_measured_fma": (achieved / fma["fp32_tflops"]
                                              if fma.get("fp32_tflops") else None)},
        "measured_fma": fma,
        "e2e": e2e,
        "gpu_launches": g["launches"] if g else r32["launches"],
        "clocks": clk,
        "status_flags": r32["status_flags"],
    }
    line.update(extra)
    if pk:
        line["measured_peaks"] = {"hbm_gbs": pk.get("hbm_gbs"), "bf16_tflops": pk.get("bf16_tflops")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(case)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
