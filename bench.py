#!/usr/bin/env python
"""Benchmark: one MPPI iteration (arXiv 2308.01654, Algorithm 1) per step on GB300.

Default workload ("roofline"): K=65536 samples, T=200 steps, dt=0.025 s, straight
2000-point lane, 64 static obstacles x 3 circles; synthetic seeded inputs.  A step
is the whole iteration: Philox noise, fused rollout+cost, argmin, softmin
weights, weighted update, Savitzky-Golay smoothing, x* rollout, warm start.

Metric: rollout-steps/s (K*T per iteration / iteration time), higher is better.
  value     device time with inputs resident in HBM (CUDA events on the planner's
            stream, L2 flushed between steps by writing a 256 MB buffer); the planner
            records two more events around the rollout kernel in each timed step,
            which end the chaining of its launch with the neighbouring kernels
            (a few microseconds per step)
  e2e       the same metric through mppi_plan() with host buffers: the input H2D
            copy and the outputs (written by the last kernel into pinned host memory)
            inside the timed region
  roofline  the rollout kernel (the dominant kernel) against the FP32-pipe peak,
            its duration from those two events
  kernel_ms per-kernel times from three untimed steps with an event at every kernel
            boundary
  cpu_baseline  the FP64 oracle on the host cores over a bounded sample (all cores, and a
            single-thread row), with the host CPU model
  error_vs_oracle  the CUDA path against that oracle run on the same K-sample: every
            sample cost, the argmin, u* and x*
  bf16_noise  the same workload with bfloat16-stored noise (device-timed), with its
            error against the oracle on the same codes and on the unrounded noise
  systems   the batched form (256 uneven plans per submission against the plain
            per-plan loop) and the serving form (512 sessions, Poisson arrivals at
            2000 and 8000 plans/s, p50/p99 latency against the plain FIFO loop), in
            shortened runs; --no-systems skips these and bf16_noise
N > 1 (torchrun): every rank runs an independent planner on its own GPU (weak
scaling, no collective on the data path); value = all ranks' rollout-steps / the
slowest rank's time.

--impl reference times the FP64 oracle itself (the CPU baseline) per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rollout-steps/s (K*T) of one MPPI iteration"
UNIT = "rollout-steps/s"
KERNEL_LAUNCHES_PER_STEP = 5   # prep + noise, rollout (with the argmin), weights, wsum, finalize (+1 noise fix-up for bf16 noise)


# ------------------------------------------------------------------------ helpers

def brute_force_ops_per_step(prob) -> float:
    """FP32 operations per rollout-step if every obstacle pair were tested and the reference
    scanned with 32-segment chunk bounds: ~60 for dynamics and costs, 6 per (ego, obstacle)
    pair, 5 per chunk bound and ~11 per segment of ~2 scanned chunks."""
    p = prob.params
    n_e, n_c, n_ref = int(p["n_ego"]), int(prob.circles.shape[0]), int(prob.ref.shape[0])
    return 60.0 + 6.0 * n_e * n_c + 5.0 * math.ceil((n_ref - 1) / 32.0) + 11.0 * 64.0


# Arithmetic (FP32/ALU pipe) operations of one unit of each piece of work the rollout
# kernel does, counted from its source: the per-step core (perturbation, Euler step with
# compensated sums, sincos and tan, cost terms, control cost, ego circles and the warp
# box of the broad phase) and, per unit counted by mppi_rollout_stats, a box bound, a
# segment distance with its key minimum, a broad-phase circle test, a candidate circle
# (three pair distances, their minimum and the band test) and an in-band circle (sqrt,
# subtract, min).
OPS_CORE = 150.0
OPS_PER = {"range_boxes": 12.0, "chunk_boxes": 12.0, "segments": 13.0, "refinements": 40.0,
           "circles_tested": 15.0, "candidates": 17.0, "in_band": 4.0}


def executed_ops_per_step(stats) -> float:
    """Arithmetic operations per rollout-step of the pruned exact algorithm, from its work counters."""
    return OPS_CORE + sum(OPS_PER[k] * stats[k] for k in OPS_PER)


KERNEL_SOURCES = ("paper_2308_01654_gb300/csrc/mppi_kernels.cu", "paper_2308_01654_gb300/csrc/mppi_device.cuh",
                  "paper_2308_01654_gb300/csrc/mppi_internal.h", "paper_2308_01654_gb300/csrc/mppi_iter.cuh",
                  "paper_2308_01654_gb300/csrc/mppi_trace.h")
TRAFFIC_PROFILE = {"roofline": "profiles/rollout_kernel_roofline_K65536_T200.md"}


def launch_desc(group: int, block: int) -> dict:
    """The rollout launch shape: lanes per sample and what they split."""
    return {"lanes_per_sample": abs(int(group)), "lanes_split": "steps" if group < 0 else "work of each step",
            "threads_per_block": int(block)}


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_value(workload: str, key: str):
    """A figure ("key = value" line) of the committed ncu summary of the rollout kernel for this
    workload, if that summary was taken on the current kernel source."""
    import re
    path = TRAFFIC_PROFILE.get(workload)
    if not path or not os.path.exists(os.path.join(ROOT, path)):
        return None
    txt = open(os.path.join(ROOT, path)).read()
    m_h = re.search(r"sha256\[:16\]\): `([0-9a-f]+)`", txt)
    m_b = re.search(re.escape(key) + r" = ([0-9.]+)", txt)
    if not m_h or not m_b or m_h.group(1) != kernel_source_hash():
        return None
    return float(m_b.group(1))


def profiled_traffic(workload: str):
    """DRAM bytes per rollout launch from the committed ncu summary (same source only)."""
    v = profiled_value(workload, "dram_bytes_per_launch")
    return None if v is None else int(v)


def counted_model(workload: str, units: float, ms: float, peak_tops: float):
    """Arithmetic thread instructions per rollout-step counted by ncu on the current build (from the
    committed summary), or None when that summary was taken on another build."""
    ops = profiled_value(workload, "counted_ops_per_rollout_step")
    fp32 = profiled_value(workload, "fp32_ops_per_rollout_step")
    inst = profiled_value(workload, "thread_inst_per_rollout_step")
    if ops is None:
        return None
    achieved = ops * units / (ms * 1e-3) / 1e12
    return {"ops_per_rollout_step": ops, "fp32_ops_per_rollout_step": fp32, "thread_inst_per_rollout_step": inst,
            "achieved": achieved, "frac": achieved / peak_tops,
            "classes": "FP32 (FADD, FMUL, FFMA and the other FP32 ops), integer, bit and conversion"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for(device_index: int) -> str:
    import torch
    try:
        u = torch.cuda.get_device_properties(device_index).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[device_index]
        return str(device_index)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(values, world: int, device):
    """Element-wise maximum of per-rank figures (the slowest rank's times) over all ranks."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def sum_over_ranks(values, world: int, device):
    """Element-wise sum of per-rank figures over all ranks."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return [float(v) for v in t.cpu()]


def dist_init(world: int, local: int):
    """One process group per job (NCCL, this rank's GPU); nothing for one rank."""
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))


def dist_done(world: int):
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def weak_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of a weak-scaling run: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


def rank_session(rank: int, session: int = 0) -> int:
    """Philox session word of a rank's problem: ranks plan independent problems."""
    return rank * 100000 + session


# ------------------------------------------------------------------------ CPU baseline (the oracle)

def oracle_sample(prob, seconds: float):
    """Time oracle.plan (the whole iteration, FP64) on a sample of K' samples of the same workload."""
    import oracle
    oracle.build()
    probe = prob.copy()
    k0 = min(prob.K, 64)
    probe.params["K"] = k0
    t = time.perf_counter()
    oracle.plan(probe)
    dt = max(time.perf_counter() - t, 1e-6)
    k = int(max(k0, min(prob.K, k0 * seconds / dt)))
    return k


def time_oracle(prob, k_sample: int, want_result: bool = False):
    import oracle
    q = prob.copy()
    q.params["K"] = k_sample
    t = time.perf_counter()
    r = oracle.plan(q)
    el = time.perf_counter() - t
    assert r.rc == 0
    return (el, r) if want_result else el


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_record(prob, seconds: float):
    """The oracle as it stands on the host cores: one full FP64 iteration on a K-sample of the
    workload with every core (OpenMP over samples), and a smaller one on a single thread.
    Returns (record, oracle result of the all-cores run) - the result doubles as the reference
    of the error-vs-oracle check."""
    import oracle
    T = prob.T
    k_s = oracle_sample(prob, seconds)
    el, r = time_oracle(prob, k_s, want_result=True)
    cores = oracle.num_threads()
    rec = {"value": k_s * T / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one full FP64 iteration at K={k_s} of the same workload (T={T}), {el:.1f} s",
           "cpu_model": cpu_model()}
    k_1 = max(16, int(k_s / max(cores, 1) * 0.5))
    oracle.set_num_threads(1)
    try:
        el1 = time_oracle(prob, k_1)
    finally:
        oracle.set_num_threads(cores)
    rec["single_thread"] = {"value": k_1 * T / el1, "unit": UNIT, "cores": 1,
                            "sample": f"one full FP64 iteration at K={k_1}, {el1:.1f} s"}
    return rec, r, k_s


def error_vs_oracle(mp, prob, k: int, orc, local: int, params=None, gated: bool = True) -> dict:
    """The CUDA path against the FP64 oracle on the same workload cut to K = k samples (the noise
    of sample j does not depend on K): every sample cost, the argmin, u* and x* of one iteration
    from a zero warm start."""
    import numpy as np
    p = dict(prob.params if params is None else params, K=int(k))
    with mp.Planner(p, device=local) as pl:
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles, prob.centres)
        S = pl.get_costs()
    rel = np.abs(S - orc.S) / np.maximum(np.abs(orc.S), 1.0)
    order = np.argsort(orc.S, kind="stable")
    s1 = orc.S[order[0]]
    near = set(np.nonzero(orc.S - s1 <= 1e-4 * max(abs(s1), 1.0))[0].tolist())
    return {"samples": int(k), "max_rel_S": float(rel.max()), "median_rel_S": float(np.median(rel)),
            "argmin_ok": bool(info["argmin"] in near), "max_abs_du_star": float(np.abs(u - orc.u_star).max()),
            "max_abs_dx_star": float(np.abs(x - orc.x_star).max()),
            **({"tolerance": {"S_rel": 1e-4, "u_abs": 1e-4, "x_abs": 1e-4}} if gated else
               {"note": "the error of storing the noise as bfloat16 itself (not a parity check)"})}


# ------------------------------------------------------------------------ the GPU arm

def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2308_01654_gb300 as mp
    from paper_2308_01654_gb300 import scenarios

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prob = scenarios.by_name(args.workload)
    prob.params["session"] = rank_session(rank)        # an independent planning problem per rank
    K, T = prob.K, prob.T
    stream = torch.cuda.Stream(device=dev)             # the planner and the timing events share it
    torch.cuda.set_stream(stream)
    pl = mp.Planner(prob.params, device=local, stream=stream.cuda_stream)
    group, block = pl.autotune(prob.x0, prob.ref, prob.circles, prob.centres, cache_path=args.tune_cache)
    work = pl.rollout_stats(prob.x0, prob.ref, prob.circles, prob.centres)     # untimed, instrumented copy
    # events around the rollout kernel only: an event between two kernels ends their chaining,
    # so the other kernels of the timed steps stay chained as in an untraced iteration
    pl.set_profiling(2)
    x0 = torch.tensor(prob.x0, dtype=torch.float64, device=dev)
    ref = torch.tensor(prob.ref, dtype=torch.float64, device=dev)
    circ = torch.tensor(prob.circles, dtype=torch.float64, device=dev)
    cen = None if prob.centres is None else torch.tensor(prob.centres, dtype=torch.float64, device=dev)
    u_out = torch.empty((T, 2), dtype=torch.float64, device=dev)
    nx = prob.x0.shape[0]                              # 4, or 5 for the steering-rate model
    x_out = torch.empty((T + 1, nx), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step():
        pl.plan_device(x0, ref, circ, cen, u_out, x_out)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    info = pl.sync()
    assert info["n_finite"] > 0

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    sampler = ClockSampler(gpu_id_for(local)) if not (args.no_clocks or args.quick) else None
    barrier()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    step_ms, roll_ms, ktimes = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        kt = pl.kernel_times()                         # waits for this step
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        roll_ms.append(kt["rollout"])
    barrier()
    clocks = sampler.stop() if sampler else None
    pl.sync()
    # per-kernel breakdown on a few untimed steps with an event at every kernel boundary
    pl.set_profiling(True)
    for _ in range(3):
        flush.zero_()
        step()
        ktimes.append(pl.kernel_times())
    pl.set_profiling(False)

    ms_step = statistics.mean(step_ms)
    ms_roll = statistics.mean(roll_ms)
    ms_step, ms_roll = max_over_ranks([ms_step, ms_roll], world, dev)
    value = weak_value(K * T, world, ms_step * 1e-3)

    # end to end through the host-buffer C ABI: H2D of inputs and D2H of outputs every step
    h2d = 8 * (prob.x0.size + prob.ref.size + prob.circles.size + (0 if prob.centres is None else prob.centres.size))
    d2h = 8 * (2 * T + nx * (T + 1))
    e2e = None
    if not args.quick:
        p_e = dict(prob.params, group=group, block=block)
        with mp.Planner(p_e, device=local) as pe:
            for _ in range(max(1, args.warmup)):
                pe.plan(prob.x0, prob.ref, prob.circles, prob.centres)
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                pe.plan(prob.x0, prob.ref, prob.circles, prob.centres)
            e2e_s = (time.perf_counter() - t0) / args.steps
        (e2e_s,) = max_over_ranks([e2e_s], world, dev)
        e2e = {"value": weak_value(K * T, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3}

    # roofline of the rollout kernel: FP32-pipe bound (no dense contraction, noise bytes << compute)
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tops = n_sm * 128 * f_max * 1e6 / 1e12
    ops_step = executed_ops_per_step(work)
    achieved = ops_step * K * T / (ms_roll * 1e-3) / 1e12
    bf_step = brute_force_ops_per_step(prob)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "TOP/s",
                "frac": achieved / peak_tops,
                "traffic": args.traffic if args.traffic is not None else profiled_traffic(args.workload),
                "kernel": "rollout_kernel", "ops_per_rollout_step": ops_step,
                # issue slots used by the same launch (ncu smsp__issue_active, committed summary)
                "issue_active_frac": (lambda v: None if v is None else v / 100.0)(
                    profiled_value(args.workload, "issue_active_pct")),
                # counted from one ncu capture of the same build (committed summary): the arithmetic
                # thread instructions per rollout-step (FP32, integer, bit and conversion classes),
                # and the fraction of the peak they would give at this launch's duration
                "counted_model": counted_model(args.workload, K * T, ms_roll, peak_tops),
                "work_per_rollout_step": {k: round(v, 4) for k, v in work.items()},
                "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {f_max:.0f} MHz (max SM clock)",
                "kernel_ms": ms_roll,
                # the dense per-step count (every ego/obstacle pair tested, 32-segment chunk bounds
                # with ~2 chunks scanned): the kernel's exact pruning skips most of it, so its
                # fraction exceeds 1 and measures work avoided rather than pipe use
                "dense_model": {"ops_per_rollout_step": bf_step,
                                "achieved": bf_step * K * T / (ms_roll * 1e-3) / 1e12,
                                "frac": bf_step * K * T / (ms_roll * 1e-3) / 1e12 / peak_tops}}
    kmean = {k: statistics.mean(d[k] for d in ktimes) for k in ktimes[0]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" + ("+bf16-noise" if prob.params["noise_bf16"] else "") + "+f64-reduce",
        "data": "synthetic (seeded generator shaped like the paper's driving scenes)",
        "config": {"workload": f"{prob.name}: K={K} T={T} dt={prob.params['dt']} n_ref={prob.ref.shape[0]} "
                               f"n_circ={prob.circles.shape[0]}", "K": K, "T": T,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed between steps (256 MB write)",
                   "rollout_launch": launch_desc(group, block)},
        "e2e": e2e, "roofline": roofline, "gpu_launches": (KERNEL_LAUNCHES_PER_STEP + int(bool(prob.params.get("noise_bf16", 0)))) * args.steps,
        "kernel_ms": kmean, "kernel_ms_note": "untimed steps with an event at every kernel boundary (unchained)",
        "clocks": clocks,
    }
    pl.close()
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.quick):
        rec, orc, k_s = cpu_baseline_record(prob, args.cpu_seconds)
        out["cpu_baseline"] = rec
        out["error_vs_oracle"] = error_vs_oracle(mp, prob, k_s, orc, local)
    if args.workload == "roofline" and not (args.quick or args.no_systems):
        # the other forms the metric names, shortened so the default run stays within minutes
        out["bf16_noise"] = bf16_report(args, world, rank, local)
        out["systems"] = {
            "batched": batched_report(args, world, rank, local, steps=5),
            "serving": serving_report(args, world, rank, local, rate=args.rate, warm=1.0, meas=3.0),
            "serving_saturated": serving_report(args, world, rank, local, rate=4.0 * args.rate, warm=1.0,
                                                meas=2.0),
            "note": ("at the 2000 plans/s offered load both the server and the plain loop keep up, so "
                     "plans/s match and the server's gain is latency; the plans/s advantage appears above "
                     "the plain loop's saturation point (serving_saturated)"),
        }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def bf16_report(args, world, rank, local, steps: int = 10) -> dict:
    """The roofline workload with the noise stored as bfloat16 (the precision form): device-timed
    rollout-steps/s, and its error against the FP64 oracle on a K-sample, both on the same bf16
    codes (the same method) and against the unrounded FP64 noise."""
    import torch

    import paper_2308_01654_gb300 as mp
    from paper_2308_01654_gb300 import scenarios
    dev = torch.device("cuda", local)
    prob = scenarios.roofline(bf16=True)
    prob.params["session"] = rank_session(rank)
    K, T = prob.K, prob.T
    stream = torch.cuda.Stream(device=dev)
    with mp.Planner(prob.params, device=local, stream=stream.cuda_stream) as pl:
        group, block = pl.autotune(prob.x0, prob.ref, prob.circles, prob.centres, cache_path=args.tune_cache)
        x0 = torch.tensor(prob.x0, dtype=torch.float64, device=dev)
        ref = torch.tensor(prob.ref, dtype=torch.float64, device=dev)
        circ = torch.tensor(prob.circles, dtype=torch.float64, device=dev)
        u_out = torch.empty((T, 2), dtype=torch.float64, device=dev)
        x_out = torch.empty((T + 1, 4), dtype=torch.float64, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                flush.zero_()
                pl.plan_device(x0, ref, circ, None, u_out, x_out)
            pl.sync()
            ms = []
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.plan_device(x0, ref, circ, None, u_out, x_out)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        pl.sync()
    (m,) = max_over_ranks([statistics.mean(ms)], world, dev)
    rec = {"value": weak_value(K * T, world, m * 1e-3), "unit": UNIT, "ms_per_step": m, "steps": steps,
           "noise_bytes_per_rollout_step": 4, "rollout_launch": launch_desc(group, block)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        k = 2048
        q = prob.copy()
        q.params["K"] = k
        rec["error_vs_oracle_same_codes"] = error_vs_oracle(mp, prob, k, oracle.plan(q), local)
        rec["error_vs_oracle_unrounded"] = error_vs_oracle(
            mp, prob, k, oracle.plan(q, params=dict(q.params, noise_bf16=0)), local, gated=False)
    return rec


# ------------------------------------------------------------------------ batched uneven plans

def run_batched(args, world, rank, local):
    """256 uneven plans per submission through mppi_batch_plan, against the plain per-plan loop."""
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = batched_report(args, world, rank, local, steps=args.steps, full_line=True)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def batched_report(args, world, rank, local, steps: int, full_line: bool = False) -> dict:
    import numpy as np
    import torch

    import paper_2308_01654_gb300 as mp
    from paper_2308_01654_gb300 import scenarios
    probs = scenarios.batched(seed=0, n=args.batch_size)
    for p in probs:
        p.params["session"] = rank_session(rank, int(p.params["session"]))
    n = len(probs)
    sum_k = sum(p.K for p in probs)
    sum_kt = sum(p.K * p.T for p in probs)
    max_t = max(p.T for p in probs)
    max_ref = max(p.ref.shape[0] for p in probs)
    max_circ = max(max(p.circles.shape[0] for p in probs), 1)
    bp = mp.BatchPlanner(max_slots=n, max_batch=n, max_samples=sum_k, max_rollout_steps=sum_kt, max_T=max_t,
                         max_ref=max_ref, max_circ=max_circ, pipelines=2, device=local)
    plans = [mp.BatchPlan(p.params, i, p.x0, p.ref, p.circles, p.centres) for i, p in enumerate(probs)]
    group, block = bp.autotune(plans)
    reqs = bp.requests(plans)
    for _ in range(args.warmup):
        bp.plan(plans, reqs)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    barrier()
    lat = []
    t0 = time.perf_counter()
    for _ in range(steps):
        a = time.perf_counter()
        bp.plan(plans, reqs)
        lat.append(time.perf_counter() - a)
    t_batch = (time.perf_counter() - t0) / steps
    barrier()
    bad = sum(p.info.n_finite == 0 for p in plans)
    bp.close()

    # the plain path: one context per plan, plans one after another on one stream
    ctxs = [mp.Planner(p.params, device=local, max_ref=max_ref, max_circ=max_circ) for p in probs]
    for pl, p in zip(ctxs, probs):
        pl.plan(p.x0, p.ref, p.circles, p.centres)
    barrier()
    t0 = time.perf_counter()
    reps = max(1, min(steps, 3))
    for _ in range(reps):
        for pl, p in zip(ctxs, probs):
            pl.plan(p.x0, p.ref, p.circles, p.centres)
    t_plain = (time.perf_counter() - t0) / reps
    for pl in ctxs:
        pl.close()
    t_batch, t_plain = max_over_ranks([t_batch, t_plain], world, "cuda")
    rec = {"value": weak_value(n, world, t_batch), "unit": "plans/s", "steps": steps,
           "workload": f"batched: {n} uneven plans per submission (K 2^10..2^14, T 30..150, 0..32 obstacles), "
                       f"sum K = {sum_k}, sum K*T = {sum_kt}",
           "rollout_launch": launch_desc(group, block),
           "timing": "wall clock of mppi_batch_plan (host packing, H2D, graph, D2H, unpacking)",
           "rollout_steps_per_s": world * sum_kt / t_batch,
           "submission_ms": {"p50": float(np.percentile(lat, 50)) * 1e3, "p99": float(np.percentile(lat, 99)) * 1e3},
           "plain_per_plan_loop": {"value": world * n / t_plain, "unit": "plans/s", "ms_per_pass": t_plain * 1e3,
                                   "rollout_steps_per_s": world * sum_kt / t_plain},
           "speedup_vs_plain": t_plain / t_batch, "plans_without_finite_cost": int(bad)}
    if not full_line:
        return rec
    return {"metric": f"plans/s ({n} uneven plans per submission, batched)", "value": rec["value"],
            "unit": "plans/s", "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64-reduce", "data": "synthetic (uneven plans: K in 2^10..2^14, T 30..150, 0..32 obstacles)",
            "config": {"workload": rec["workload"], "rollout_launch": rec["rollout_launch"], "timing": rec["timing"]},
            **{k: rec[k] for k in ("rollout_steps_per_s", "submission_ms", "plain_per_plan_loop", "speedup_vs_plain",
                                   "plans_without_finite_cost")}}


# ------------------------------------------------------------------------ closed loop

def run_closed_loop(args, world, rank, local):
    """The 200-cycle receding-horizon loop on the curved lane through mppi_plan (host buffers)."""
    import numpy as np
    import torch

    from paper_2308_01654_gb300 import closed_loop, scenarios

    torch.cuda.set_device(local)
    dist_init(world, local)
    prob = scenarios.closed_loop()
    prob.params["session"] = rank_session(rank)
    res = closed_loop.run(prob, cycles=args.cycles, device=local)
    t = res.plan_ms[3:] if len(res.plan_ms) > 6 else res.plan_ms
    K, T = prob.K, prob.T
    (p50,) = max_over_ranks([float(np.median(t))], world, "cuda")
    out = {"metric": "rollout-steps/s (K*T) of one MPPI iteration per control cycle, closed loop",
           "value": weak_value(K * T, world, p50 * 1e-3), "unit": "rollout-steps/s", "n_gpus": world,
           "steps": args.cycles, "warmup": 3, "ms_per_step": p50, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64-reduce", "data": "synthetic",
           "config": {"workload": f"closed_loop: K={K} T={T}, {args.cycles} cycles, sinusoidal lane, 8 obstacles "
                                  f"(4 moving, per-step centre table)",
                      "timing": "wall clock of mppi_plan per cycle (host buffers, CUDA graph replay)"},
           "cycle_ms": {"p50": float(np.median(t)), "p99": float(np.percentile(t, 99)), "mean": float(np.mean(t))},
           "run": {"min_clearance_m": res.min_clearance, "max_abs_steer": float(np.abs(res.controls[:, 1]).max()),
                   "max_abs_accel": float(np.abs(res.controls[:, 0]).max()),
                   "final_state": [float(v) for v in res.states[-1]],
                   "max_speed": float(res.states[:, 3].max())}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_done(world)


def scenario_report(name: str, cycles: int, device: int = 0) -> dict:
    """One closed-loop primitive on the steering-rate model with the paper's preset: what its
    qualitative gates look at (clearance, speed against v_G, steering, lateral offset)."""
    import numpy as np

    from paper_2308_01654_gb300 import closed_loop, scenarios
    prob = scenarios.by_name(name)
    res = closed_loop.run(prob, cycles=cycles, device=device)
    xs = res.states
    t = res.plan_ms[3:] if len(res.plan_ms) > 6 else res.plan_ms
    return {"cycles": cycles, "min_clearance_m": res.min_clearance,
            "max_speed": float(xs[:, 3].max()), "v_G": float(prob.params["v_max"]),
            "max_abs_steer": float(np.abs(xs[:, 4]).max()), "max_abs_rate": float(np.abs(res.controls[:, 1]).max()),
            "final_y": float(xs[-1, 1]), "final_speed": float(xs[-1, 3]), "final_x": float(xs[-1, 0]),
            "plan_ms": {"p50": float(np.median(t)), "p99": float(np.percentile(t, 99))}}


def run_scenarios(args, world, rank, local):
    """The scenario primitives (merge, follow, avoid) as closed loops on one GPU."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    rep = {n: scenario_report(n, args.cycles, local) for n in ("merge", "follow", "avoid")}
    p50 = float(np.median([r["plan_ms"]["p50"] for r in rep.values()]))
    out = {"metric": "closed-loop plans/s (scenario primitives, steering-rate model, Table I preset)",
           "value": 1e3 / p50, "unit": "plans/s", "n_gpus": world, "steps": 3 * args.cycles, "warmup": 3,
           "ms_per_step": p50, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64-reduce", "data": "synthetic",
           "config": {"workload": f"scenarios: merge, follow, avoid; {args.cycles} cycles of 0.25 s each; "
                                  f"K=2560 T=16"},
           "scenarios": rep}
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------ serving

def serving_trace(sessions, rate: float, seconds: float, seed: int = 5, variants: int = 4):
    """Poisson arrivals at `rate` plans/s, sessions drawn uniformly, obstacles redrawn per request
    (one of `variants` perturbed copies of the session's obstacle set)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    obst = []
    for p in sessions:
        vs = []
        for _ in range(variants):
            c = p.circles.copy()
            if c.shape[0]:
                c[:, :2] += rng.normal(scale=0.5, size=(c.shape[0], 2))
            vs.append(np.ascontiguousarray(c))
        obst.append(vs)
    t, out = 0.0, []
    while t < seconds:
        t += rng.exponential(1.0 / rate)
        s = int(rng.integers(0, len(sessions)))
        out.append((t, s, obst[s][int(rng.integers(0, variants))]))
    return out


def run_serving(args, world, rank, local):
    """Continuous batching of 512 sessions at a Poisson 2000 plans/s against the plain FIFO loop."""
    import torch
    torch.cuda.set_device(local)
    dist_init(world, local)
    rec = serving_report(args, world, rank, local, rate=args.rate, warm=args.serve_warmup_s, meas=args.serve_seconds)
    out = {"metric": f"served plans/s ({args.sessions} sessions, Poisson {args.rate:.0f} plans/s offered)",
           "value": rec["value"], "unit": "plans/s", "n_gpus": world, "steps": rec["requests"], "warmup": 0,
           "ms_per_step": rec["latency_ms"]["p50"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64-reduce", "data": "synthetic sessions (K 2^10..2^14, T 30..150, 0..32 obstacles)",
           "config": {"workload": rec["workload"], "pipelines": args.pipelines, "max_wait_us": args.max_wait_us},
           **{k: rec[k] for k in ("latency_ms", "server", "plain_per_plan_loop")}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_done(world)


def serving_report(args, world, rank, local, rate: float, warm: float, meas: float) -> dict:
    """One Poisson trace at `rate` plans/s through the server and through the plain FIFO loop
    (one context per session, requests one at a time in arrival order).  Latency = completion -
    arrival; plans/s = completions inside the measured window.  Every request must complete."""
    import queue as queue_mod

    import numpy as np

    import paper_2308_01654_gb300 as mp
    from paper_2308_01654_gb300 import scenarios

    sessions = scenarios.serving_sessions(seed=0, n=args.sessions)
    for p in sessions:
        p.params["shift"] = 1
        p.params["session"] = rank_session(rank, int(p.params["session"]))
    cparams = [mp.make_params(p.params) for p in sessions]
    trace = serving_trace(sessions, rate, warm + meas)
    max_t = max(p.T for p in sessions)
    max_ref = max(p.ref.shape[0] for p in sessions)
    max_circ = max(max(p.circles.shape[0] for p in sessions), 1)

    def summarise(lat_arr, t_arr, done_t, label):
        lat_arr, t_arr, done_t = np.asarray(lat_arr), np.asarray(t_arr), np.asarray(done_t)
        m = (t_arr >= warm) & (t_arr < warm + meas)
        completed = int(np.sum((done_t >= warm) & (done_t < warm + meas)))
        return {"plans_per_s": completed / meas, "p50_ms": float(np.percentile(lat_arr[m], 50)) / 1e3,
                "p99_ms": float(np.percentile(lat_arr[m], 99)) / 1e3, "max_ms": float(lat_arr[m].max()) / 1e3,
                "requests": int(m.sum()), "label": label}

    # --- continuous batching server
    srv = mp.Server(max_sessions=len(sessions), max_batch=256, max_samples=2_000_000, max_rollout_steps=200_000_000,
                    max_T=max_t, max_ref=max_ref, max_circ=max_circ, pipelines=args.pipelines,
                    hbm_budget_bytes=args.hbm_budget_gb << 30, max_wait_us=args.max_wait_us, device=local)
    # tune for the micro-batches the trace produces: a few plans of median size
    by_size = sorted(range(len(sessions)), key=lambda i: sessions[i].K * sessions[i].T)
    mid = by_size[len(by_size) // 2]
    tune_n = max(1, min(8, int(round(rate * 1e-3))))             # ~ plans arriving per millisecond
    group, block = srv.autotune(cparams[mid], sessions[mid].x0, sessions[mid].ref, sessions[mid].circles, tune_n)
    ids = {}                     # request id -> trace index (written after enqueue returns)
    got = {}                     # request id -> (latency_us, completion time, status), in any order
    n_enq = [0]
    t0 = [0.0]
    stop = threading.Event()

    def collector():
        deadline = None
        while True:
            for r in srv.poll(1024, wait_ms=20):
                # a result may come back before its enqueue has returned and its id is registered:
                # keep it by id and match it to the trace afterwards
                got[r["request_id"]] = (r["latency_us"], time.perf_counter() - t0[0], r["status"])
            if stop.is_set():
                if len(got) >= n_enq[0]:
                    return
                deadline = deadline or time.perf_counter() + 60.0
                if time.perf_counter() > deadline:
                    return

    th = threading.Thread(target=collector, daemon=True)
    t0[0] = time.perf_counter()
    th.start()
    for j, (t, s, circ) in enumerate(trace):
        now = time.perf_counter() - t0[0]
        if t > now:
            time.sleep(t - now)
        p = sessions[s]
        rid = srv.enqueue(cparams[s], s, p.x0, p.ref, circ if circ.shape[0] else None)
        ids[rid] = j
        n_enq[0] += 1
    stop.set()
    th.join(timeout=90)
    st = srv.pending()
    srv.close()
    lost = [rid for rid in ids if rid not in got]
    failed = sum(1 for rid in ids if rid in got and got[rid][2] != 0)
    if lost or failed:
        raise RuntimeError(f"serving: {len(lost)} of {len(ids)} requests never completed, {failed} failed")
    order = sorted(ids, key=lambda rid: ids[rid])
    served = summarise([got[r][0] for r in order], [trace[ids[r]][0] for r in order], [got[r][1] for r in order],
                       "server")
    served.update(batches=st["batches"], plans=st["plans"], mean_batch=st["plans"] / max(st["batches"], 1),
                  lost=len(lost), failed=failed, rollout_launch=launch_desc(group, block))

    # --- plain loop: one context per session, one request at a time in arrival order
    ctxs = [mp.Planner(p.params, device=local, max_ref=max_ref, max_circ=max_circ) for p in sessions]
    q = queue_mod.Queue()
    plat, parr, pdone = [], [], []

    def worker():
        while True:
            item = q.get()
            if item is None:
                return
            j, ta = item
            t, s, circ = trace[j]
            p = sessions[s]
            ctxs[s].plan(p.x0, p.ref, circ if circ.shape[0] else None)
            tdone = time.perf_counter() - t0[0]
            plat.append((tdone - ta) * 1e6)
            parr.append(t)
            pdone.append(tdone)

    w = threading.Thread(target=worker, daemon=True)
    t0[0] = time.perf_counter()
    w.start()
    for j, (t, s, circ) in enumerate(trace):
        now = time.perf_counter() - t0[0]
        if t > now:
            time.sleep(t - now)
        q.put((j, time.perf_counter() - t0[0]))
    q.put(None)
    w.join(timeout=600)
    for c in ctxs:
        c.close()
    plain = summarise(plat, parr, pdone, "plain FIFO mppi_plan loop")
    mean_kt = float(np.mean([sessions[s].K * sessions[s].T for _, s, _ in trace]))
    # every rank serves its own sessions: plans/s add up, latency is the worst rank's
    (total, plain_total) = sum_over_ranks([served["plans_per_s"], plain["plans_per_s"]], world, "cuda")
    p50_all, p99_all = max_over_ranks([served["p50_ms"], served["p99_ms"]], world, "cuda")
    return {"value": total, "unit": "plans/s", "offered_plans_per_s": rate * world, "requests": len(trace),
            "workload": f"serving: {len(sessions)} sessions, Poisson {rate:.0f} plans/s, {warm:.0f} s warm-up + "
                        f"{meas:.0f} s measured, mean K*T {mean_kt:.0f}",
            "latency_ms": {"p50": p50_all, "p99": p99_all, "max": served["max_ms"]},
            "server": served, "plain_per_plan_loop": dict(plain, plans_per_s_all_ranks=plain_total)}


# ------------------------------------------------------------------------ the reference arm (the oracle)

def run_reference(args, world, rank, local):
    if rank != 0:
        return
    import oracle
    from paper_2308_01654_gb300 import scenarios
    if args.workload in ("batched", "serving"):
        prob = scenarios.batched(seed=0, n=1)[0]        # one instance of the uneven mix
    elif args.workload == "closed_loop_run":
        prob = scenarios.closed_loop()                 # one cycle's iteration
    else:
        prob = scenarios.by_name(args.workload)
    T = prob.T
    budget = max(2.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    k_s = oracle_sample(prob, budget)
    for _ in range(args.warmup):
        time_oracle(prob, min(k_s, 64))
    times = [time_oracle(prob, k_s) for _ in range(args.steps)]
    s = statistics.mean(times)
    value = k_s * T / s
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"{prob.name}: K={prob.K} T={T} (timed on a K={k_s} sample per step)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"one full FP64 iteration at K={k_s} of the same workload per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="roofline",
                    choices=["roofline", "roofline_bf16", "closed_loop", "single_plan", "batched", "serving",
                             "closed_loop_run", "paper_preset", "scenarios"])
    ap.add_argument("--cycles", type=int, default=200)
    ap.add_argument("--batch-size", type=int, default=256)
    ap.add_argument("--sessions", type=int, default=512)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--serve-warmup-s", type=float, default=2.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--pipelines", type=int, default=3)
    ap.add_argument("--max-wait-us", type=float, default=0.0)
    ap.add_argument("--hbm-budget-gb", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-systems", action="store_true",
                    help="default workload only: skip the bf16, batched and serving records")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (read first, appended after tuning)")
    ap.add_argument("--quick", action="store_true",
                    help="device timing only (no e2e, clocks or CPU baseline): the profiling run")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per rollout launch from an ncu capture of the current kernel")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "serving":
        run_serving(args, world, rank, local)
    elif args.workload == "closed_loop_run":
        run_closed_loop(args, world, rank, local)
    elif args.workload == "scenarios":
        run_scenarios(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)


if __name__ == "__main__":
    main()
