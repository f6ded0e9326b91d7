#!/usr/bin/env python
"""Benchmark of the exact ddKS hot path on GB300.

Default workload: exact ddKS, d = 4, NP = NT = 20,000 float32 (P ~ N(0, I4);
T with corr(x0, x1) = 0.5 and 1% of its rows exact copies of P rows).  One step
is one ddks_distance call over the device-resident inputs (rank encoding,
orthant counts, max over origins, result to the host).  The metric is
origin*point*dim compares per second: N^2 * d per step, N = NP + NT.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead.
Under torchrun every rank runs its own replica of the workload (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ddks_compares_per_s"
UNIT = "compares/s"


PATH_NAMES = ["auto", "register", "lane", "warp", "sort", "dominance", "byte"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["cfg2", "cfg1", "cfg3", "perm", "batch", "serve", "vdks", "rdks",
                                           "rdks_large", "dom2d"], default="cfg2")
    ap.add_argument("--perms", type=int, default=1000)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--path", type=int, default=0, help="force a kernel path (0 = auto)")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-study", action="store_true", help="perm workload: skip the significance study")
    ap.add_argument("--shard", choices=["origins", "replicas"], default="origins",
                    help="N > 1: split one problem's origins across the ranks (strong scaling, exact max "
                         "merge) or run one whole problem per rank (weak scaling)")
    return ap.parse_args()


WORKLOADS = {
    "cfg2": ("cfg2_d4_20000x20000_f32_ties", "exact ddKS d=4 NP=NT=20000 f32, corr(x0,x1)=0.5, 1% tied T rows"),
    "cfg1": ("cfg1_d3_200x200_f32", "exact ddKS d=3 NP=NT=200 f32 gaussian, T shifted by 0.2"),
    "cfg3": ("cfg3_d12_4096x4096_f64", "exact ddKS d=12 NP=NT=4096 f64 uniform, T coord 5 ~ Beta(2,2)"),
}


# The approximations of Sec. 2.2, each measured under its own metric.
APPROX = {
    "vdks": ("vdKS (Alg. vdKS) d=3 NP=NT=8,000,000 f32, P ~ N(0,I3), T ~ N(0.2*1,I3), 32 voxels per dimension",
             "vdks_points_per_s", "points/s"),
    "rdks": ("rdKS (Alg. rdKS) d=1000 NP=NT=100 f32, diagonal versus uniform (Sec. 4's 1000-dimensional case)",
             "rdks_tests_per_s", "tests/s"),
    "rdks_large": ("rdKS (Alg. rdKS) d=3 NP=NT=1,000,000 f32, P ~ N(0,I3), T ~ N(0.05*1,I3)",
                   "rdks_points_per_s", "points/s"),
}


def approx_inputs(name):
    """(P, T, voxels per dimension or None) of an approximation workload."""
    from paper_2106_13706_gb300 import workloads as wl
    if name == "vdks":
        return wl.gaussian_pair(0, 8_000_000, 8_000_000, 3, shift=0.2) + (32,)
    if name == "rdks":
        return wl.dvu_pair(0, 100, 100, 1000) + (None,)
    return wl.gaussian_pair(0, 1_000_000, 1_000_000, 3, shift=0.05) + (None,)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed loop runs."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "20", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peak_lane_ops(torch, dev, sm_max_mhz):
    """Integer issue roofline: SMs x 4 sub-partitions x 32 lanes x max SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    return sms * 128 * mhz * 1e6, sms, mhz


def pipe_mix(torch, dev, sm_max_mhz, path, d, NP, NT, origins, count_ms):
    """Instruction-mix roofline of the bit-sliced count kernel (register path,
    d = 2..4): its algorithmic operations per launch on each pipe against the
    pipe's rate, and the count stage's time against the slowest pipe.

    Per origin and group of 32 points: 7 (d - 1) three-input logic ops for the
    compares and one AND per subset of two or more of dimensions 1..d-1 (ALU
    pipe, 64 lanes/clk/SM), one popcount (XU pipe, 32 lanes/clk/SM, measured)
    and one add (FMA pipe, 64 lanes/clk/SM) per non-empty subset; the shared
    group loads add 2 (d - 1) 16-byte broadcast loads per 2 origins.  Issue:
    one warp instruction per clock per scheduler (4 per SM)."""
    if path != "register" or not 2 <= d <= 4:
        return None
    p = torch.cuda.get_device_properties(dev)
    f = (sm_max_mhz or 2070.0) * 1e6
    sms = p.multi_processor_count
    ds = d - 1
    subsets = (1 << ds) - 1
    og = float(origins) * ((NP + 31) // 32 + (NT + 31) // 32)  # origin x group-of-32 units
    alu = og * (7 * ds + (subsets - ds))
    xu = og * subsets
    fma = og * subsets
    lds = og * ds  # two 16-byte loads per dimension, shared by two origins
    t = {"alu": alu / (sms * 64 * f), "xu": xu / (sms * 32 * f), "fma": fma / (sms * 64 * f),
         "issue": (alu + xu + fma + lds) / 32 / (sms * 4 * f)}
    bound = max(t, key=t.get)
    return {"lane_ops_per_launch": {"alu": alu, "xu": xu, "fma": fma},
            "pipe_ms": {k: v * 1e3 for k, v in t.items()}, "bound_pipe": bound,
            "frac_of_bound": t[bound] * 1e3 / count_ms,
            "note": "count stage (re-rank pack + count kernel) time against the count kernel's slowest pipe"}


def peak_compares(torch, dev, sm_max_mhz, path, d):
    """Compare-rate roofline of the count kernel's path, in compares/s.

    Register path (d = 2..4, bit-sliced): one 3-input logic op on the ALU pipe
    (64 lanes/clk/SM) decides one bit of 32 seven-bit comparisons, so a pair
    costs 7 (d - 1) / 32 ALU lane-ops and its dimension 0 none (sorted order):
    peak = SMs x 64 x clock x 32 d / (7 (d - 1)).  Other paths compare one
    dimension of one pair per lane-op: peak = SMs x 128 lanes x clock."""
    lanes, sms, mhz = peak_lane_ops(torch, dev, sm_max_mhz)
    if path == "register" and d >= 2:
        peak = sms * 64 * mhz * 1e6 * 32.0 * d / (7.0 * (d - 1))
        basis = (f"{sms} SMs x 64 ALU lanes x {mhz:.0f} MHz x 32 bit slices x d/(7(d-1)) "
                 "(7 logic ops per 32 seven-bit compares; dimension 0 by sorted order)")
        return peak, basis
    return lanes, f"{sms} SMs x 128 int lanes x {mhz:.0f} MHz (max SM clock)"


def load_traffic(kernel_key):
    """DRAM bytes per launch of the count kernel from the committed ncu summary
    (profiles/traffic.json), if it was taken on the current kernel source."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p)).get(kernel_key)
    except (ValueError, OSError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec.get("source_sha256_16"):
        return None
    return rec.get("bytes_per_launch")


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2106_13706_gb300 as pkg
    from paper_2106_13706_gb300 import build as bld
    from paper_2106_13706_gb300 import workloads as wl

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    bld.build()
    key, desc = WORKLOADS[args.workload]
    P, T = wl.CONFIGS[key]()
    NP, d = P.shape
    NT = T.shape[0]
    N = NP + NT
    units = float(N) * N * d
    Pd = torch.from_numpy(P).cuda()
    Td = torch.from_numpy(T).cuda()
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device="cuda")
    ctx = pkg.Context(device=local, path=args.path)
    from paper_2106_13706_gb300 import sharding
    shard = args.shard if world > 1 else "none"
    if shard == "origins":
        o_begin, o_end = sharding.shard_range(N, world, rank)
        call = lambda A, B: ctx.distance_range(A, B, o_begin, o_end)  # noqa: E731
    else:
        call = ctx.distance
    tuned = None
    if args.path == 0 and not args.no_autotune:
        tuned = ctx.autotune(Pd, Td)  # the project's autotuner picks the kernel shape
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        ref = call(Pd, Td)  # repeated calls are replayed as one CUDA graph
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = ctx.stats()["kernel_launches"]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        r = call(Pd, Td)
        ev[s][1].record(stream)
        if r["num_max"] != ref["num_max"]:
            raise RuntimeError("result changed between steps")
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = ctx.stats()["kernel_launches"] - launches0
    sampler.stop()
    # the stages, kernel by kernel with events between them (stage timing
    # turns graph replay off), for the roofline of the count stage
    count_ms, enc_ms, red_ms = [], [], []
    ctx.set_stage_timing(True)
    for s in range(min(args.steps, 50)):
        flush.zero_()
        call(Pd, Td)
        st3 = ctx.stage_times()
        enc_ms.append(st3[0])
        count_ms.append(st3[1])
        red_ms.append(st3[2])
    ctx.set_stage_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    mult = world if shard == "replicas" else 1  # origin shards make up one problem together
    value = units * args.steps * mult / (total_ms * 1e-3)
    if shard == "origins":
        ref = sharding.all_merge(ref)  # the whole problem's result, on every rank

    # end to end through the same C call with pinned host inputs: the H2D copy
    # of P and T and the D2H copy of the result are inside each timed call
    e2e = None
    if not args.no_e2e:
        Ph = torch.from_numpy(P).pin_memory()
        Th = torch.from_numpy(T).pin_memory()
        for _ in range(3):
            call(Ph, Th)
        torch.cuda.synchronize()
    if not args.no_e2e:
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = time.perf_counter()
            r2 = call(Ph, Th)
            tot += time.perf_counter() - a
        if shard == "origins":
            r2 = sharding.all_merge(r2)
            t2 = torch.tensor([tot], dtype=torch.float64, device="cuda")
            dist.all_reduce(t2, op=dist.ReduceOp.MAX)
            tot = float(t2.item())
        if r2["num_max"] != ref["num_max"]:
            raise RuntimeError("host-input result differs")
        e2e = {"value": units * args.steps * mult / tot, "unit": UNIT,
               "h2d_bytes_per_step": int(Ph.numel() * Ph.element_size() + Th.numel() * Th.element_size()),
               "d2h_bytes_per_step": 3 * 8 + 4}

    clocks = sampler.summary()
    path_name = (PATH_NAMES[tuned[0]] if tuned else
                 PATH_NAMES[args.path])
    if path_name == "auto":
        path_name = "register" if 2 <= d <= 4 else ("warp" if d <= 13 else "sort")
    peak, basis = peak_compares(torch, local, clocks.get("sm_max_mhz"), path_name, d)
    lane_peak = peak_lane_ops(torch, local, clocks.get("sm_max_mhz"))[0]
    cnt = statistics.mean(count_ms) if count_ms else None
    roof = None
    if cnt:
        # this rank's compares: all points against its origins
        units_rank = units * ((o_end - o_begin) / N if shard == "origins" else 1.0)
        achieved = units_rank / (cnt * 1e-3)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": UNIT,
                "frac": achieved / peak, "traffic": load_traffic({"cfg2": "count_d4_20k"}.get(args.workload, "")),
                "kernel": "orthant count stage (re-rank pack + count + fused reduction)", "kernel_ms": cnt,
                "peak_basis": basis, "compares_per_lane_op": achieved / lane_peak,
                "pipe_mix": pipe_mix(torch, local, clocks.get("sm_max_mhz"), path_name, d, NP, NT,
                                     (o_end - o_begin) if shard == "origins" else N, cnt),
                "stage_ms": {"encode": statistics.mean(enc_ms), "count": cnt, "reduce": statistics.mean(red_ms)}}

    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, oref = cpu_baseline(P, T, d)
        # the oracle ran over every origin: the timed result must equal it
        got = (ref["num_max"], ref["denom"], ref["argmax_origin"], ref["argmax_orthant"])
        want = (oref["num_max"], oref["denom"], oref["argmax_origin"], oref["argmax_orthant"])
        if got != want:
            raise RuntimeError(f"parity failure: GPU {got} != oracle {want}")
        parity = {"equal": True, "num_max_oracle": oref["num_max"],
                  "checked": "num_max, denom, arg-max origin and orthant against the oracle over all origins"}
    ctx.close()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if shard == "origins" else "weak", "vs_baseline": None,
        "dtype": "u32 ranks (f32 input)" if P.dtype == np.float32 else "u32 ranks (f64 input)",
        "data": "synthetic (seeded numpy PCG64)",
        "config": {"workload": desc, "N": N, "d": d, "units_per_step": units,
                   "kernel_path": (PATH_NAMES[tuned[0]] if tuned else
                                   PATH_NAMES[args.path]),
                   "l2": f"flushed between steps ({args.flush_mb} MB write)",
                   "parallelism": ("origin-sharded x%d (exact max merge)" % world if shard == "origins"
                                   else "replicas x%d" % world)},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "num_max": ref["num_max"], "denom": ref["denom"], "parity": parity,
        "wall_s_timed": wall,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(P, T, d, max_origins=None):
    """The CPU oracle as it stands, all host cores, on the same workload."""
    from oracle import oracle as orc
    N = len(P) + len(T)
    nthr = orc.num_threads()
    o_end = N if max_origins is None else min(N, max_origins)
    t0 = time.perf_counter()
    res = orc.ddks(P, T, origins=(0, o_end), nthreads=nthr)
    dt = time.perf_counter() - t0
    return ({"value": float(o_end) * N * d / dt, "unit": UNIT, "cores": nthr, "kind": "oracle",
             "sample": f"origins [0,{o_end}) of {N} (all points per origin), one pass, {dt:.2f} s"}, res)


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2106_13706_gb300 import workloads as wl
    from oracle import oracle as orc
    key, desc = WORKLOADS[args.workload]
    P, T = wl.CONFIGS[key]()
    NP, d = P.shape
    N = NP + len(T)
    nthr = orc.num_threads()
    # each step: a bounded sample of origins (all points per origin)
    sample = min(N, 2048)
    for w in range(max(args.warmup, 0)):
        orc.ddks(P, T, origins=(0, min(N, 256)), nthreads=nthr)
    tot = 0.0
    for s in range(args.steps):
        a = (s * sample) % N
        b = min(N, a + sample)
        t0 = time.perf_counter()
        orc.ddks(P, T, origins=(a, b), nthreads=nthr)
        tot += time.perf_counter() - t0
    done = sum(min(N, (s * sample) % N + sample) - (s * sample) % N for s in range(args.steps))
    value = float(done) * N * d / tot
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot * 1e3 / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 compares" if P.dtype == np.float32 else "f64 compares",
        "data": "synthetic (seeded numpy PCG64)", "impl": "reference",
        "config": {"workload": desc, "N": N, "d": d},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "kind": "oracle",
                         "sample": f"{sample} origins per step (all points per origin)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def approx_cpu(name, P, T, V, budget_s=8.0):
    """The oracle as it stands (one host core) on a bounded sample of the
    workload: the first n points of each sample, n doubled until the budget."""
    from oracle import oracle as orc
    d = P.shape[1]
    if name == "rdks":
        reps, t0 = 0, time.perf_counter()
        while reps < 3 or time.perf_counter() - t0 < 1.0:
            orc.rdks(P, T)
            reps += 1
        dt = time.perf_counter() - t0
        return {"value": reps / dt, "unit": "tests/s", "cores": 1, "kind": "oracle",
                "sample": f"the full test, {reps} repetitions in {dt:.2f} s"}
    n, best = 25_000, None
    while True:
        Ps, Ts = P[:n], T[:n]
        t0 = time.perf_counter()
        (orc.vdks(Ps, Ts, V) if V else orc.rdks(Ps, Ts))
        dt = time.perf_counter() - t0
        best = (n, dt)
        if dt * 2.2 > budget_s or 2 * n > len(P):
            break
        n *= 2
    n, dt = best
    return {"value": 2 * n / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} points of each sample ({2 * n} pooled, d={d}), one call, {dt:.2f} s"}


def run_approx(args):
    """vdKS / rdKS: one ddks_vdks / ddks_rdks call per step on device-resident
    inputs (graph-replayed), then a few steps with stage timing for the
    roofline of the dominant stage."""
    import torch
    import torch.distributed as dist

    import paper_2106_13706_gb300 as pkg
    from paper_2106_13706_gb300 import build as bld

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    bld.build()
    desc, metric, unit = APPROX[args.workload]
    P, T, V = approx_inputs(args.workload)
    NP, d = P.shape
    NT = T.shape[0]
    N = NP + NT
    units = 1.0 if unit == "tests/s" else float(N)

    def call(c, A, B):
        return c.vdks(A, B, V) if V else c.rdks(A, B)

    Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device="cuda")
    ctx = pkg.Context(device=local)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        ref = call(ctx, Pd, Td)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = ctx.stats()["kernel_launches"]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        r = call(ctx, Pd, Td)
        ev[s][1].record(stream)
        if r["num_max"] != ref["num_max"]:
            raise RuntimeError("result changed between steps")
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = ctx.stats()["kernel_launches"] - l0
    sampler.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = units * args.steps * world / (total_ms * 1e-3)

    # stages (kernel by kernel while stage timing is on)
    ctx.set_stage_timing(True)
    stages = []
    for _ in range(max(5, min(args.steps, 20))):
        flush.zero_()
        call(ctx, Pd, Td)
        stages.append(ctx.stage_times())
    ctx.set_stage_timing(False)
    st = [statistics.mean(x[i] for x in stages) for i in range(3)]
    peaks = measured_peaks()
    if V:
        # dominant: the voxel pass, HBM-bound: reads every coordinate once
        # and updates the 2 x V^d voxel counters
        nbytes = N * d * P.itemsize + 8 * V ** d
        ach = nbytes / (st[1] * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs") or 6800.0
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": load_traffic("vdks_voxel"), "kernel": "voxel pass (k_vdks_thresholds + k_vdks_voxel)",
                "kernel_ms": st[1], "algorithmic_bytes": nbytes,
                "peak_basis": "measured copy bandwidth" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s",
                "range_stage": {"kernel": "k_minmax", "ms": st[0],
                                "achieved_gbs": N * d * P.itemsize / (st[0] * 1e-3) / 1e9},
                "stage_ms": {"range": st[0], "voxel": st[1], "suffix_and_orthants": st[2]}}
    else:
        # rdKS stages: range + corner distances (reads the coordinates, writes
        # one 8-byte key per point and corner), the sort of the d + 1 lists
        # (algorithmic: each key read and written once), the KS walk.  The
        # roofline is taken on the slowest stage, all HBM-bound.
        S = d + 1
        stage_bytes = [N * d * P.itemsize + S * N * 8, S * N * 16, S * N * 16]
        sort_name = ("per-corner warp sort and walk (k_rdks_small)" if N <= 1024 else
                     "sort of the corner distance lists (radix: k_radix_hist/tile_scan/scatter, k_radix_rank_tiles)"
                     if N >= 131072 else "sort of the corner distance lists (k_chunk_sort + k_merge_tile)")
        names = ["range + corner distances (k_minmax + k_rdks_dist_*)", sort_name,
                 "KS walk (k_rdks_walk + k_rdks_final)"]
        k = max(range(3), key=lambda i: st[i])
        ach = stage_bytes[k] / (st[k] * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs") or 6800.0
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None, "kernel": names[k], "kernel_ms": st[k], "algorithmic_bytes": stage_bytes[k],
                "peak_basis": "measured copy bandwidth" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s",
                "stage_ms": {"range_and_distances": st[0], "sort": st[1], "ks_walk": st[2]}}

    e2e = None
    if not args.no_e2e:
        Ph, Th = torch.from_numpy(P).pin_memory(), torch.from_numpy(T).pin_memory()
        for _ in range(3):
            call(ctx, Ph, Th)
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = time.perf_counter()
            r2 = call(ctx, Ph, Th)
            tot += time.perf_counter() - a
        if r2["num_max"] != ref["num_max"]:
            raise RuntimeError("host-input result differs")
        e2e = {"value": units * args.steps * world / tot, "unit": unit,
               "h2d_bytes_per_step": int(P.nbytes + T.nbytes),
               "d2h_bytes_per_step": 3 * 8 + 4 + (0 if V else 8 * (d + 1))}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = approx_cpu(args.workload, P, T, V)
    clocks = sampler.summary()
    ctx.close()
    out = {
        "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 normalisation, u32 voxel counts" if V else "f64 distances, u64 keys",
        "data": "synthetic (seeded numpy PCG64)",
        "config": {"workload": desc, "N": N, "d": d, "voxels_per_dim": V, "units_per_step": units,
                   "l2": f"flushed between steps ({args.flush_mb} MB write)", "replicas": world},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "num_max": ref["num_max"], "denom": ref["denom"],
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_reference_dom2d(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2106_13706_gb300 import workloads as wl
    P, T = wl.gaussian_pair(0, 1_000_000, 1_000_000, 2, shift=0.05)
    N = len(P) + len(T)
    no = 1000  # origins per step, all points per origin
    nthr = orc.num_threads()
    for _ in range(max(args.warmup, 0)):
        orc.ddks(P, T, origins=(0, 100), nthreads=nthr)
    tot = 0.0
    for s_ in range(args.steps):
        a = (s_ * no) % N
        t0 = time.perf_counter()
        orc.ddks(P, T, origins=(a, a + no), nthreads=nthr)
        tot += time.perf_counter() - t0
    value = no * args.steps / tot
    print(json.dumps({
        "metric": "ddks_d2_points_per_s", "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot * 1e3 / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 compares", "data": "synthetic (seeded numpy PCG64)",
        "impl": "reference", "config": {"workload": DOM2D, "N": N, "d": 2},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": nthr, "kind": "oracle",
                         "sample": f"{no} origins per step by the O(N^2) definition, scaled to the whole test"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_reference_approx(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    desc, metric, unit = APPROX[args.workload]
    P, T, V = approx_inputs(args.workload)
    d = P.shape[1]
    from oracle import oracle as orc
    # each step: the oracle on a bounded sample (rdks: the whole 200-point test)
    n = len(P) if args.workload == "rdks" else 50_000
    Ps, Ts = P[:n], T[:n]
    for _ in range(max(args.warmup, 0)):
        (orc.vdks(Ps, Ts, V) if V else orc.rdks(Ps, Ts))
    tot = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        (orc.vdks(Ps, Ts, V) if V else orc.rdks(Ps, Ts))
        tot += time.perf_counter() - t0
    per = 1.0 if unit == "tests/s" else 2.0 * n
    value = per * args.steps / tot
    sample = "the full test per step" if args.workload == "rdks" else f"first {n} points of each sample per step"
    print(json.dumps({
        "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot * 1e3 / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded numpy PCG64)",
        "impl": "reference", "config": {"workload": desc, "N": len(P) + len(T), "d": d, "voxels_per_dim": V},
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


DOM2D = ("exact ddKS d=2 NP=NT=1,000,000 f32, P ~ N(0,I2), T ~ N(0.05*1,I2), range-query path "
         "(O(N log N), no pairwise compares)")


def run_dom2d(args):
    """Exact d = 2 statistic by the range-query path (a separate metric: it
    skips the pairwise compares).  One ddks_distance call per step on
    device-resident inputs."""
    import torch

    import paper_2106_13706_gb300 as pkg
    from paper_2106_13706_gb300 import build as bld
    from paper_2106_13706_gb300 import workloads as wl
    bld.build()
    P, T = wl.gaussian_pair(0, 1_000_000, 1_000_000, 2, shift=0.05)
    N, d = len(P) + len(T), 2
    Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device="cuda")
    ctx = pkg.Context(device=0, path=pkg.PATH_DOMINANCE)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        ref = ctx.distance(Pd, Td)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = ctx.stats()["kernel_launches"]
    torch.cuda.synchronize()
    for s_ in range(args.steps):
        flush.zero_()
        ev[s_][0].record(stream)
        r = ctx.distance(Pd, Td)
        ev[s_][1].record(stream)
        if r["num_max"] != ref["num_max"]:
            raise RuntimeError("result changed between steps")
    torch.cuda.synchronize()
    launches = ctx.stats()["kernel_launches"] - l0
    sampler.stop()
    tot = sum(a.elapsed_time(b) for a, b in ev)
    ctx.set_stage_timing(True)
    stages = []
    for _ in range(5):
        flush.zero_()
        ctx.distance(Pd, Td)
        stages.append(ctx.stage_times())
    ctx.set_stage_timing(False)
    st = [statistics.mean(x[i] for x in stages) for i in range(3)]
    # the range queries: per origin two wavelet-matrix walks (all points, P
    # points) of L levels, two 8-byte record lookups (range ends) per level
    L = max(1, (N - 1).bit_length())
    nbytes = N * 2 * L * 2 * 8
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    ach = nbytes / (st[1] * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
            "kernel": "matrix build + range queries (k_dom_bits/scatter/query)", "kernel_ms": st[1],
            "algorithmic_bytes": nbytes,
            "peak_basis": "measured copy bandwidth" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s",
            "note": "the lookups are random 8-byte reads of L2-resident bit vectors; HBM is the reference only",
            "stage_ms": {"encode": st[0], "count": st[1], "reduce": st[2]}}
    e2e = None
    if not args.no_e2e:
        Ph, Th = torch.from_numpy(P).pin_memory(), torch.from_numpy(T).pin_memory()
        for _ in range(3):
            ctx.distance(Ph, Th)
        t_e = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = time.perf_counter()
            r2 = ctx.distance(Ph, Th)
            t_e += time.perf_counter() - a
        assert r2["num_max"] == ref["num_max"]
        e2e = {"value": N * args.steps / t_e, "unit": "points/s", "h2d_bytes_per_step": int(P.nbytes + T.nbytes),
               "d2h_bytes_per_step": 3 * 8 + 4}
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as orc
        no = 2000
        t0 = time.perf_counter()
        orc.ddks(P, T, origins=(0, no), nthreads=orc.num_threads())
        dt = time.perf_counter() - t0
        cpu = {"value": no / dt, "unit": "points/s", "cores": orc.num_threads(), "kind": "oracle",
               "sample": f"origins [0,{no}) of {N} by the O(N^2) definition ({dt:.2f} s), scaled to the whole "
                         "test: N / (time x N / origins)"}
    clocks = sampler.summary()
    ctx.close()
    ms = tot / args.steps
    print(json.dumps({
        "metric": "ddks_d2_points_per_s", "value": N / (ms * 1e-3), "unit": "points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 ranks (f32 input)", "data": "synthetic (seeded numpy PCG64)",
        "config": {"workload": DOM2D, "N": N, "d": d, "l2": f"flushed between steps ({args.flush_mb} MB write)",
                   "equivalent_compares_per_s": float(N) * N * d / (ms * 1e-3)},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "num_max": ref["num_max"], "denom": ref["denom"]}))


def run_perm(args):
    """Permutation test of the 3-component mixture (2 x 2,000 points, d = 3)
    with B relabellings in one batched launch per step."""
    import torch

    import paper_2106_13706_gb300 as pkg
    from paper_2106_13706_gb300 import build as bld
    from paper_2106_13706_gb300 import workloads as wl
    bld.build()
    P, T = wl.CONFIGS["cfg4_d3_2000x2000_mixture_null"]()
    N, d = len(P) + len(T), P.shape[1]
    B = args.perms
    Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device="cuda")
    ctx = pkg.Context(device=0)
    for _ in range(max(args.warmup, 3)):
        ref = ctx.permutation_test(Pd, Td, B, 2021)
    ms = []
    stream = torch.cuda.current_stream()
    l0 = ctx.stats()["kernel_launches"]
    for s in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = ctx.permutation_test(Pd, Td, B, 2022 + s)  # a new seed (new relabellings) every step
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        assert r["observed"]["num_max"] == ref["observed"]["num_max"]
    launches = ctx.stats()["kernel_launches"] - l0
    tot = sum(ms)
    cpu = None
    parity = None
    if not args.no_cpu_baseline:
        from oracle import oracle as orc
        nb = 4
        t0 = time.perf_counter()
        oref = orc.permutation_test(P, T, nb, 2021, nthreads=orc.num_threads())
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / (dt * (B + 1) / (nb + 1)), "unit": "tests/s", "cores": orc.num_threads(),
               "kind": "oracle", "sample": f"{nb} relabellings + observed ({dt:.2f} s), scaled to B={B}"}
        # relabelling b depends on (seed, b) only: the first nb of the warm-up
        # call (seed 2021) must equal the oracle's
        got = [int(x) for x in ref["perm_num_max"][:nb]]
        want = [int(x) for x in oref["perm_num_max"][:nb]]
        if got != want or ref["observed"]["num_max"] != oref["num_obs"]:
            raise RuntimeError(f"parity failure: GPU {got} != oracle {want}")
        parity = {"equal": True, "num_max_oracle": int(oref["num_obs"]),
                  "checked": f"observed num_max and the first {nb} relabellings' num_max against the oracle"}
    study = significance_study(ctx, torch, wl, quick=args.steps < 5) if not args.no_study else None
    ctx.close()
    print(json.dumps({
        "metric": "ddks_perm_tests_per_s", "value": args.steps / (tot * 1e-3), "unit": "tests/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 ranks (f32 input)",
        "data": "synthetic (seeded numpy PCG64)",
        "config": {"workload": f"permutation test, 3-component Gaussian mixture d=3 NP=NT=2000, B={B}",
                   "logical_compares_per_s": (B + 1) * float(N) * N * d * args.steps / (tot * 1e-3)},
        "cpu_baseline": cpu, "gpu_launches": launches, "p_value": ref["p_value"], "parity": parity,
        "significance_vs_permutation": study}))


def significance_study(ctx, torch, wl, quick=False, alpha=0.05, B=1000):
    """Analytic significance S (Sec. 3, Eq. ddks_significance; binomial and
    Poisson cells, Bayes rate) beside the permutation p-value of the same
    samples, under the null and an alternative, over many seeds: the
    comparison of Sec. 3 (its type I / power statement uses DVU, d = 3,
    50 points per sample).  Everything runs on the GPU."""
    def one(P, T, seed):
        Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
        pr = ctx.permutation_test(Pd, Td, B, 7000 + seed, want_perm=False)
        num = pr["observed"]["num_max"]
        S_bin, _ = ctx.significance(Pd, Td, num, 1, 0)
        S_poi, _ = ctx.significance(Pd, Td, num, 1, 1)
        return S_bin, S_poi, pr["p_value"]

    cases = {
        "dvu_d3_50x50": (lambda s: wl.dvu_null_pair(s, 50, 50, 3), lambda s: wl.dvu_pair(s, 50, 50, 3),
                         40 if quick else 200),
        "mixture_d3_2000x2000": (lambda s: wl.mixture_pair(seed=s, shift=0.0),
                                 lambda s: wl.mixture_pair(seed=s, shift=0.2), 5 if quick else 20),
    }
    out = {"alpha": alpha, "B": B}
    for name, (null_fn, alt_fn, seeds) in cases.items():
        row = {"seeds": seeds}
        for hyp, fn in (("null", null_fn), ("alt", alt_fn)):
            r = np.array([one(*fn(s), s) for s in range(seeds)])
            Sb, Sp, pp = r[:, 0], r[:, 1], r[:, 2]
            row[hyp] = {
                "reject_rate_S_binomial": float((Sb < alpha).mean()),
                "reject_rate_S_poisson": float((Sp < alpha).mean()),
                "reject_rate_p_perm": float((pp < alpha).mean()),
                "median_S_binomial": float(np.median(Sb)), "median_p_perm": float(np.median(pp)),
                "same_decision": float(((Sb < alpha) == (pp < alpha)).mean()),
            }
        out[name] = row
    return out


def oracle_problems(problems, results, picks, budget_s=20.0):
    """The CPU oracle (all host cores) on chosen problems of a batch or a
    request stream, within a time budget: whole problems per second and a
    parity check of each checked problem's num_max against the GPU result."""
    from oracle import oracle as orc
    nthr = orc.num_threads()
    done, mism, t_used = 0, 0, 0.0
    for i in picks:
        P, T = problems[i]
        t0 = time.perf_counter()
        ref = orc.ddks(P, T, nthreads=nthr)
        t_used += time.perf_counter() - t0
        done += 1
        mism += int(ref["num_max"] != results[i])
        if t_used > budget_s:
            break
    return done, mism, t_used, nthr


def run_batch(args):
    """256 uneven problems (NP, NT log-uniform in [64, 8192], d in 2..8): one
    batched persistent launch per step vs one ddks_distance call per problem."""
    import torch

    import paper_2106_13706_gb300 as pkg
    from paper_2106_13706_gb300 import build as bld
    from paper_2106_13706_gb300 import workloads as wl
    bld.build()
    probs = wl.uneven_problems(seed=0, count=256)
    dev = [(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs]
    units = sum(float(len(P) + len(T)) ** 2 * P.shape[1] for P, T in probs)
    ctx = pkg.Context(device=0)
    shapes = None
    if not args.no_autotune:
        tuned = ctx.autotune_batch(dev)  # the project's autotuner picks each dimension's tile shape
        shapes = {str(d): list(tuned[d]) for d in sorted({P.shape[1] for P, _ in probs})}
    for _ in range(max(args.warmup, 3)):
        ref = ctx.batch_distance(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        got = ctx.batch_distance(dev)
    tb = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 4)):
        one = [ctx.distance(P, T) for P, T in dev]
    t1 = (time.perf_counter() - t0) / max(1, args.steps // 4)
    assert [g["num_max"] for g in got] == [o["num_max"] for o in one] == [r["num_max"] for r in ref]
    ctx.close()
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on a seeded sample of the batch's problems, with parity
        order = list(np.random.default_rng(1).permutation(len(probs)))
        done, mism, t_used, nthr = oracle_problems(probs, [g["num_max"] for g in got], order, budget_s=15.0)
        if mism:
            raise SystemExit(f"batch parity: {mism} of {done} sampled problems differ from the oracle")
        cpu = {"value": done / t_used, "unit": "tests/s", "cores": nthr, "kind": "oracle",
               "sample": f"{done} of the 256 problems in seeded random order (15 s budget), "
                         f"num_max equal to the GPU batch for all {done}"}
    print(json.dumps({
        "metric": "ddks_batch_tests_per_s", "value": 256 / tb, "unit": "tests/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tb * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 ranks (f32 input)",
        "data": "synthetic (seeded numpy PCG64)",
        "config": {"workload": "256 problems, NP,NT log-uniform [64,8192], d uniform 2..8, mixtures",
                   "one_call_per_problem_tests_per_s": 256 / t1, "compares_per_s": units / tb,
                   "tile_shapes": shapes},
        "cpu_baseline": cpu}))


def run_serve(args):
    """Poisson arrivals (200/s) of requests with NP, NT log-uniform in [100, 50000]
    and d in {2,3,4,6,8}: submit/poll latency percentiles and throughput, against
    the same stream served one request per call."""
    import threading

    import torch

    import paper_2106_13706_gb300 as pkg
    from paper_2106_13706_gb300 import build as bld
    from paper_2106_13706_gb300 import workloads as wl
    bld.build()
    reqs = wl.serving_requests(seed=0, count=args.requests)

    def replay(serve_fn, saturated=False):
        lat = [None] * len(reqs)
        t_start = time.perf_counter()
        threads = []
        for i, (arr, P, T) in enumerate(reqs):
            dt = arr - (time.perf_counter() - t_start)
            if dt > 0 and not saturated:
                time.sleep(dt)
            threads.append(serve_fn(i, P, T, lat))
        for th in threads:
            if th is not None:
                th.join()
        return lat, time.perf_counter() - t_start

    ctx = pkg.Context(device=0, max_batch=64)
    nums = [None] * len(reqs)  # num_max of each request as served
    import queue
    # a pool of client threads started beforehand waits for the tickets (a
    # thread started per request would put its start-up into the latency)
    tq = queue.Queue()

    errors = []

    def poller():
        while True:
            item = tq.get()
            if item is None:
                return
            try:
                i, tk, t0, lat = item
                while True:
                    rc, r = ctx.poll(tk, 200000)
                    if rc != pkg.DDKS_PENDING:
                        if rc == pkg.DDKS_OK:
                            lat[i] = time.perf_counter() - t0
                            nums[i] = r["num_max"]
                        break
            except Exception as ex:  # a failed request fails the run, it must not hang it
                errors.append(repr(ex))
            finally:
                tq.task_done()

    def drain_tickets(limit_s=300.0):
        end = time.perf_counter() + limit_s
        while tq.unfinished_tasks and not errors:
            if time.perf_counter() > end:
                raise RuntimeError("served requests still pending after %.0f s" % limit_s)
            time.sleep(0.0005)
        if errors:
            raise RuntimeError("served request failed: " + errors[0])

    pollers = [threading.Thread(target=poller, daemon=True) for _ in range(8)]
    for th in pollers:
        th.start()

    def submit_fn(i, P, T, lat):
        t0 = time.perf_counter()
        tq.put((i, ctx.submit(P, T), t0, lat))
        return None

    lat_b, wall_b = replay(submit_fn)
    drain_tickets()
    wall_b = max(wall_b, max(a + l for (a, _, _), l in zip(reqs, lat_b)))
    st = ctx.stats()
    # saturated: every request submitted at once, throughput of the batching loop
    t_sat = time.perf_counter()
    replay(submit_fn, saturated=True)
    drain_tickets()
    wall_bs = time.perf_counter() - t_sat
    for _ in pollers:
        tq.put(None)
    for th in pollers:
        th.join()
    ctx.close()
    # one request per call, FIFO on one worker thread
    ctx1 = pkg.Context(device=0)
    qq = queue.Queue()

    def worker():
        while True:
            item = qq.get()
            if item is None:
                return
            if isinstance(item, threading.Event):  # everything queued before it is done
                item.set()
                continue
            i, P, T, t0, lat = item
            ctx1.distance(P, T)
            lat[i] = time.perf_counter() - t0

    wth = threading.Thread(target=worker, daemon=True)
    wth.start()

    def single_fn(i, P, T, lat):
        qq.put((i, P, T, time.perf_counter(), lat))
        return None

    def drain():
        ev = threading.Event()
        qq.put(ev)
        ev.wait()

    try:
        lat_s, _ = replay(single_fn)
        drain()
        wall_s = max(a + l for (a, _, _), l in zip(reqs, lat_s))
        lat_ss, _ = replay(single_fn, saturated=True)
        drain()
        wall_ss = max(lat_ss)
    finally:
        qq.put(None)
        wth.join()
    ctx1.close()
    cpu = None
    if not args.no_cpu_baseline:
        # parity with the oracle: every request with N <= 5,000, then a seeded
        # 5% sample of the larger ones, within a 30 s budget
        sizes = [len(P) + len(T) for _, P, T in reqs]
        small = [i for i, n in enumerate(sizes) if n <= 5000]
        large = [i for i, n in enumerate(sizes) if n > 5000]
        rng = np.random.default_rng(5)
        pick_large = list(rng.choice(large, size=max(1, len(large) // 20), replace=False)) if large else []
        done, mism, t_used, nthr = oracle_problems([(P, T) for _, P, T in reqs], nums, small + pick_large,
                                                   budget_s=30.0)
        if mism:
            raise SystemExit(f"serving parity: {mism} of {done} checked requests differ from the oracle")
        n_small = min(done, len(small))
        cpu = {"value": done / t_used, "unit": "tests/s", "cores": nthr, "kind": "oracle",
               "sample": f"{n_small} of {len(small)} requests with N <= 5,000 and {done - n_small} of a seeded "
                         f"5% sample of the {len(large)} larger ones (30 s budget); num_max equal to the "
                         f"served result for all {done}"}
    pct = lambda xs, q: float(np.percentile(np.array(xs) * 1e3, q))
    print(json.dumps({
        "metric": "ddks_serve_tests_per_s", "value": len(reqs) / wall_b, "unit": "tests/s", "n_gpus": 1,
        "steps": len(reqs), "warmup": 0, "ms_per_step": wall_b * 1e3 / len(reqs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 ranks (f32 input)",
        "data": "synthetic (seeded numpy PCG64)",
        "config": {"workload": f"{len(reqs)} Poisson(200/s) requests, NP,NT log-uniform [100,50000], d in {{2,3,4,6,8}}",
                   "p50_ms": pct(lat_b, 50), "p99_ms": pct(lat_b, 99), "batches": st["batches"],
                   "one_per_call": {"tests_per_s": len(reqs) / wall_s, "p50_ms": pct(lat_s, 50),
                                    "p99_ms": pct(lat_s, 99)},
                   "saturated": {"tests_per_s": len(reqs) / wall_bs,
                                 "one_per_call_tests_per_s": len(reqs) / wall_ss,
                                 "note": "all requests submitted at once"},
                   "bytes_resident_peak": st["bytes_resident_peak"]},
        "cpu_baseline": cpu}))


def main():
    args = parse()
    if args.impl == "reference":
        if args.workload in APPROX:
            run_reference_approx(args)
        elif args.workload == "dom2d":
            run_reference_dom2d(args)
        else:
            run_reference(args)
    elif args.workload in APPROX:
        run_approx(args)
    elif args.workload == "dom2d":
        run_dom2d(args)
    elif args.workload == "perm":
        run_perm(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
