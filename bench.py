#!/usr/bin/env python
"""Throughput benchmark of the FD-LBM (five-point) and MRT D2Q9 steps.

Workload: 8192 x 8192 periodic lattice, 32 seeded transverse modes of
amplitude 1e-3 (random wave vectors and phases), nu = 0.01, s_e = 1.5,
FP32 storage and arithmetic.  One bench step = one FD-LBM five-point time
step of the whole lattice; the MRT step of the same lattice is timed beside
it with the same step count.  The state (805 MB for FD-LBM, 2.4 GB for MRT)
is larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded band of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FD-LBM D2Q9 MLUPS & %HBM peak vs MRT-LBM; served solves/s, p99 latency"
N_SIDE = 8192
N_MODES = 32
AMP = 1e-3
NU = 0.01
S_E = 1.5
BYTES_PER_LUP = {"fd5": 24, "mrt": 72, "lwacm": 24}  # read + write of the state per node update (FP32)
WORKLOAD = (f"FD-LBM five-point and MRT D2Q9 (and LW-ACM) side by side, {N_SIDE}x{N_SIDE} periodic, "
            f"{N_MODES} seeded transverse modes A={AMP}, nu={NU}, s_e={S_E}, FP32")
FALLBACK_HBM_GBS = 6800.0
# GB300's HBM3e data rate as specified (8 stacks at 3996 MHz); ncu's DRAM
# throughput percentages are of this figure (the MRT step's 6.81 TB/s reads
# as 85.9 % of peak).  The measured copy bandwidth above is the roofline's
# denominator; this one is reported beside it.
SPEC_HBM_GBS = 7900.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--side", type=int, default=N_SIDE, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the cost model's row segments for the streaming steps")
    ap.add_argument("--workload", choices=["throughput", "batched", "serving"],
                    default="throughput",
                    help="throughput: the 8192^2 headline line (default); batched: 4096 "
                         "lattices of sides 32..512; serving: the request stream")
    ap.add_argument("--lattices", type=int, default=4096, help=argparse.SUPPRESS)
    ap.add_argument("--batched-lattices", type=int, default=4096,
                    help="lattices of the batched workload in the default line (all 4096 of it)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=300,
                    help="requests of the serving sample in the default line")
    ap.add_argument("--no-serving", action="store_true")
    return ap.parse_args()


# ---- distributed plumbing (one process per GPU, independent lattices) -------------------

def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def all_max(value, world, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def all_sum(value, world, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_mlups(nodes, ms_per_step, world, device=None):
    """Whole-job throughput of independent replicas: the node updates of all
    ranks in one step over the slowest rank's step time.  Returns (MLUPS,
    max ms per step)."""
    ms = all_max(ms_per_step, world, device)
    return all_sum(nodes, world, device) / (ms / 1e3) / 1e6, ms


# ---- peaks, traffic, clocks ----------------------------------------------------------------

def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The translation unit of each profiled kernel; its hash covers the code (not
# the comments) of the unit and of every header it includes (transitively), so
# a recorded DRAM figure is used only while that kernel's code is unchanged.
KERNEL_UNITS = {"fd_step": "fd_step_stream.cu", "mrt_step": "mrt_step.cu",
                "lwacm_step": "fd_step_stream.cu"}


def kernel_source_hash(kernel: str) -> str:
    import re
    csrc = os.path.join(ROOT, "paper_1803_00437_gb300", "csrc")
    inc = os.path.join(ROOT, "include")
    seen, todo = [], [KERNEL_UNITS[kernel]]
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        seen.append(name)
        for d in (csrc, inc):
            path = os.path.join(d, name)
            if os.path.exists(path):
                with open(path) as fh:
                    todo += re.findall(r'#include "([^"]+)"', fh.read())
                break
    h = hashlib.sha256()
    for name in sorted(seen):
        for d in (csrc, inc):
            path = os.path.join(d, name)
            if os.path.exists(path):
                with open(path) as fh:
                    code = _strip_comments(fh.read())
                h.update(name.encode() + b"\0" + code.encode())
                break
    return h.hexdigest()[:16]


def _strip_comments(src: str) -> str:
    """C/C++ source without comments and with whitespace collapsed, so that
    only code changes alter a kernel's hash."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def recorded_traffic(kernel: str, nodes: int):
    """DRAM bytes per launch from the committed ncu summary, scaled to `nodes`
    node updates, or None if the kernel changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        with open(path) as fh:
            rec = json.loads("".join(ln for ln in fh if not ln.startswith("#")))
    except Exception:
        return None
    k = rec.get("kernels", {}).get(kernel)
    if not k or k.get("source_hash") != kernel_source_hash(kernel):
        return None
    return k["dram_bytes_per_launch"] * nodes / k["nodes_per_launch"]


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            ident = str(self.dev)
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            if vis:
                ident = vis.split(",")[self.dev].strip()
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", ident, f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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
        self.out.close()
        rows = []
        with open(self.path) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---- CPU oracle timing -------------------------------------------------------------------------

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_band(rows, side, seed):
    import numpy as np
    from paper_1803_00437_gb300 import inputs
    modes = inputs.random_modes(side, rows, N_MODES, AMP, seed=seed)
    d, ux, uy = inputs.transverse_modes(side, rows, modes)
    return 1.0 + d, ux, uy


def quartic_s_q(s_xx: float) -> float:
    """MRT's s_q for the oracle: Eq. sigsig, (1/s_xx - 1/2)(1/s_q - 1/2) = 1/6,
    the rate the library applies when s_q is left to it."""
    return 1.0 / (1.0 / (6.0 * (1.0 / s_xx - 0.5)) + 0.5)


def time_oracle(scheme: str, side: int, target_s: float, max_rows: int | None = None):
    """Run the FP64 oracle on side x rows periodic bands of the workload until
    about target_s seconds of CPU work; returns (MLUPS, rows, steps, cores)."""
    from oracle import ref
    from paper_1803_00437_gb300 import fdlbm as F
    cores = host_cores()
    ref.set_threads(cores)
    s_xx = F.nu_to_s(NU)
    code = ref.FD5 if scheme == "fd5" else ref.MRT
    # calibrate on a thin band
    rows = 16
    p = ref.params(side, rows, code, s_xx, S_E, quartic_s_q(s_xx), 1.5)
    r, x, y = oracle_band(rows, side, 1017)
    t0 = time.perf_counter()
    if code == ref.MRT:
        ref.mrt_step(p, ref.mrt_init(p, r, x, y), 1)
    else:
        ref.fd_run(p, r, x, y, 1)
    rate = side * rows / max(time.perf_counter() - t0, 1e-6)
    rows = int(min(max(16, rate * min(target_s, 5.0) / side), max_rows or 4096))
    p = ref.params(side, rows, code, s_xx, S_E, quartic_s_q(s_xx), 1.5)
    r, x, y = oracle_band(rows, side, 1017)
    f = ref.mrt_init(p, r, x, y) if code == ref.MRT else None
    steps, elapsed = 0, 0.0
    while elapsed < target_s and steps < 1000:
        t0 = time.perf_counter()
        if code == ref.MRT:
            f = ref.mrt_step(p, f, 1)
        else:
            r, x, y = ref.fd_run(p, r, x, y, 1)
        elapsed += time.perf_counter() - t0
        steps += 1
    return side * rows * steps / elapsed / 1e6, rows, steps, cores


# ---- our implementation ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, "nccl")
    from paper_1803_00437_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    barrier(world)
    from paper_1803_00437_gb300 import fdlbm as F
    from paper_1803_00437_gb300 import inputs

    side = args.side
    nodes = side * side
    s_xx = F.nu_to_s(NU)
    stream = torch.cuda.Stream(dev)
    modes = inputs.random_modes(side, side, N_MODES, AMP, seed=inputs.seed_for(1) + rank)
    lats = {}
    for scheme in ("fd5", "mrt", "lwacm"):
        cfg = F.LatticeConfig(side, side, scheme, s_xx=s_xx, s_e=S_E)
        lat = F.Lattice(cfg, device=dev, stream=stream)
        lat.init_modes(modes)
        lats[scheme] = lat
    # set-up, untimed: the streaming steps' row segments are chosen by timing
    # the library's candidate plans on this device (the state is restored)
    plans = {}
    if not args.no_tune:
        for scheme in ("fd5", "lwacm"):
            tuned = lats[scheme].tune()
            if tuned is not None:
                plans[scheme] = lats[scheme].stream_plan()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    results = {}
    sampler.start()
    for scheme, lat in lats.items():
        lat.step(args.warmup)
        torch.cuda.synchronize(dev)
        barrier(world)
        torch.cuda.synchronize(dev)
        launches0 = lat.launches
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ms = ev0.elapsed_time(ev1)
        results[scheme] = {"ms": ms, "launches": lat.launches - launches0}
    clocks = sampler.stop()

    # health of the run: finite, mass conserved (FP64 reductions on the device)
    health = {}
    for scheme, lat in lats.items():
        mx = lat.reduce("maxabs")
        health[scheme] = {"max_u": float(mx[0]), "mass": float(lat.reduce("mass")[0])}

    # end to end through the C ABI with host buffers: H2D of the inputs from pinned
    # host memory, one step, D2H of an FP64 reduction, every step
    e2e = None
    if not args.no_e2e:
        lat = lats["fd5"]
        fields = lat.moments()
        lat.sync()
        host = [t.cpu().pin_memory() for t in fields]
        torch.cuda.synchronize(dev)
        e2e_steps = max(1, min(args.steps, 20))
        lib = lat.lib
        import ctypes
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in host]
        out = np.zeros(4)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            lat._check(lib.fdlbm_init_host(lat._h, *ptrs), "init_host")
            lat._check(lib.fdlbm_step(lat._h, 1), "step")
            lat._check(lib.fdlbm_reduce(lat._h, 0, None, ctypes.c_void_p(out.ctypes.data)),
                       "reduce")
        dt = time.perf_counter() - t0
        dt_max = all_max(dt, world, dev)
        e2e = {"value": round(all_sum(nodes * e2e_steps, world, dev) / dt_max / 1e6, 2),
               "unit": "MLUPS", "h2d_bytes_per_step": 3 * 4 * nodes,
               "d2h_bytes_per_step": 4 * 8, "steps": e2e_steps}

    # batched lattices beside the headline lattice (a sample of the batched
    # workload, timed the same way), one per rank
    batched = None
    if not args.no_batched:
        batched = measure_batched(args.batched_lattices, min(args.steps, 50), max(args.warmup, 3),
                                  local)
        batched["value"] = round(all_sum(batched["value"], world, dev), 1)

    # served requests beside them: the first requests of the specified stream
    # (Poisson arrivals at 200/s, an overload), their latencies and solves/s
    serving = None
    if not args.no_serving:
        from paper_1803_00437_gb300 import serve
        torch.cuda.empty_cache()
        serving = serve.measure_stream(args.serving_requests, device=dev)
        torch.cuda.empty_cache()

    peak, peak_kind = hbm_peak()

    def roofline(scheme, kernel):
        per_launch_s = results[scheme]["ms"] / 1e3 / args.steps
        achieved = BYTES_PER_LUP[scheme] * nodes / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "peak_spec": SPEC_HBM_GBS, "frac_spec": round(achieved / SPEC_HBM_GBS, 4),
                "traffic": recorded_traffic(kernel, nodes),
                "algorithmic_bytes_per_launch": BYTES_PER_LUP[scheme] * nodes,
                "kernel": kernel}

    value, fd_ms = job_mlups(nodes, results["fd5"]["ms"] / args.steps, world, dev)
    mrt_value, mrt_ms = job_mlups(nodes, results["mrt"]["ms"] / args.steps, world, dev)
    lw_value, lw_ms = job_mlups(nodes, results["lwacm"]["ms"] / args.steps, world, dev)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(fd_ms, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": side, "ny": side, "scheme": "fd5",
                   "l2": "state larger than L2 (805 MB FD-LBM and LW-ACM, 2.4 GB MRT): no flush",
                   "parallelism": f"{world} independent lattice(s), one per GPU",
                   "stream_plans": {k: {q: v[q] for q in ("seg_rows", "nsegs", "tail_rows",
                                                          "ntail", "ctas")}
                                    for k, v in plans.items()},
                   "plan_choice": "tuned: fastest of the library's candidate plans"
                                  if plans else "the library's cost model"},
        "roofline": roofline("fd5", "fd_step"),
        "mrt": {"value": round(mrt_value, 1), "unit": "MLUPS",
                "ms_per_step": round(mrt_ms, 5), "roofline": roofline("mrt", "mrt_step")},
        "fd_over_mrt_speedup": round(mrt_ms / fd_ms, 3),
        "lwacm": {"value": round(lw_value, 1), "unit": "MLUPS",
                  "ms_per_step": round(lw_ms, 5), "roofline": roofline("lwacm", "lwacm_step")},
        "gpu_launches": int(sum(r["launches"] for r in results.values())
                            + (batched["gpu_launches"] if batched else 0)
                            + (serving["gpu_launches"] if serving else 0)),
        "clocks": clocks, "health": health, "e2e": e2e,
    }
    if serving:
        serving["workload"] = (f"the first {args.serving_requests} requests of the serving stream "
                               "(Poisson 200/s, sides log-U[64,4096], steps log-U[100,20000], "
                               "shear wave / 1-4 modes / Poiseuille, nu U[0.002,0.1]), FD-LBM "
                               "five-point FP32, 80 GB HBM budget, continuous batching")
        serving["unit"] = "solves/s"
        serving["value"] = serving["solves_per_s"]
        line["serving"] = serving
    if batched:
        batched["workload"] = (f"{batched['lattices']} periodic lattices of the batched workload "
                               "(sides U{32..512}, nu U[0.002,0.1], one transverse mode A=1e-3 "
                               "each), FD-LBM five-point FP32, graph-captured runs")
        line["batched"] = batched
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups, rows, steps, cores = time_oracle("fd5", side, 15.0)
        line["cpu_baseline"] = {
            "value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, FD-LBM five-point, {steps} step(s) of a {side}x{rows} "
                      f"periodic band of the same {N_MODES}-mode workload"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    from oracle import ref
    ref.build()
    side = args.side
    # size each step so that warmup + steps take about two minutes
    budget = 120.0
    mlups0, _, _, cores = time_oracle("fd5", side, 1.0, max_rows=64)
    rows = int(max(8, min(2048, mlups0 * 1e6 * budget / max(args.steps + args.warmup, 1) / side)))
    from paper_1803_00437_gb300 import fdlbm as F
    p = ref.params(side, rows, ref.FD5, F.nu_to_s(NU), S_E)
    r, x, y = oracle_band(rows, side, 1017)
    for _ in range(args.warmup):
        r, x, y = ref.fd_run(p, r, x, y, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, x, y = ref.fd_run(p, r, x, y, 1)
    dt = time.perf_counter() - t0
    value = side * rows * args.steps / dt / 1e6
    sample = (f"FP64 oracle, FD-LBM five-point, each step a {side}x{rows} periodic band of the "
              f"{N_MODES}-mode workload")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": side, "ny": side, "scheme": "fd5",
                       "sample_rows": rows},
            "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def batch_arena_bytes(sides, strip=120, ghost=8, align=32):
    """Arena bytes for square lattices of the given sides (two FP32 copies of
    3 planes; rows padded as the batch layout pads them)."""
    total = 0
    for L in sides:
        pitch = max(L + 2 * ghost, -(-L // strip) * strip + 2 * ghost)
        pitch = -(-pitch // align) * align
        total += 2 * 3 * L * pitch * 4
    return total


def measure_batched(n_lattices: int, steps: int, warmup: int, dev_index: int = 0):
    """The batched workload: n periodic lattices, sides ~ U{32..512}, nu ~
    U[0.002, 0.1], each one seeded transverse mode of amplitude 1e-3, FD-LBM
    five-point FP32, advanced together by the batched kernel in
    graph-captured runs (rows per item chosen by the autotuner).  Returns a
    dict: useful MLUPS, ms per step, roofline against 24 B per useful node,
    launches and clocks of the timed region."""
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    from paper_1803_00437_gb300 import inputs
    lats = inputs.batch_lattices(n_lattices, inputs.seed_for(2))
    sides = [L for L, _, _ in lats]
    nodes = sum(L * L for L in sides)
    arena = int(batch_arena_bytes(sides) * 1.02) + (1 << 20)
    dev = torch.device("cuda", dev_index)
    b = F.Batch("fd5", max_lattices=len(lats), arena_bytes=arena, max_side=512, device=dev)
    slots = [b.add(F.LatticeConfig(L, L, "fd5", s_xx=F.nu_to_s(nu), s_e=S_E)) for L, nu, _ in lats]
    seg = b.tune(steps=4)
    for s, (L, nu, md) in zip(slots, lats):
        b.init_modes(s, [md])
    b.step(warmup)
    b.sync()
    launches0 = b.launches
    sampler = ClockSampler(dev_index)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    b.sync()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    peak, peak_kind = hbm_peak()
    gbs = 24 * nodes * steps / (ms / 1e3) / 1e9
    maxu = max(float(b.reduce(s, "maxabs")[0]) for s in slots[:64])
    out = {"value": round(nodes * steps / ms / 1e3, 1), "unit": "MLUPS", "steps": steps,
           "warmup": warmup, "ms_per_step": round(ms / steps, 4), "lattices": len(lats),
           "total_nodes": nodes, "rows_per_item": seg,
           "narrow_last_strips": bool(b.tuned[1]),
           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(gbs / peak, 4), "peak_kind": peak_kind,
                        "peak_spec": SPEC_HBM_GBS, "frac_spec": round(gbs / SPEC_HBM_GBS, 4),
                        "traffic": None},
           "gpu_launches": int(b.launches - launches0), "clocks": clocks,
           "health": {"max_u_first_64": maxu}}
    b.close()
    del b
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    """bench.py --workload batched: 4096 lattices (the batched workload)."""
    import torch
    from paper_1803_00437_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    r = measure_batched(args.lattices, args.steps, args.warmup)
    line = {
        "metric": METRIC, "workload": "batched", "value": r["value"], "unit": "MLUPS",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{r['lattices']} periodic lattices, sides U{{32..512}}, nu "
                               "U[0.002,0.1], one transverse mode A=1e-3 each, FD-LBM five-point "
                               "FP32", "lattices": r["lattices"], "total_nodes": r["total_nodes"],
                   "rows_per_item": r["rows_per_item"],
                   "narrow_last_strips": r["narrow_last_strips"],
                   "l2": "state larger than L2: no flush"},
        "roofline": r["roofline"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
        "health": r["health"],
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        from paper_1803_00437_gb300 import serve
        serve.bench_main(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
