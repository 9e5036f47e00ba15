"""Serving FD-LBM simulations with continuous batching.

Requests (a lattice, a number of steps, an initial field) arrive over time.
The server keeps every admitted request's state resident in one batch arena
on the device (fdlbm_batch_* in the C ABI), admits waiting requests in
arrival order as soon as a slot and arena space are free (the arena size is
the HBM budget), and advances all admitted requests together: each run of
up to `run_steps` steps is one replay of a captured CUDA graph in which every
slot takes only the steps it still needs.  Finished requests are reduced on
the device (FP64 mass, momentum, energy, max |u| and the first mode's
amplitude), released, and their latency (finish - arrival) recorded.

The batch path computes exactly what a single lattice computes (the tests
check each result alone and in the mix), so a request's answer does not
depend on what it was batched with.
"""
from __future__ import annotations

import collections
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import fdlbm as F
from . import inputs

KINDS = ("shear", "modes", "poiseuille")


@dataclass
class Request:
    rid: int
    kind: str
    nx: int
    ny: int
    steps: int
    nu: float
    arrival: float                       # seconds after the stream starts
    modes: list = field(default_factory=list)
    force: tuple = (0.0, 0.0)
    # filled by the server
    admitted: float | None = None
    finished: float | None = None
    result: dict | None = None

    def config(self, scheme: str) -> F.LatticeConfig:
        walls = self.kind == "poiseuille"
        return F.LatticeConfig(self.nx, self.ny, scheme, s_xx=F.nu_to_s(self.nu), s_e=1.5,
                               boundary="walls_y" if walls else "periodic", wall_xi=0.5,
                               force=self.force)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    @property
    def work(self) -> int:
        return self.nodes * self.steps


def make_requests(n: int, rate: float, seed: int, side_range=(64, 4096),
                  step_range=(100, 20000), nu_range=(0.002, 0.1)):
    """Poisson arrivals (mean rate per second), sides and steps log-uniform,
    kinds uniform among a shear wave, 1-4 transverse modes and a Poiseuille
    channel (side x side/4, walls in y, force for u_max = 0.05)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        L = int(round(math.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1])))))
        steps = int(round(math.exp(rng.uniform(math.log(step_range[0]),
                                               math.log(step_range[1])))))
        nu = float(rng.uniform(*nu_range))
        kind = KINDS[int(rng.integers(0, 3))]
        if kind == "poiseuille":
            ny = max(16, L // 4)
            H = ny
            force = (8.0 * nu * 0.05 / (H * H), 0.0)
            out.append(Request(rid, kind, L, ny, steps, nu, t, [], force))
            continue
        nmodes = 1 if kind == "shear" else int(rng.integers(1, 5))
        modes = inputs.random_modes(L, L, nmodes, 1e-3, seed=int(rng.integers(0, 2 ** 31)))
        out.append(Request(rid, kind, L, L, steps, nu, t, modes))
    return out


class Server:
    """Continuous-batching server on one GPU.

    hbm_budget: device bytes reserved for the admitted requests' states (the
    batch arena); requests wait until their state fits."""

    def __init__(self, hbm_budget: int = 80 << 30, max_slots: int = 1024, max_side: int = 4096,
                 scheme: str = "fd5", run_steps: int = 64, segment_rows: int | None = None,
                 device=None, return_fields: bool = False):
        self.scheme = scheme
        # also hand each finished request its final (rho - 1, ux, uy) fields
        # (host float32 arrays [ny, nx]), copied before its slot is released
        self.return_fields = bool(return_fields)
        self.run_steps = int(run_steps)
        self.batch = F.Batch(scheme, max_lattices=max_slots, arena_bytes=int(hbm_budget),
                             max_side=max_side, device=device)
        if segment_rows:
            self.batch.set_segment_rows(segment_rows)
        self.queue = collections.deque()
        self.active = {}        # slot -> [request, steps left]
        self.done = []
        self.gpu_steps = 0      # runs issued x steps
        self.work_done = 0      # node updates completed

    def submit(self, req: Request):
        self.queue.append(req)

    def _admit(self, now: float) -> int:
        n = 0
        while self.queue and self.queue[0].arrival <= now:
            req = self.queue[0]
            try:
                slot = self.batch.add(req.config(self.scheme))
            except F.FdlbmError as e:
                if e.status == F.ERR_NOMEM and self.active:
                    break       # wait for slots or arena space to free up
                raise           # larger than the whole budget, or invalid
            self.queue.popleft()
            self.batch.init_modes(slot, req.modes)
            req.admitted = now
            self.active[slot] = [req, req.steps]
            n += 1
        return n

    def _retire(self, slot: int, now: float):
        req, _ = self.active.pop(slot)
        b = self.batch
        res = {"mass": float(b.reduce(slot, "mass")[0]),
               "momentum": [float(v) for v in b.reduce(slot, "momentum")],
               "energy": float(b.reduce(slot, "energy")[0]),
               "max_u": float(b.reduce(slot, "maxabs")[0])}
        if req.modes:
            md = req.modes[0]
            res["mode0"] = [float(v) for v in b.reduce(slot, "mode", (md.m, md.n))]
        if self.return_fields:
            fields = b.moments(slot)
            res["fields"] = [t.cpu().numpy() for t in fields]
            b.sync()
        req.result = res
        req.finished = now
        b.remove(slot)
        self.done.append(req)

    def serve(self, requests, clock=time.perf_counter):
        """Run a request stream to completion; arrival times are relative to
        the call.  Returns the finished requests in completion order."""
        for r in sorted(requests, key=lambda r: r.arrival):
            self.submit(r)
        t0 = clock()
        while self.queue or self.active:
            now = clock() - t0
            self._admit(now)
            if not self.active:
                # idle: wait for the next arrival
                if self.queue:
                    time.sleep(max(0.0, min(0.05, self.queue[0].arrival - (clock() - t0))))
                continue
            run = self.run_steps
            counts = {s: min(left, run) for s, (req, left) in self.active.items()}
            self.batch.step(run, counts)
            self.batch.sync()
            self.gpu_steps += run
            now = clock() - t0
            for s in list(self.active):
                req, left = self.active[s]
                took = counts[s]
                self.work_done += took * req.nodes
                left -= took
                if left <= 0:
                    self._retire(s, now)
                else:
                    self.active[s][1] = left
        return self.done


def latency_stats(done, wall: float):
    lat = np.array([r.finished - r.arrival for r in done])
    q = np.array([r.admitted - r.arrival for r in done])
    return {"requests": len(done), "wall_s": round(wall, 3),
            "solves_per_s": round(len(done) / wall, 3) if wall > 0 else None,
            "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "mean_queue_s": round(float(q.mean()), 4),
            "node_updates": int(sum(r.work for r in done))}


def measure_stream(n: int, rate: float = 200.0, hbm_budget: int = 80 << 30, device=None):
    """Serve the first n requests of the specified stream (Poisson arrivals at
    `rate` per second, sides log-uniform in [64, 4096], 100-20000 steps,
    shear wave / 1-4 modes / Poiseuille channel, nu U[0.002, 0.1]) under an
    HBM budget; returns the latency statistics and the sustained MLUPS."""
    reqs = make_requests(n, rate, inputs.seed_for(4))
    srv = Server(hbm_budget=hbm_budget, max_slots=1024, max_side=4096, device=device)
    t0 = time.perf_counter()
    done = srv.serve(reqs)
    wall = time.perf_counter() - t0
    out = latency_stats(done, wall)
    out["mlups"] = round(srv.work_done / wall / 1e6, 1)
    out["gpu_launches"] = int(srv.batch.launches)
    srv.batch.close()
    return out


def bench_main(args):
    """bench.py --workload serving: the Poisson stream (mean 200 requests/s) of
    mixed FD-LBM requests, 80 GB HBM budget; then the same mix at 25/50/75 %
    of the measured capacity.  Prints one JSON line."""
    import torch
    from . import build
    build.build()
    torch.cuda.set_device(0)
    n = int(getattr(args, "requests", 0) or 2000)
    reqs = make_requests(n, 200.0, inputs.seed_for(4))
    srv = Server(hbm_budget=80 << 30, max_slots=1024, max_side=4096)
    t0 = time.perf_counter()
    done = srv.serve(reqs)
    wall = time.perf_counter() - t0
    main = latency_stats(done, wall)
    capacity = srv.work_done / wall  # node updates per second under overload
    main["mlups"] = round(capacity / 1e6, 1)
    sweeps = {}
    mean_work = float(np.mean([r.work for r in reqs]))
    for frac in (0.25, 0.5, 0.75):
        rate = frac * capacity / mean_work
        sub = make_requests(max(40, n // 20), rate, inputs.seed_for(4) + int(frac * 100))
        s2 = Server(hbm_budget=80 << 30, max_slots=1024, max_side=4096)
        t1 = time.perf_counter()
        d2 = s2.serve(sub)
        sweeps[f"{int(frac * 100)}%"] = dict(latency_stats(d2, time.perf_counter() - t1),
                                             rate_per_s=round(rate, 3))
        del s2
        torch.cuda.empty_cache()
    line = {"metric": "FD-LBM D2Q9 MLUPS & %HBM peak vs MRT-LBM; served solves/s, p99 latency",
            "workload": "serving", "value": main["solves_per_s"], "unit": "solves/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n} requests, Poisson 200/s, sides log-U[64,4096], steps "
                                   "log-U[100,20000], shear wave / 1-4 modes / Poiseuille, "
                                   "nu U[0.002,0.1], FD-LBM five-point FP32, 80 GB HBM budget",
                       "run_steps": srv.run_steps},
            "p50_latency_s": main["p50_latency_s"], "p99_latency_s": main["p99_latency_s"],
            "overload": main, "sub_saturation": sweeps, "vs_baseline": None}
    print(json.dumps(line), flush=True)
