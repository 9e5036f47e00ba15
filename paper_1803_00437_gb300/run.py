"""Run one lattice for a number of steps and report its throughput.

    python -m paper_1803_00437_gb300.run --side 4096 --scheme fd5 --steps 5

Builds the library if needed, initialises a periodic side x side lattice
with 32 seeded transverse modes (amplitude 1e-3, nu = 0.01, s_e = 1.5),
advances it, and prints one JSON line (steps, milliseconds per step, MLUPS,
max |u| and any FP64 reductions asked for with --reduce).  Used to drive
profiler captures of a single kernel.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--scheme", default="fd5", choices=["fd3", "fd5", "fd9", "mrt", "lwacm"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "i16"])
    ap.add_argument("--range", type=float, default=0.02,
                    help="largest |value| of the i16 fixed-point storage")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=0, help="untimed steps before the timed ones")
    ap.add_argument("--per-step", action="store_true",
                    help="one fdlbm_step call per step")
    ap.add_argument("--plan", default=None,
                    help="row segments of the streaming step, SEG_ROWS,NSEGS,TAIL_ROWS "
                         "(fdlbm_set_stream_plan)")
    ap.add_argument("--tune", action="store_true",
                    help="time the streaming step's candidate plans first and keep the "
                         "fastest (Lattice.tune; the state is restored)")
    ap.add_argument("--nu", type=float, default=0.01)
    ap.add_argument("--walls", type=float, default=None, metavar="XI",
                    help="a channel: walls in y at offset XI (Sec. 3-b), periodic in x")
    ap.add_argument("--force", type=float, default=0.0, help="body force along x (channels)")
    ap.add_argument("--modes", type=int, default=32)
    ap.add_argument("--reduce", nargs="*", default=[],
                    choices=["mass", "momentum", "energy", "maxabs"],
                    help="FP64 reductions of the final state to report")
    args = ap.parse_args(argv)

    import torch
    from . import build, fdlbm as F, inputs
    build.build()
    n = args.side
    walls = {} if args.walls is None else dict(boundary="walls_y", wall_xi=args.walls,
                                               force=(args.force, 0.0))
    lat = F.Lattice(F.LatticeConfig(n, n, args.scheme, s_xx=F.nu_to_s(args.nu), s_e=1.5,
                                    storage=args.storage, storage_range=args.range, **walls))
    lat.init_modes(inputs.random_modes(n, n, args.modes, 1e-3, seed=inputs.seed_for(1)))
    if args.plan:
        lat.set_stream_plan(*[int(v) for v in args.plan.split(",")])
    if args.tune:
        lat.tune()
    lat.step(args.warmup)
    lat.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    if args.per_step:
        for _ in range(args.steps):
            lat.step(1)
    else:
        lat.step(args.steps)
    e1.record(lat.stream)
    lat.sync()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    reductions = {w: [float(v) for v in lat.reduce(w)] for w in args.reduce}
    print(json.dumps({"side": n, "scheme": args.scheme, "storage": args.storage,
                      "boundary": "periodic" if args.walls is None else f"walls_y xi={args.walls}",
                      "steps": args.steps, "ms_per_step": round(ms, 4),
                      "mlups": round(n * n / ms / 1e3, 1), "launches": lat.launches,
                      "stream_plan": lat.stream_plan(),
                      "max_u": float(lat.reduce("maxabs")[0]), "reductions": reductions}))


if __name__ == "__main__":
    main()
