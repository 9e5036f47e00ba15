"""The sharding design for one lattice over several GPUs (y-slabs, each step
preceded by an exchange of the h rows nearest each slab edge with the two
neighbours), checked on the CPU with the FP64 oracle as two gloo ranks.

Each rank holds half of a periodic lattice, sends its top and bottom h rows
to its neighbours, builds its slab padded with the h rows it received on
each side, advances the padded slab one step as a periodic lattice of its
own (the padding's rows come out wrong and are dropped) and keeps its own
rows.  After several steps the gathered halves equal the whole lattice's
run bit for bit when h = r + 1 (the stencil's radius plus the one link of
the propagation, Eq. 2): 3 rows for five points, 2 for three points, 1 for
LW-ACM; with h - 1 rows they do not.  No GPU and no data path of the
library are involved: the ranks run the oracle."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, STEPS = 24, 40, 6
SCHEMES = {"fd5": (5, 3), "fd3": (3, 2), "lwacm": (200, 1)}  # oracle code, halo rows h


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fields():
    sys.path.insert(0, ROOT)
    from paper_1803_00437_gb300 import inputs
    d, ux, uy = inputs.random_fields(NX, NY, 0.02, seed=51, rho_amp=0.01)
    return np.stack([1.0 + d, ux, uy])


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import ref
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ref.set_threads(1)
    rows = NY // world
    mine = _fields()[:, rank * rows:(rank + 1) * rows].copy()
    up, down = (rank + 1) % world, (rank - 1) % world
    out = {}
    for name, (code, h) in SCHEMES.items():
        for depth in (h, h - 1):
            f = mine.copy()
            for _ in range(STEPS):
                if depth == 0:
                    below = above = np.zeros((3, 0, NX))
                else:
                    # my top rows go up (they are the row block below the upper
                    # neighbour); my bottom rows go down
                    top = torch.from_numpy(np.ascontiguousarray(f[:, -depth:]))
                    bot = torch.from_numpy(np.ascontiguousarray(f[:, :depth]))
                    from_below = torch.empty_like(top)
                    from_above = torch.empty_like(bot)
                    reqs = [dist.isend(top, up), dist.isend(bot, down),
                            dist.irecv(from_below, down), dist.irecv(from_above, up)]
                    for r in reqs:
                        r.wait()
                    below, above = from_below.numpy(), from_above.numpy()
                padded = np.concatenate([below, f, above], axis=1)
                p = ref.params(NX, padded.shape[1], code, 1.0 / (3 * 0.02 + 0.5), 1.5)
                r_, x_, y_ = ref.run(p, padded[0], padded[1], padded[2], 1)
                f = np.stack([r_, x_, y_])[:, depth:depth + rows]
            out[(name, depth)] = f
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_slab_halo_depth_two_gloo_ranks():
    sys.path.insert(0, ROOT)
    from oracle import ref
    ref.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    f0 = _fields()
    for name, (code, h) in SCHEMES.items():
        p = ref.params(NX, NY, code, 1.0 / (3 * 0.02 + 0.5), 1.5)
        whole = np.stack(ref.run(p, f0[0], f0[1], f0[2], STEPS))
        halves = np.concatenate([got[0][(name, h)], got[1][(name, h)]], axis=1)
        assert np.array_equal(halves, whole), name  # h rows suffice, exactly
        short = np.concatenate([got[0][(name, h - 1)], got[1][(name, h - 1)]], axis=1)
        assert np.abs(short - whole).max() > 1e-12, name  # h - 1 rows do not
