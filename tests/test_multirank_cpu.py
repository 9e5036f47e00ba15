"""Host logic of the N>1 bench path, run as two gloo ranks on the CPU: each
rank holds an independent lattice (replicas, no data-path collective), the
step time is the slowest rank's, and the whole-job throughput sums the node
updates of all ranks.  The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_info()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    # rank r: (r+1) * 1000 nodes per step, (r+1) * 2 ms per step
    nodes = (r + 1) * 1000
    ms = (r + 1) * 2.0
    mlups, ms_max = bench.job_mlups(nodes, ms, w)
    mx = bench.all_max(float(r), w)
    sm = bench.all_sum(float(r + 1), w)

    class A:
        steps, warmup, side = 1, 0, 64
    # non-zero ranks of the reference arm exit without work or output
    ref = bench.run_reference(A) if r != 0 else None
    q.put((r, w, local, mlups, ms_max, mx, sm, ref))
    bench.barrier(w)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_aggregate_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    total_nodes, slowest_ms = 1000 + 2000, 4.0
    for r, (rank, w, local, mlups, ms_max, mx, sm, ref) in enumerate(out):
        assert (rank, w, local) == (r, 2, r)
        assert ms_max == slowest_ms
        assert mlups == pytest.approx(total_nodes / (slowest_ms / 1e3) / 1e6, rel=1e-15)
        assert mx == 1.0 and sm == 3.0
        assert ref is None


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_info() == (0, 1, 0)
    bench.dist_init(1, "gloo")
    bench.barrier(1)
    assert bench.job_mlups(4096, 2.0, 1) == (4096 / 2e-3 / 1e6, 2.0)
