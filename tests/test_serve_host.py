"""Host logic of the serving loop on the CPU: the batch is replaced by a
fake that keeps the bookkeeping of fdlbm_batch_* (slots, an arena budget in
bytes, per-slot steps taken) without a device, so admission order, waiting
for budget, per-slot step counts, retirement and the latency statistics are
checked without a GPU."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import fdlbm as F
from paper_1803_00437_gb300 import serve


class FakeBatch:
    """Slots and an arena of `arena_bytes`; a lattice takes 24 B per node
    (two FP32 copies of three fields), like the real arena up to padding."""

    def __init__(self, scheme="fd5", max_lattices=64, arena_bytes=1 << 30, max_side=512,
                 device=None):
        self.max_lattices, self.arena, self.max_side = max_lattices, arena_bytes, max_side
        self.slots = {}       # slot -> [cfg, steps taken]
        self.used = 0
        self.step_calls = []
        self.log = []

    def add(self, cfg):
        need = 24 * cfg.nx * cfg.ny
        if max(cfg.nx, cfg.ny) > self.max_side:
            raise F.FdlbmError(F.ERR_INVALID, "too large")
        if len(self.slots) >= self.max_lattices or self.used + need > self.arena:
            raise F.FdlbmError(F.ERR_NOMEM, "no room")
        slot = min(set(range(self.max_lattices)) - set(self.slots))
        self.slots[slot] = [cfg, 0]
        self.used += need
        self.log.append(("add", slot))
        return slot

    def remove(self, slot):
        cfg, _ = self.slots.pop(slot)
        self.used -= 24 * cfg.nx * cfg.ny
        self.log.append(("remove", slot))

    def init_modes(self, slot, modes, mean_velocity=(0.0, 0.0)):
        self.slots[slot][1] = 0

    def set_segment_rows(self, rows):
        pass

    def step(self, nsteps, slot_steps=None):
        self.step_calls.append((nsteps, dict(slot_steps or {})))
        for s in self.slots:
            self.slots[s][1] += min(nsteps, (slot_steps or {}).get(s, nsteps))

    def sync(self):
        pass

    def reduce(self, slot, what, args=None):
        taken = self.slots[slot][1]
        return np.array([float(taken), 0.0]) if what in ("momentum", "mode", "maxabs") \
            else np.array([float(taken)])


class FakeClock:
    """Time advances only when the server steps (1 ms per run), so arrival
    handling is deterministic."""

    def __init__(self, batch):
        self.batch, self.t = batch, 0.0

    def __call__(self):
        return self.t + 1e-3 * len(self.batch.step_calls)


@pytest.fixture
def server(monkeypatch):
    monkeypatch.setattr(F, "Batch", FakeBatch)
    monkeypatch.setattr(serve.time, "sleep", lambda s: None)

    def make(budget, slots=8, run_steps=64):
        return serve.Server(hbm_budget=budget, max_slots=slots, max_side=4096,
                            run_steps=run_steps)
    return make


def _req(rid, side, steps, arrival=0.0):
    return serve.Request(rid, "shear", side, side, steps, 0.01, arrival,
                         [serve.inputs.Mode(0, 1, 1e-3, 0.0)])


def test_every_request_takes_exactly_its_steps(server):
    srv = server(1 << 30)
    reqs = [_req(0, 64, 100), _req(1, 128, 64), _req(2, 32, 1), _req(3, 96, 300)]
    done = srv.serve(reqs, clock=FakeClock(srv.batch))
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    for r in done:
        assert r.result["mass"] == r.steps  # the fake reports the steps it was given
    # runs are run_steps long; each slot's count is min(remaining, run)
    nsteps, counts = srv.batch.step_calls[0]
    assert nsteps == 64 and sorted(counts.values()) == [1, 64, 64, 64]
    assert srv.work_done == sum(r.work for r in reqs)


def test_admission_is_fifo_and_waits_for_budget(server):
    # the budget holds one 128^2 lattice (393 kB) or several small ones
    srv = server(24 * 128 * 128 + 24 * 32 * 32)
    reqs = [_req(0, 128, 200), _req(1, 128, 10), _req(2, 32, 10)]
    done = srv.serve(reqs, clock=FakeClock(srv.batch))
    adds = [e for e in srv.batch.log if e[0] == "add"]
    # request 2 fits beside request 0, but must not overtake request 1
    order = [r.rid for r in sorted(done, key=lambda r: r.admitted)]
    assert order == [0, 1, 2]
    r0, r1, r2 = sorted(done, key=lambda r: r.rid)
    assert r1.admitted >= r0.finished and r2.admitted >= r1.admitted
    assert len(adds) == 3 and srv.batch.used == 0


def test_request_larger_than_budget_is_an_error(server):
    srv = server(24 * 64 * 64)
    with pytest.raises(F.FdlbmError):
        srv.serve([_req(0, 128, 10)], clock=FakeClock(srv.batch))


def test_slots_are_reused_and_latencies_reported(server):
    srv = server(1 << 30, slots=2)
    reqs = [_req(i, 64, 50 + 10 * i, arrival=0.0) for i in range(5)]
    done = srv.serve(reqs, clock=FakeClock(srv.batch))
    assert len(done) == 5
    assert all(s in (0, 1) for e, s in srv.batch.log if e == "add")
    st = serve.latency_stats(done, wall=1.0)
    assert st["requests"] == 5 and st["p99_latency_s"] >= st["p50_latency_s"] >= 0.0
    assert st["node_updates"] == sum(r.work for r in reqs)


def test_request_stream_statistics():
    reqs = serve.make_requests(400, 200.0, seed=7)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    assert 0.5 / 200 < np.diff(t).mean() < 2.0 / 200
    sides = np.array([r.nx for r in reqs])
    assert sides.min() >= 64 and sides.max() <= 4096
    steps = np.array([r.steps for r in reqs])
    assert steps.min() >= 100 and steps.max() <= 20000
    kinds = {r.kind for r in reqs}
    assert kinds == set(serve.KINDS)
    for r in reqs:
        if r.kind == "poiseuille":
            assert r.ny == max(16, r.nx // 4) and r.force[0] > 0 and not r.modes
        else:
            assert r.nx == r.ny and 1 <= len(r.modes) <= 4
