"""GPU tests of the streaming step's launch plans: any plan (equal row
segments, or long segments followed by short ones) gives the lattice of the
FP64 oracle, the same lattice bit for bit whatever the plan, and the
autotuner (Lattice.tune) times the candidates without advancing the state."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import amplitude, as_f32, max_err, oracle_run

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build
    build.build()


def _nu(nu):
    return 1.0 / (3.0 * nu + 0.5)


def _run(cfg, fields32, nsteps, plan=None):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    lat = F.Lattice(cfg)
    if plan is not None:
        lat.set_stream_plan(*plan)
    lat.init(*[torch.from_numpy(np.ascontiguousarray(f)).to(lat.device) for f in fields32])
    lat.step(nsteps)
    out = [t.cpu().numpy() for t in lat.moments()]
    return out, lat


# (seg_rows, nsegs, tail_rows): long segments then short ones with a ragged
# last one, a first part of one segment, odd lengths, and equal segments
PLANS = [(48, 2, 16), (40, 1, 7), (96, 1, 13), (24, 5, 24), (17, 100, 17)]


@pytest.mark.parametrize("scheme", ["fd3", "fd5"])
@pytest.mark.parametrize("plan", PLANS)
def test_plans_match_the_oracle_periodic(oracle, scheme, plan):
    """264 x 150 periodic (a partial last strip, two-warp and one-warp CTAs),
    32 seeded modes plus density noise, 120 steps."""
    from paper_1803_00437_gb300 import fdlbm as F
    nx, ny = 264, 150
    modes = inputs.random_modes(nx, ny, 32, 2e-3, seed=11)
    d, ux, uy = inputs.transverse_modes(nx, ny, modes)
    d = inputs.random_fields(nx, ny, 0.0, seed=4, rho_amp=1e-3)[0]
    f = as_f32((d, ux, uy))
    cfg = F.LatticeConfig(nx, ny, scheme, s_xx=_nu(0.01), s_e=1.5, flags=F.FLAG_STREAM)
    gpu, lat = _run(cfg, f, 120, plan)
    p = lat.stream_plan()
    assert (p["seg_rows"], p["tail_rows"]) == (plan[0], plan[2] if p["ntail"] else plan[0])
    ref = oracle_run(oracle, cfg, f, 120)
    assert max_err([g.astype(np.float64) for g in gpu], ref, amplitude(f)) <= TOL32


@pytest.mark.parametrize("scheme,xi", [("fd5", 0.3), ("fd3", 0.8)])
@pytest.mark.parametrize("plan", [(48, 1, 16), (24, 2, 9)])
def test_plans_match_the_oracle_channel(oracle, scheme, xi, plan):
    """Channel 264 x 101 with body force: the virtual rows above and below sit
    in the first long and the last short segment; 200 steps."""
    from paper_1803_00437_gb300 import fdlbm as F
    nx, ny = 264, 101
    f = as_f32(inputs.random_fields(nx, ny, 0.01, seed=5, rho_amp=0.002))
    cfg = F.LatticeConfig(nx, ny, scheme, s_xx=_nu(1 / np.sqrt(108)), s_e=1.5,
                          boundary="walls_y", wall_xi=xi, force=(2e-5, -1e-6),
                          flags=F.FLAG_STREAM)
    gpu, _ = _run(cfg, f, 200, plan)
    ref = oracle_run(oracle, cfg, f, 200)
    assert max_err([g.astype(np.float64) for g in gpu], ref, amplitude(f)) <= TOL32


@pytest.mark.parametrize("storage", ["f32", "i16"])
def test_every_plan_gives_the_same_lattice(storage):
    """The plan only moves the segment boundaries: each node's arithmetic is
    the same, so the lattices agree bit for bit (FD-5, 1032 x 517, 20 steps)."""
    from paper_1803_00437_gb300 import fdlbm as F
    nx, ny = 1032, 517
    f = as_f32(inputs.random_fields(nx, ny, 0.01, seed=9, rho_amp=0.002))
    cfg = F.LatticeConfig(nx, ny, "fd5", s_xx=_nu(0.01), s_e=1.5, storage=storage,
                          storage_range=0.05, flags=F.FLAG_STREAM)
    base, lat = _run(cfg, f, 20)
    assert lat.stream_plan() is not None
    for plan in [(64, 7, 16), (200, 2, 24), (16, 33, 16), (517, 1, 517), (72, 1, 5)]:
        got, _ = _run(cfg, f, 20, plan)
        for g, b in zip(got, base):
            assert np.array_equal(g, b), plan


def test_tune_keeps_the_state_and_picks_a_candidate():
    """Lattice.tune on a 2048 x 1024 FD-5 lattice: the chosen plan is one of
    the candidates, the state after tuning is the state before it, and the
    tuned lattice then steps exactly like an untuned one."""
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    nx, ny = 2048, 1024
    f = as_f32(inputs.random_fields(nx, ny, 0.01, seed=12, rho_amp=0.002))
    cfg = F.LatticeConfig(nx, ny, "fd5", s_xx=_nu(0.01), s_e=1.5)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in f]
    lat = F.Lattice(cfg)
    lat.init(*dev)
    lat.step(3)
    before = [t.cpu().numpy() for t in lat.moments()]
    best, timings = lat.tune(steps=2, max_candidates=6)
    after = [t.cpu().numpy() for t in lat.moments()]
    for a, b in zip(after, before):
        assert np.array_equal(a, b)
    resident = lat.stream_plan()["resident_ctas"]
    cands = F.stream_plan_candidates(nx, ny, "fd5", "f32", resident, 6)
    assert best in cands and set(timings) == set(cands)
    assert all(t > 0 for t in timings.values())
    p = lat.stream_plan()
    assert (p["seg_rows"], p["nsegs"]) == (best[0], best[1])
    lat.step(5)
    ref = F.Lattice(cfg)
    ref.init(*dev)
    ref.step(8)
    for a, b in zip(lat.moments(), ref.moments()):
        assert torch.equal(a, b)
    lat.set_stream_plan()  # back to the model's plan
    p = lat.stream_plan()
    m = F.stream_plan(nx, ny, "fd5", "f32", resident)
    assert (p["seg_rows"], p["nsegs"], p["ntail"]) == (m["seg_rows"], m["nsegs"], m["ntail"])


def test_set_stream_plan_rejects_lattices_that_do_not_stream_and_bad_values():
    from paper_1803_00437_gb300 import fdlbm as F
    for cfg in (F.LatticeConfig(512, 256, "mrt", s_xx=_nu(0.01)),
                F.LatticeConfig(512, 256, "fd5", s_xx=_nu(0.01), flags=F.FLAG_TILED),
                F.LatticeConfig(512, 256, "fd9", s_xx=_nu(0.15))):
        lat = F.Lattice(cfg)
        with pytest.raises(F.FdlbmError):
            lat.set_stream_plan(64, 2, 16)
        lat.step(1)
        assert lat.stream_plan() is None
    lat = F.Lattice(F.LatticeConfig(512, 256, "fd5", s_xx=_nu(0.01), flags=F.FLAG_STREAM))
    assert lat.stream_plan() is None  # not stepped yet
    for bad in [(0, 2, 16), (64, 0, 16), (64, 2, 0), (257, 1, 16), (-8, 2, 16)]:
        with pytest.raises(F.FdlbmError):
            lat.set_stream_plan(*bad)
    lat.set_stream_plan(64, 2, 16)
    lat.step(1)
    p = lat.stream_plan()
    assert (p["seg_rows"], p["nsegs"], p["tail_rows"], p["ntail"]) == (64, 2, 16, 8)
