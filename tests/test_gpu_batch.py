"""Batched FD-LBM lattices (fdlbm_batch_* through the C ABI): every slot of a
mixed batch -- uneven sizes (odd sides, sides below one strip, several
strips and segments), its own viscosity, periodic or channel with force --
equals the same lattice stepped alone by the single-lattice path, and a few
slots are checked against the FP64 oracle directly."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import amplitude, as_f32, gpu_run, max_err, oracle_run

pytestmark = pytest.mark.gpu
TOL32 = 1e-5

SHAPES = [(16, 16), (40, 33), (97, 131), (128, 96), (131, 257), (256, 64), (300, 17), (385, 200)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build
    build.build()


def _fields(nx, ny, seed):
    d, ux, uy = inputs.random_fields(nx, ny, 0.01, seed=seed, rho_amp=0.003)
    return as_f32((d, ux, uy))


def _to_dev(f):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in f]


@pytest.mark.parametrize("scheme", ["fd3", "fd5"])
def test_batch_equals_single_lattices(scheme):
    from paper_1803_00437_gb300 import fdlbm as F
    b = F.Batch(scheme, max_lattices=16, arena_bytes=64 << 20, max_side=512)
    cfgs, fields, slots = [], [], []
    for i, (nx, ny) in enumerate(SHAPES):
        nu = 0.005 + 0.01 * i
        cfg = F.LatticeConfig(nx, ny, scheme, s_xx=F.nu_to_s(nu), s_e=1.5)
        f = _fields(nx, ny, 100 + i)
        s = b.add(cfg)
        b.init(s, *_to_dev(f))
        cfgs.append(cfg), fields.append(f), slots.append(s)
    b.step(37)
    b.sync()
    for cfg, f, s in zip(cfgs, fields, slots):
        single, _ = gpu_run(cfg, f, 37)
        got = [t.cpu().numpy().astype(np.float64) for t in b.moments(s)]
        b.sync()
        assert max_err(got, single, amplitude(f)) <= TOL32, (cfg.nx, cfg.ny)


def test_batch_against_oracle(oracle):
    from paper_1803_00437_gb300 import fdlbm as F
    b = F.Batch("fd5", max_lattices=4, arena_bytes=16 << 20, max_side=256)
    for i, (nx, ny) in enumerate([(37, 29), (130, 50)]):
        cfg = F.LatticeConfig(nx, ny, "fd5", s_xx=F.nu_to_s(0.02 + 0.01 * i), s_e=1.4)
        f = _fields(nx, ny, 7 + i)
        s = b.add(cfg)
        b.init(s, *_to_dev(f))
        b.step(60)
        got = [t.cpu().numpy().astype(np.float64) for t in b.moments(s)]
        b.sync()
        ref = oracle_run(oracle, cfg, f, 60)
        b.step(0)
        assert max_err(got, ref, amplitude(f)) <= TOL32
        b.remove(s)


def test_batch_channels_with_force_and_per_slot_steps():
    from paper_1803_00437_gb300 import fdlbm as F
    b = F.Batch("fd5", max_lattices=8, arena_bytes=32 << 20, max_side=256)
    nu = 1 / np.sqrt(108)
    cases = [(64, 24, 0.5, (2e-5, 0.0), 120), (40, 33, 0.3, (1e-5, -3e-6), 75),
             (200, 48, 1.0, (0.0, 0.0), 40), (96, 64, 0.5, (0.0, 0.0), 0)]
    slots = []
    for i, (nx, ny, xi, force, n) in enumerate(cases):
        cfg = F.LatticeConfig(nx, ny, "fd5", s_xx=F.nu_to_s(nu), s_e=1.5,
                              boundary="walls_y" if i < 3 else "periodic", wall_xi=xi, force=force)
        f = _fields(nx, ny, 40 + i)
        s = b.add(cfg)
        b.init(s, *_to_dev(f))
        slots.append((s, cfg, f, n))
    b.step(120, {s: n for s, _, _, n in slots})
    b.sync()
    for s, cfg, f, n in slots:
        single, _ = gpu_run(cfg, f, n)
        got = [t.cpu().numpy().astype(np.float64) for t in b.moments(s)]
        b.sync()
        assert max_err(got, single, amplitude(f)) <= TOL32, (cfg.nx, cfg.ny, n)


def test_batch_slots_come_and_go():
    """Continuous batching: slots removed and added between steps keep the
    others' results unchanged; arena space is reused."""
    from paper_1803_00437_gb300 import fdlbm as F
    b = F.Batch("fd5", max_lattices=4, arena_bytes=8 << 20, max_side=256)
    cfg_a = F.LatticeConfig(200, 100, "fd5", s_xx=F.nu_to_s(0.01))
    cfg_b = F.LatticeConfig(150, 120, "fd5", s_xx=F.nu_to_s(0.03))
    fa, fb = _fields(200, 100, 1), _fields(150, 120, 2)
    sa = b.add(cfg_a)
    b.init(sa, *_to_dev(fa))
    sb = b.add(cfg_b)
    b.init(sb, *_to_dev(fb))
    b.step(10)
    b.remove(sb)
    b.step(5)
    sc = b.add(cfg_b)
    assert sc == sb  # the freed slot and space are reused
    b.init(sc, *_to_dev(fb))
    b.step(20)
    b.sync()
    single_a, _ = gpu_run(cfg_a, fa, 35)
    single_b, _ = gpu_run(cfg_b, fb, 20)
    for s, ref, f in ((sa, single_a, fa), (sc, single_b, fb)):
        got = [t.cpu().numpy().astype(np.float64) for t in b.moments(s)]
        b.sync()
        assert max_err(got, ref, amplitude(f)) <= TOL32
    with pytest.raises(F.FdlbmError):
        for _ in range(10):
            b.add(F.LatticeConfig(256, 256, "fd5"))


def test_batch_tuner_and_reductions():
    from paper_1803_00437_gb300 import fdlbm as F
    b = F.Batch("fd5", max_lattices=8, arena_bytes=64 << 20, max_side=512)
    slots = [b.add(F.LatticeConfig(L, L, "fd5", s_xx=F.nu_to_s(0.01))) for L in (64, 200, 512)]
    best = b.tune(steps=2)
    assert best in (16, 32, 64, 128, 256)
    for s, L in zip(slots, (64, 200, 512)):
        modes = inputs.random_modes(L, L, 4, 1e-3, seed=L)
        b.init_modes(s, modes)
        m = b.reduce(s, "mode", (modes[0].m, modes[0].n))
        ref = inputs.transverse_modes(L, L, modes)
        X, Y = np.meshgrid(np.arange(L), np.arange(L))
        kx, ky = 2 * np.pi * modes[0].m / L, 2 * np.pi * modes[0].n / L
        k = np.hypot(kx, ky)
        c = (((-ky * ref[1] + kx * ref[2]) / k) * np.exp(-1j * (kx * X + ky * Y))).mean()
        assert abs(m[0] - c.real) < 1e-9 and abs(m[1] - c.imag) < 1e-9
