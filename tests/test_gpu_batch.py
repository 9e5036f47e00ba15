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


@pytest.mark.parametrize("scheme", ["fd3", "fd5"])
def test_narrow_last_strips_equal_wide_ones(scheme):
    """A lattice's last strip of <= 56 columns on 2-column lanes gives the same
    lattice bit for bit as 4-column lanes (the same operations per column):
    single narrow strips (16, 40, 56 columns), a narrow last strip after full
    ones (128, 176, 385), one just too wide (57, 300), periodic and channels
    with force."""
    from paper_1803_00437_gb300 import fdlbm as F
    shapes = [(16, 20), (40, 33), (56, 24), (57, 31), (128, 40), (176, 45), (300, 17), (385, 26)]
    out = {}
    for narrow in (True, False):
        b = F.Batch(scheme, max_lattices=2 * len(shapes), arena_bytes=64 << 20, max_side=512)
        b.set_narrow_strips(narrow)
        slots = []
        for i, (nx, ny) in enumerate(shapes):
            for walls in (False, True):
                kw = dict(boundary="walls_y", wall_xi=0.4, force=(1e-5, 0.0)) if walls else {}
                cfg = F.LatticeConfig(nx, ny, scheme, s_xx=F.nu_to_s(0.01 + 0.005 * i), s_e=1.5,
                                      **kw)
                s = b.add(cfg)
                b.init(s, *_to_dev(_fields(nx, ny, 300 + i)))
                slots.append(s)
        b.step(23)
        b.sync()
        out[narrow] = [[t.cpu().numpy() for t in b.moments(s)] for s in slots]
        b.sync()
        b.close()
    for a, w in zip(out[True], out[False]):
        for x, y in zip(a, w):
            assert np.array_equal(x, y)


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


def test_full_batched_workload_sample_vs_oracle(oracle):
    """The batched throughput workload at full size -- 4096 periodic lattices,
    sides U{32..512}, nu U[0.002, 0.1], one transverse mode of A = 1e-3 each
    -- in the benchmark's configuration (arena sized as the benchmark sizes
    it, tuned rows per item, graph-captured runs of 64 steps), 200 steps.
    A seeded sample of 64 lattices starts from host-generated fields and is
    compared element by element with the oracle (FP32 bound 1e-5 of A); their
    mode decay rates are compared where the field bound resolves them
    (relative error <= 2 sqrt(2) B / (a_n Gamma n), a_n >= 10 B, B = 1e-5 A),
    and reported against the linear shear root (single transverse modes are
    linear; modes decayed below FP64 resolution are left out)."""
    import json
    import os
    import sys
    from oracle import linear
    from paper_1803_00437_gb300 import fdlbm as F
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    steps, A = 200, 1e-3
    lats = inputs.batch_lattices(4096, inputs.seed_for(2))
    sides = [L for L, _, _ in lats]
    arena = int(bench.batch_arena_bytes(sides) * 1.02) + (1 << 20)
    b = F.Batch("fd5", max_lattices=len(lats), arena_bytes=arena, max_side=512)
    slots = [b.add(F.LatticeConfig(L, L, "fd5", s_xx=F.nu_to_s(nu), s_e=1.5))
             for L, nu, _ in lats]
    b.tune(steps=4)
    rng = np.random.default_rng(2017)
    sample = set(int(i) for i in rng.choice(len(lats), 64, replace=False))
    host = {}
    for i, (s, (L, nu, md)) in enumerate(zip(slots, lats)):
        if i in sample:
            host[i] = as_f32(inputs.transverse_modes(L, L, [md]))
            b.init(s, *_to_dev(host[i]))
        else:
            b.init_modes(s, [md])
    b.step(steps)
    b.sync()
    oracle.set_threads(os.cpu_count() or 1)
    worst, rates, lin = 0.0, [], []
    for i in sorted(sample):
        L, nu, md = lats[i]
        got = [t.cpu().numpy().astype(np.float64) for t in b.moments(slots[i])]
        b.sync()
        cfg = F.LatticeConfig(L, L, "fd5", s_xx=F.nu_to_s(nu), s_e=1.5)
        ref = oracle_run(oracle, cfg, host[i], steps)
        err = max_err(got, ref, A)
        worst = max(worst, err)
        assert err <= TOL32, (i, L, nu)
        X, Y = np.meshgrid(np.arange(L), np.arange(L))
        kx, ky = 2 * np.pi * md.m / L, 2 * np.pi * md.n / L
        k = np.hypot(kx, ky)

        def amp(f):
            return (((-ky * f[1] + kx * f[2]) / k) * np.exp(-1j * (kx * X + ky * Y))).mean()
        a0 = amp([a.astype(np.float64) for a in host[i]])
        a_ref = amp(ref)
        g_ref = -np.log(abs(a_ref / a0)) / steps
        g_gpu = -np.log(abs(amp(got) / a0)) / steps
        if abs(a_ref) >= 1e-9 * A:  # resolved in FP64 (fast modes decay by up to e^-73)
            lin.append(abs(g_ref / linear.shear_gamma("5", k, np.arctan2(ky, kx),
                                                       F.nu_to_s(nu), 1.5) - 1.0))
        B = TOL32 * A
        if abs(a_ref) >= 10 * B and g_ref * steps > 0:
            bound = 2 * np.sqrt(2) * B / (abs(a_ref) * g_ref * steps)
            rates.append(abs(g_gpu / g_ref - 1.0) / bound)
            assert rates[-1] <= 1.0, (i, L, nu)
    print(json.dumps({"lattices": len(lats), "sampled": len(sample), "max_err_over_A": worst,
                      "rates_checked": len(rates), "max_rate_err_over_bound": max(rates),
                      "linear_compared": len(lin),
                      "oracle_vs_linear_median_max": [float(np.median(lin)), max(lin)]}))
