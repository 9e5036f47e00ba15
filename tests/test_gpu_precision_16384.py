"""Precision sweep at full size: 16384 x 16384 periodic FD-LBM five points,
32 seeded transverse modes of amplitude A = 1e-3, nu = 0.01, s_e = 1.5,
5000 steps, FP32 arithmetic with FP32 / FP16 / BF16 storage of (rho - 1, ux,
uy), in the launch configuration the benchmark uses.

The 32 modes are drawn for a 512 x 512 tile (|m'|, |n'| <= 32, as in the
512^2 precision workload) and the lattice is that tile repeated 32 x 32 times,
i.e. wave numbers 32 (m', n') on 16384^2.  The FP32 inputs are tiled exactly,
and the step is translation invariant, so every one of the 1024 slices of
512 x 512 must follow the oracle's 512^2 run: each slice is compared with it
element by element (all 268M nodes), and each mode's decay rate (FP64
projections of the field folded onto one tile) with the oracle's.

Bounds, from the arithmetic (unit roundoff u_s of the storage; the stored
values are rounded once per step and each step changes them by only
~nu k^2 <= 2e-3 of their value, so rounding errors add up like a random walk
of n steps), on max |u_gpu - u_oracle| over all nodes, as a fraction of the
initial field amplitude:
  FP32 (u_s = 2^-24): sqrt(n) u_s ~ 4e-6; bound B = 1e-5 (the FP32 target).
  FP16 (u_s = 2^-11): sqrt(n) u_s ~ 3.5e-2; bound B = 5e-2.
  BF16 (u_s = 2^-8): the per-step change is below the storage resolution,
        so the decay is rounded away; checked to stay finite and bounded
        only (recorded, not a target).
  I16 (fixed point, range 1.25 of the initial field amplitude, spacing
        3.8e-5 of it): sqrt(n) half-spacings ~ 1.4e-3; asserted at the
        reduced-storage target B = 2e-3.
FP16 and BF16 do not meet the 2e-3 target; I16 does.
Decay rates follow from the field bound: a mode projection is an average
of (-ky ux + kx uy)/k against a unit phase, so its error is at most sqrt(2) B
(absolute); for a mode whose oracle amplitude after n steps is a_n >= 10 B,
|log(a_gpu / a_n)| <= 2 sqrt(2) B / a_n, i.e. a relative rate error of at most
2 sqrt(2) B / (a_n Gamma n).  Modes that decayed below 10 B (all of them under
16-bit storage) are reported, not asserted: their rates are not resolved by
the storage."""
import json
import os

import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import as_f32, oracle_run

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TILE, REP, STEPS, AMP, NU = 512, 32, 5000, 1e-3, 0.01
N = TILE * REP
# field error bound B / initial field amplitude
BOUNDS = {"f32": 1e-5, "f16": 5e-2, "bf16": 1.0, "i16": 2e-3}
RANGE_OVER_FIELD = 1.25  # I16 storage range, relative to the initial max |u|


def _fold(t):
    """Sum of a 16384^2 device field over its 32 x 32 tiles, FP64, on the host."""
    import torch
    return t.view(REP, TILE, REP, TILE).to(torch.float64).sum(dim=(0, 2)).cpu().numpy() / REP ** 2


def _mode_amp(ux, uy, md):
    kx, ky = 2 * np.pi * md.m / TILE, 2 * np.pi * md.n / TILE
    k = np.hypot(kx, ky)
    X, Y = np.meshgrid(np.arange(TILE), np.arange(TILE))
    ut = (-ky * ux + kx * uy) / k
    return (ut * np.exp(-1j * (kx * X + ky * Y))).mean()


@pytest.fixture(scope="module")
def tile_reference(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build, fdlbm as F
    build.build()
    modes = inputs.random_modes(TILE, TILE, 32, AMP, seed=inputs.seed_for(3))
    f = as_f32(inputs.transverse_modes(TILE, TILE, modes))
    cfg = F.LatticeConfig(TILE, TILE, "fd5", s_xx=F.nu_to_s(NU), s_e=1.5)
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle_run(oracle, cfg, f, STEPS)
    return modes, f, ref


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "i16"])
def test_16384_slices_and_decay_vs_oracle(tile_reference, storage):
    import torch
    from oracle import linear
    from paper_1803_00437_gb300 import fdlbm as F
    modes, f, ref = tile_reference
    field0 = max(float(np.abs(f[1]).max()), float(np.abs(f[2]).max()))
    cfg = F.LatticeConfig(N, N, "fd5", s_xx=F.nu_to_s(NU), s_e=1.5, storage=storage,
                          storage_range=RANGE_OVER_FIELD * field0 if storage == "i16" else 0.0)
    lat = F.Lattice(cfg)
    dev = [torch.from_numpy(a).cuda().repeat(REP, REP) for a in f]
    lat.init(*dev)
    del dev
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(STEPS)
    e1.record(stream)
    lat.sync()
    torch.cuda.synchronize()
    mlups = N * N * STEPS / (e0.elapsed_time(e1) / 1e3) / 1e6
    out = lat.moments()
    lat.sync()
    lat.close()
    del lat
    amp0 = max(float(np.abs(f[1]).max()), float(np.abs(f[2]).max()))
    emax, slice_max, erms2 = 0.0, [], 0.0
    for g, r in zip(out, ref):
        rt = torch.from_numpy(r).cuda()
        d = (g.view(REP, TILE, REP, TILE).to(torch.float64) - rt[None, :, None, :]).abs()
        per_slice = d.amax(dim=(1, 3))
        slice_max.append(per_slice)
        emax = max(emax, float(per_slice.max()))
        erms2 += float((d * d).mean())
        del d, rt
    per_slice = torch.stack(slice_max).amax(dim=0)
    folded = [_fold(t) for t in out]
    del out
    torch.cuda.empty_cache()
    assert all(np.all(np.isfinite(x)) for x in folded)
    B = BOUNDS[storage] * amp0
    rel_rate, rel_lin, checked = [], [], []
    f0 = [a.astype(np.float64) for a in f]
    for md in modes:
        a0 = _mode_amp(f0[1], f0[2], md)
        a_ref = _mode_amp(ref[1], ref[2], md)
        g_gpu = -np.log(abs(_mode_amp(folded[1], folded[2], md) / a0)) / STEPS
        g_ref = -np.log(abs(a_ref / a0)) / STEPS
        k = np.hypot(md.m, md.n) * 2 * np.pi / TILE
        g_lin = linear.shear_gamma("5", k, np.arctan2(md.n, md.m), F.nu_to_s(NU), 1.5)
        err = abs(g_gpu / g_ref - 1.0)
        rel_rate.append(err)
        rel_lin.append(abs(g_ref / g_lin - 1.0))
        if abs(a_ref) >= 10 * B:
            checked.append((err, 2 * np.sqrt(2) * B / (abs(a_ref) * g_ref * STEPS)))
    rec = {"storage": storage, "lattice": N, "steps": STEPS, "mlups": round(mlups, 1),
           "max_err_over_amp0": emax / amp0, "rms_err_over_amp0": float(np.sqrt(erms2 / 3)) / amp0,
           "slice_max_spread": [float(per_slice.min()) / amp0, float(per_slice.max()) / amp0],
           "decay_rate_rel_err_median_max": [float(np.median(rel_rate)), max(rel_rate)],
           "modes_rate_checked": len(checked),
           "max_rate_err_over_bound": max((e / b for e, b in checked), default=None),
           "oracle_vs_linear_theory_median_max": [float(np.median(rel_lin)), max(rel_lin)]}
    print(json.dumps(rec))
    assert emax <= B, rec
    for e, b in checked:
        assert e <= b, rec
