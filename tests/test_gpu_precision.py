"""Reduced-precision storage (FP16 / BF16 of rho - 1, ux, uy with FP32
arithmetic) against the FP64 oracle, on a 512 x 512 periodic slice of the
precision workload (32 seeded transverse modes of amplitude A = 1e-3 each,
nu = 0.01, five-point stencil, 1000 steps).

Reported per storage type: max and RMS of |field - oracle| over the lattice
(relative to A and to the field amplitude max|u|) and the relative error of
each mode's decay rate (FP64 mode projections on the device).

Bounds, from the arithmetic: each step rebuilds u from the stored fields and
changes it by only ~nu k^2 ~ 1e-4 of its value.
  FP32 (2^-24): 1e-5 of A, the FP32 target.
  FP16 (2^-11 spacing): the stored value moves by less than a spacing per
       step, so errors accumulate like a random walk of half-spacings:
       ~ sqrt(n) 2^-12 |u| ~ 8e-3 |u| after 1000 steps; bound 1e-2 of the
       field amplitude pointwise (that walk's scale, rounded up) and 1 % on
       decay rates.
  BF16 (2^-8 spacing): the per-step change is below half a spacing, so the
       decay is rounded away; the storage cannot hold this state and is only
       checked to stay finite and bounded (recorded, not a target).
  I16 (fixed point, range 1.25 max|u(0)|, spacing range / 32767 ~ 3.8e-5 of
       the field amplitude): the random walk of half-spacings gives
       ~ sqrt(n) 1.9e-5 ~ 6e-4 of the field amplitude; asserted at the
       reduced-storage target, 2e-3 of the field amplitude pointwise and
       2e-3 of A in RMS, and 5e-3 on decay rates.
FP16 and BF16 do not meet the 2e-3 target; I16 does."""
import json
import os

import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import as_f32, oracle_run

pytestmark = pytest.mark.gpu

N, STEPS, AMP = 512, 1000, 1e-3
# (max error / A, max error / field amplitude, decay-rate error)
BOUNDS = {"f32": (1e-5, None, 1e-5), "f16": (None, 1e-2, 1e-2), "bf16": (None, 0.5, None),
          "i16": (None, 2e-3, 5e-3)}
# the reduced-storage target on the RMS error, as a fraction of A
RMS_TARGET = {"i16": 2e-3}
RANGE_OVER_FIELD = 1.25  # I16 storage range, relative to the initial max |u|


@pytest.fixture(scope="module")
def reference(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build, fdlbm as F
    build.build()
    modes = inputs.random_modes(N, N, 32, AMP, seed=inputs.seed_for(3))
    f = as_f32(inputs.transverse_modes(N, N, modes))
    cfg = F.LatticeConfig(N, N, "fd5", s_xx=F.nu_to_s(0.01), s_e=1.5)
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle_run(oracle, cfg, f, STEPS)
    return modes, f, ref


def _mode_amp(ux, uy, md):
    kx, ky = 2 * np.pi * md.m / N, 2 * np.pi * md.n / N
    k = np.hypot(kx, ky)
    X, Y = np.meshgrid(np.arange(N), np.arange(N))
    ut = (-ky * ux + kx * uy) / k
    return (ut * np.exp(-1j * (kx * X + ky * Y))).mean()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "i16"])
def test_storage_error_vs_fp64_oracle(reference, storage):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    modes, f, ref = reference
    field0 = max(float(np.abs(f[1]).max()), float(np.abs(f[2]).max()))
    cfg = F.LatticeConfig(N, N, "fd5", s_xx=F.nu_to_s(0.01), s_e=1.5, storage=storage,
                          storage_range=RANGE_OVER_FIELD * field0 if storage == "i16" else 0.0)
    lat = F.Lattice(cfg)
    lat.init(*[torch.from_numpy(a).cuda() for a in f])
    # rates measured from the device's FP64 mode projections at t = 0 and t = STEPS
    a0 = [complex(*lat.reduce("mode", (md.m, md.n))) for md in modes]
    lat.step(STEPS)
    a1 = [complex(*lat.reduce("mode", (md.m, md.n))) for md in modes]
    got = [t.cpu().numpy().astype(np.float64) for t in lat.moments()]
    err = np.stack([np.abs(g - r) for g, r in zip(got, ref)])
    emax, erms = float(err.max()) / AMP, float(np.sqrt((err[1:] ** 2).mean())) / AMP
    rel_rate = []
    for md, b0, b1 in zip(modes, a0, a1):
        r_ref = _mode_amp(ref[1], ref[2], md)
        r0 = _mode_amp(f[1].astype(np.float64), f[2].astype(np.float64), md)
        g_ref = -np.log(abs(r_ref / r0)) / STEPS
        g_gpu = -np.log(abs(b1 / b0)) / STEPS
        rel_rate.append(abs(g_gpu / g_ref - 1.0))
    field = max(float(np.abs(ref[1]).max()), float(np.abs(ref[2]).max()))
    efield = emax * AMP / field
    print(json.dumps({"storage": storage, "max_err_over_A": emax, "rms_err_over_A": erms,
                      "max_err_over_field": efield, "max_rel_decay_rate_err": max(rel_rate)}))
    assert np.all(np.isfinite(err))
    b_a, b_field, b_rate = BOUNDS[storage]
    if b_a is not None:
        assert emax <= b_a, emax
    if b_field is not None:
        assert efield <= b_field, efield
    if b_rate is not None:
        assert max(rel_rate) <= b_rate, max(rel_rate)
    if storage in RMS_TARGET:
        assert erms <= RMS_TARGET[storage], erms
    lat.sync()  # no saturated store (FDLBM_ERR_RANGE would raise)
