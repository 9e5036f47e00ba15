"""Fixed-point storage (FDLBM_STORAGE_I16): (rho - 1, ux, uy) stored as
int16 q standing for q * storage_range / 32767, FP32 arithmetic.

- The stored values are the inputs rounded to the nearest step of the grid
  (checked against numpy's rounding of the same FP32 products).
- Against the FP64 oracle on a ragged streaming lattice and a channel, the
  error stays within a few grid steps per hundred time steps.
- A value beyond the range saturates at +-range and is reported as
  FDLBM_ERR_RANGE, from the initialisation and from a step (a forced
  channel that accelerates past the range), on both FD-LBM kernels; a
  lattice within its range reports nothing."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import amplitude, as_f32, gpu_run, max_err, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build
    build.build()


def _cfg(nx, ny, scheme, rng, **kw):
    from paper_1803_00437_gb300 import fdlbm as F
    return F.LatticeConfig(nx, ny, scheme, s_xx=F.nu_to_s(0.02), s_e=1.5, storage="i16",
                           storage_range=rng, **kw)


def test_stored_values_are_the_rounded_grid_points():
    f = as_f32(inputs.random_fields(96, 40, 0.02, seed=41, rho_amp=0.01))
    rng = 0.03
    got, _ = gpu_run(_cfg(96, 40, "fd5", rng), f, 0)
    scale = np.float32(rng / 32767.0)
    inv = np.float32(1.0) / scale
    for g, a in zip(got, f):
        q = np.rint((a * inv).astype(np.float32))  # ties to even, as the kernels round
        assert np.array_equal(g, (q.astype(np.float32) * scale).astype(np.float64))


@pytest.mark.parametrize("scheme,shape,flags,walls", [
    ("fd5", (264, 40), 2, False), ("fd3", (100, 37), 1, False), ("fd5", (256, 33), 2, True),
    ("fd5", (70, 30), 1, True)])
def test_fixed_point_against_the_oracle(oracle, scheme, shape, flags, walls):
    """Each step rounds the state to the grid once: after n steps the error
    is a random walk of half-steps, sqrt(n) / 2 spacings, far below 20.  The
    noise start (|u| <= 0.01) reaches 0.022 in places as sound forms, so the
    range is 0.04."""
    nx, ny = shape
    f = as_f32(inputs.random_fields(nx, ny, 0.01, seed=nx * 3 + ny, rho_amp=0.002))
    rng = 0.04
    kw = dict(flags=flags)
    if walls:
        kw.update(boundary="walls_y", wall_xi=0.5, force=(1e-6, 0.0))
    cfg = _cfg(nx, ny, scheme, rng, **kw)
    gpu, lat = gpu_run(cfg, f, 200)
    lat.sync()
    ref = oracle_run(oracle, cfg, f, 200)
    spacing = rng / 32767.0
    assert max_err(gpu, ref, spacing) <= 20.0


@pytest.mark.parametrize("flags", [1, 2])
def test_saturation_is_reported(flags):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    f = as_f32(inputs.random_fields(256, 32, 0.02, seed=42, rho_amp=0.001))
    # initial values beyond the range: clamped and reported by the next sync
    lat = F.Lattice(_cfg(256, 32, "fd5", 0.01, flags=flags))
    lat.init(*[torch.from_numpy(a).cuda() for a in f])
    with pytest.raises(F.FdlbmError) as e:
        lat.sync()
    assert e.value.status == F.ERR_RANGE
    lat.sync()  # the status word was cleared
    got = [t.cpu().numpy() for t in lat.moments()]
    lat.sync()
    top = np.float32(np.float32(0.01 / 32767.0) * 32767)
    assert np.abs(got[1]).max() == top and np.abs(got[0]).max() < 0.0011
    # a forced channel at rest, within its range at first, accelerated past it
    ch = F.Lattice(_cfg(256, 32, "fd5", 2e-3, flags=flags, boundary="walls_y", wall_xi=0.5,
                        force=(1e-5, 0.0)))
    z = torch.zeros((32, 256), dtype=torch.float32, device="cuda")
    ch.init(z, z, z)
    ch.step(20)
    ch.sync()  # u <= 20 F = 2e-4: nothing to report
    ch.step(400)  # u grows towards F H^2 / (8 nu) ~ 0.02 > 2e-3
    with pytest.raises(F.FdlbmError) as e:
        ch.sync()
    assert e.value.status == F.ERR_RANGE


@pytest.mark.parametrize("flags", [1, 2])
def test_step_saturates_symmetrically(flags):
    """Values a step carries past the range are stored as +-32767 steps
    (never -32768) by both FD-LBM kernels: channels driven upward and
    downward past a range of 2e-3 end with max |ux| equal to it."""
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    scale = np.float32(2e-3 / 32767.0)
    top = np.float32(scale * np.float32(32767))
    for fx in (1e-5, -1e-5):
        ch = F.Lattice(_cfg(256, 32, "fd5", 2e-3, flags=flags, boundary="walls_y",
                            wall_xi=0.5, force=(fx, 0.0)))
        z = torch.zeros((32, 256), dtype=torch.float32, device="cuda")
        ch.init(z, z, z)
        ch.step(400)
        with pytest.raises(F.FdlbmError):
            ch.sync()
        ux = ch.moments()[1].cpu().numpy()
        ch.sync()
        assert np.abs(ux).max() == top
        assert (ux.max() if fx > 0 else -ux.min()) == top
        q = np.rint(ux / scale)
        assert np.abs(q).max() <= 32767 and np.array_equal(q.astype(np.float32) * scale, ux)
