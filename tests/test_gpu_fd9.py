"""FD-LBM with the nine-point differences of Sec. 2 (D2Q9 footprint) on the
tiled kernel, against the FP64 oracle: element-wise parity where the stencil
is stable (nu = 0.15), and the linear instability of Sec. 3-a at nu = 0.01,
whose growth per step equals the largest |z| of the step's Fourier symbol
on the lattice's wave vectors."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import amplitude, as_f32, gpu_run, max_err, oracle_run

pytestmark = pytest.mark.gpu

# FP32 parity bound: max |GPU - oracle| over the field amplitude
TOL32 = 1e-5


def _s(nu):
    return 1.0 / (3.0 * nu + 0.5)


def _cfg(nx, ny, scheme="fd9", **kw):
    from paper_1803_00437_gb300 import fdlbm as F
    return F.LatticeConfig(nx, ny, scheme, **kw)


@pytest.mark.parametrize("shape", [(64, 48), (100, 37), (33, 17), (256, 40)])
def test_fd9_parity_periodic(oracle, shape):
    """Random fields (u ~ 0.02, rho - 1 ~ 0.01), 300 steps: several tiles in
    both directions and ragged edges; tolerance 1e-5 of the amplitude."""
    nx, ny = shape
    f = as_f32(inputs.random_fields(nx, ny, 0.02, seed=nx + ny, rho_amp=0.01))
    cfg = _cfg(nx, ny, s_xx=_s(0.15), s_e=1.5)
    gpu, _ = gpu_run(cfg, f, 300)
    ref = oracle_run(oracle, cfg, f, 300)
    assert max_err(gpu, ref, amplitude(f)) <= TOL32


@pytest.mark.parametrize("xi", [0.5, 0.8])
def test_fd9_channel_with_force(oracle, xi):
    """Walls in y (the linear extrapolation closure) and a body force,
    96 x 40 from rest plus a small random field, 500 steps."""
    nx, ny, nu = 96, 40, 0.15
    H = ny - 1 + 2 * xi
    F = 8 * nu * 0.02 / H ** 2
    d, x, y = inputs.random_fields(nx, ny, 0.005, seed=7, rho_amp=0.002)
    f = as_f32((d, x, y))
    cfg = _cfg(nx, ny, s_xx=_s(nu), s_e=1.5, boundary="walls_y", wall_xi=xi, force=(F, 0.0))
    gpu, _ = gpu_run(cfg, f, 500)
    ref = oracle_run(oracle, cfg, f, 500)
    assert max_err(gpu, ref, max(amplitude(f), 0.02)) <= TOL32


def test_fd9_half_storage_close_to_fp32(oracle):
    """FP16 storage of (rho - 1, u) with FP32 arithmetic stays within 2e-3 of
    the amplitude of the FP64 oracle after 300 steps."""
    nx, ny = 64, 48
    f = as_f32(inputs.random_fields(nx, ny, 0.02, seed=3, rho_amp=0.01))
    cfg = _cfg(nx, ny, s_xx=_s(0.15), s_e=1.5, storage="f16")
    gpu, _ = gpu_run(cfg, f, 300)
    ref = oracle_run(oracle, cfg, f, 300)
    assert max_err(gpu, ref, amplitude(f)) <= 2e-3


def _norm(fields):
    return float(np.sqrt(sum((np.asarray(a, np.float64) ** 2).sum() for a in fields)))


@pytest.mark.parametrize("scheme", ["fd9", "fd3", "fd5"])
def test_nine_points_unstable_three_and_five_stable(oracle, scheme):
    """Sec. 3-a at nu = 0.01 on a 16 x 16 periodic lattice seeded with
    random deviations of 1e-8 (linear regime).  Between steps 60 and 80 the
    nine-point state grows by the largest |z| of the symbol H(k) over the
    lattice's wave vectors (1.1954), on the GPU and in the oracle alike; the
    three- and five-point states decay."""
    from oracle import linear
    N, nu = 16, 0.01
    s = _s(nu)
    ks = 2 * np.pi * np.arange(N) / N
    st = {"fd3": 3, "fd5": 5, "fd9": 9}[scheme]
    zmax = max(np.max(np.abs(np.linalg.eigvals(linear.H_fd(st, kx, ky, s, 1.5))))
               for kx in ks for ky in ks)
    f = as_f32(inputs.random_fields(N, N, 1e-8, seed=3, rho_amp=1e-8))
    cfg = _cfg(N, N, scheme, s_xx=s, s_e=1.5)
    g60, lat = gpu_run(cfg, f, 60)
    lat.step(20)
    g80 = [t.cpu().numpy().astype(np.float64) for t in lat.moments()]
    r60 = oracle_run(oracle, cfg, f, 60)
    r80 = oracle_run(oracle, cfg, f, 80)
    rate_gpu = (_norm(g80) / _norm(g60)) ** (1 / 20)
    rate_ref = (_norm(r80) / _norm(r60)) ** (1 / 20)
    print(f"{scheme}: growth per step GPU {rate_gpu:.6f}, oracle {rate_ref:.6f}, "
          f"max |z| {zmax:.6f}")
    if scheme == "fd9":
        assert abs(rate_gpu / zmax - 1) < 1e-3 and abs(rate_ref / zmax - 1) < 1e-3
    else:
        assert zmax <= 1 + 1e-12 and rate_gpu < 1 and rate_ref < 1
