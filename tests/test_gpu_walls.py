"""Curved walls (Sec. 3-b) on the GPU: the wall table's fill kernel plus
the unchanged FD-LBM step kernels, against the FP64 oracle's closure.

- A disk, element by element at the fluid nodes (tiled kernel at 68^2,
  streaming kernel at 256 x 64), three, five and nine points.
- A straight channel written as a wall table equals the channel path of
  FDLBM_BOUNDARY_WALLS_Y.
- The Stokes modes of a disk of radius 29.9 (Tables 2 and 3): decay rates
  against nu a^2 / R^2 with a the Bessel zeros, at nu_0 = 0.05 and
  1/sqrt(108); the GPU rates equal the oracle's."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import as_f32, gpu_run

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _s(nu):
    return 1.0 / (3.0 * nu + 0.5)


def _lattice(nx, ny, scheme, walls, fields32, **kw):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    lat = F.Lattice(F.LatticeConfig(nx, ny, scheme, **kw))
    lat.set_walls(walls)
    lat.init(*[torch.from_numpy(np.ascontiguousarray(a)).to(lat.device) for a in fields32])
    return lat


def _moments(lat):
    return [t.cpu().numpy().astype(np.float64) for t in lat.moments()]


def _disk_fields(N, M, radius, seed):
    """A Stokes mode plus seeded noise, both only in the fluid."""
    walls = inputs.disk_walls(N, M, radius, reach=3)
    fluid = walls.kind == 0
    d, ux, uy = inputs.stokes_disk_mode(N, M, radius, 1, 5.1356223, 0.02)
    nd, nx_, ny_ = inputs.random_fields(N, M, 0.002, seed=seed, rho_amp=0.002)
    return walls, fluid, as_f32((np.where(fluid, nd, 0.0), np.where(fluid, ux + nx_, 0.0),
                                 np.where(fluid, uy + ny_, 0.0)))


@pytest.mark.parametrize("scheme,nu", [("fd3", 0.05), ("fd5", 0.05), ("fd9", 0.15)])
@pytest.mark.parametrize("shape", [(68, 68, 29.9, 0), (256, 64, 25.0, 2)])
def test_disk_parity_with_oracle(oracle, scheme, nu, shape):
    """300 steps; fluid nodes within 1e-5 of the amplitude (u ~ 0.02)."""
    from oracle import ref
    nx, ny, radius, flags = shape
    if scheme == "fd9":
        flags = 0  # nine points run on the tiled kernel only
    walls, fluid, f = _disk_fields(nx, ny, radius, seed=nx + ny)
    lat = _lattice(nx, ny, scheme, walls, f, s_xx=_s(nu), s_e=1.5, flags=flags)
    lat.step(300)
    gpu = _moments(lat)
    st = {"fd3": 3, "fd5": 5, "fd9": 9}[scheme]
    r, x, y = ref.fd_run_walls(ref.params(nx, ny, st, _s(nu), 1.5), walls,
                               1 + f[0].astype(np.float64), f[1], f[2], 300)
    amp = max(np.abs(f[1]).max(), np.abs(f[2]).max())
    err = max(np.abs(g[fluid] - o[fluid]).max() for g, o in zip(gpu, (r - 1, x, y)))
    print(f"{scheme} {nx}x{ny}: max error / amplitude {err / amp:.2e}")
    assert err <= TOL32 * amp


@pytest.mark.parametrize("flags", [1, 2])
def test_channel_table_equals_channel_path(flags):
    """256 x 40 channel with force, xi = 0.3: the periodic lattice of 46
    rows with the channel's wall table against FDLBM_BOUNDARY_WALLS_Y, on
    the tiled (flags 1) and the streaming (flags 2) kernel, 500 steps."""
    from paper_1803_00437_gb300 import fdlbm as F
    nx, nyf, reach, xi, nu = 256, 40, 3, 0.3, 0.05
    F_ = 8 * nu * 0.02 / (nyf - 1 + 2 * xi) ** 2
    d, ux, uy = inputs.random_fields(nx, nyf, 0.005, seed=9, rho_amp=0.002)
    f = as_f32((d, ux, uy))
    native, _ = gpu_run(F.LatticeConfig(nx, nyf, "fd5", s_xx=_s(nu), s_e=1.5,
                                        boundary="walls_y", wall_xi=xi, force=(F_, 0.0),
                                        flags=flags), f, 500)
    pad = [np.vstack([np.zeros((reach, nx), np.float32), a, np.zeros((reach, nx), np.float32)])
           for a in f]
    lat = _lattice(nx, nyf + 2 * reach, "fd5", inputs.channel_walls(nx, nyf, xi, reach), pad,
                   s_xx=_s(nu), s_e=1.5, force=(F_, 0.0), flags=flags)
    lat.step(500)
    tab = _moments(lat)
    amp = max(np.abs(f[1]).max(), 0.02)
    err = max(np.abs(t[reach:reach + nyf] - n).max() for t, n in zip(tab, native))
    print(f"flags {flags}: table vs channel path {err / amp:.2e}")
    assert err <= TOL32 * amp


def _disk_modes():
    from scipy.special import jn_zeros
    return ([("singlet", l + 1, 0, a) for l, a in enumerate(jn_zeros(1, 6))] +
            [("doublet", m, m, jn_zeros(m + 1, 1)[0]) for m in range(1, 12)])


def _gpu_disk_rate(scheme, nu, m, a, N=68, radius=29.9):
    walls = inputs.disk_walls(N, N, radius, reach=3)
    fluid = walls.kind == 0
    d, ux0, uy0 = inputs.stokes_disk_mode(N, N, radius, m, a, 1e-4)
    lat = _lattice(N, N, scheme, walls, as_f32((d, ux0, uy0)), s_xx=_s(nu), s_e=1.5)
    n = int(2.0 / (nu * a * a / radius ** 2))
    lat.step(n // 2)
    _, x, y = _moments(lat)
    a1 = ((x * ux0 + y * uy0)[fluid]).sum()
    lat.step(n - n // 2)
    _, x, y = _moments(lat)
    a2 = ((x * ux0 + y * uy0)[fluid]).sum()
    return -np.log(a2 / a1) / (n - n // 2) * radius ** 2 / nu


@pytest.mark.parametrize("nu", [0.05, 1 / np.sqrt(108)])
def test_tables_2_and_3_stokes_modes_in_a_disk(oracle, nu):
    """Relative error of the measured rate against a^2 for the six singlets
    and eleven doublets of Tables 2 (nu_0 = 0.05) and 3 (nu_0 = 1/sqrt 108):
    five points within 0.004 (the largest printed for that stencil is 0.004),
    three points above, growing along the singlets (as printed); both
    against the printed columns (tests/golden/tables2_3_stokes_disk.txt)
    within the spread of this reading of the closure.  The rates
    of the first singlet and doublet equal the oracle's (the same measurement
    on the FP64 oracle) to 1e-4."""
    import test_oracle_walls as W
    rows = []
    for kind, l, m, a in _disk_modes():
        e3 = _gpu_disk_rate("fd3", nu, m, a) / a ** 2 - 1
        e5 = _gpu_disk_rate("fd5", nu, m, a) / a ** 2 - 1
        rows.append((kind, l, a * a, e3, e5))
    print(f"nu_0 = {nu:.5f}: kind, l, a^2, error three points, error five points")
    for r in rows:
        print(f"  {r[0]} {r[1]:2d} {r[2]:10.5f} {r[3]:+.5f} {r[4]:+.5f}")
    assert max(abs(r[4]) for r in rows) <= 0.004
    assert min(r[3] for r in rows) > 0.0
    singlets = [r[3] for r in rows if r[0] == "singlet"]
    assert all(b > a for a, b in zip(singlets, singlets[1:]))
    # against the printed columns.  Sec. 3-b only sketches the closure and
    # does not give the disk's centre, so these bounds are not derived: they
    # record how closely this reading follows the printed errors (the oracle
    # gives three points within a factor 0.83 .. 1.30 of them and five points
    # within 0.0027), not the printed digits
    table = 2 if abs(nu - 0.05) < 1e-9 else 3
    printed = {(k, l): (e3, e5) for t, k, l, _, e3, e5 in W.printed_tables_2_3() if t == table}
    for kind, l, _, e3, e5 in rows:
        p3, p5 = printed[(kind, l)]
        assert 0.75 <= e3 / p3 <= 1.35, (kind, l, e3, p3)
        assert abs(e5 - p5) <= 0.003, (kind, l, e5, p5)
    for kind, l, m, a in (_disk_modes()[0], _disk_modes()[6]):
        g = _gpu_disk_rate("fd5", nu, m, a)
        o = W.disk_rate(oracle, 5, nu, m, a)
        assert abs(g / o - 1) <= 1e-4, (kind, l, g, o)


def test_half_storage_with_walls(oracle):
    """FP16 storage of (rho - 1, u), FP32 arithmetic: fluid nodes within
    2e-3 of the amplitude of the FP64 oracle after 300 steps."""
    from oracle import ref
    walls, fluid, f = _disk_fields(68, 68, 29.9, seed=5)
    lat = _lattice(68, 68, "fd5", walls, f, s_xx=_s(0.05), s_e=1.5, storage="f16")
    lat.step(300)
    gpu = _moments(lat)
    r, x, y = ref.fd_run_walls(ref.params(68, 68, 5, _s(0.05), 1.5), walls,
                               1 + f[0].astype(np.float64), f[1], f[2], 300)
    amp = max(np.abs(f[1]).max(), np.abs(f[2]).max())
    err = max(np.abs(g[fluid] - o[fluid]).max() for g, o in zip(gpu, (r - 1, x, y)))
    assert err <= 2e-3 * amp


def test_set_walls_rejects_inconsistent_tables():
    """fdlbm_set_walls validates the geometry on the host and leaves the
    lattice without walls when it refuses one."""
    import dataclasses
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    N = 40
    good = inputs.disk_walls(N, N, 15.0, reach=3)
    lat = F.Lattice(F.LatticeConfig(N, N, "fd5"))
    bad_cases = [
        dataclasses.replace(good, kind=np.where(good.kind == 2, 3, good.kind).astype(np.uint8)),
        dataclasses.replace(good, node=good.node[1:], link=good.link[1:], xi=good.xi[1:]),
        dataclasses.replace(good, link=np.where(np.arange(good.link.size) == 0, 9,
                                                good.link).astype(np.int8)),
        dataclasses.replace(good, xi=np.where(np.arange(good.xi.size) == 0, 0.0, good.xi)),
        inputs.disk_walls(N, N, 15.0, reach=2),  # five points read three nodes deep
    ]
    for w in bad_cases:
        with pytest.raises(F.FdlbmError) as e:
            lat.set_walls(w)
        assert e.value.status == F.ERR_INVALID
    lat.set_walls(good)
    lat.set_walls(None)
    for scheme in ("mrt", "lwacm"):
        with pytest.raises(F.FdlbmError) as e:
            F.Lattice(F.LatticeConfig(N, N, scheme)).set_walls(good)
        assert e.value.status == F.ERR_UNSUPPORTED
    with pytest.raises(F.FdlbmError):
        F.Lattice(F.LatticeConfig(N, N, "fd5", boundary="walls_y", wall_xi=0.5)).set_walls(good)
    torch.cuda.synchronize()
