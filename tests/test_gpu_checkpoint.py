"""Checkpoint and resume of FD-LBM lattices.  The scheme keeps only
(rho - 1, ux, uy) per node (Sec. 2), so the fields read by moments() are the
whole state: a lattice started from them continues exactly where the first
one stopped.  Resuming n steps from the checkpoint of step m therefore equals
running m + n steps, bit for bit, for every kernel, stencil and storage type,
and with curved walls (whose virtual nodes are rewritten from the fluid
before every step)."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import as_f32

pytestmark = pytest.mark.gpu


def _run(cfg, fields, n, walls=None):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    lat = F.Lattice(cfg)
    if walls is not None:
        lat.set_walls(walls)
    lat.init(*[torch.from_numpy(np.ascontiguousarray(a)).to(lat.device) for a in fields])
    lat.step(n)
    out = [t.cpu().numpy() for t in lat.moments()]
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("scheme,storage,flags,shape", [
    ("fd5", "f32", 2, (256, 64)),
    ("fd3", "f32", 1, (100, 37)),
    ("fd5", "f16", 2, (256, 64)),
    ("fd5", "bf16", 1, (96, 40)),
    ("lwacm", "f32", 2, (256, 48)),
    ("fd9", "f32", 0, (64, 48)),
    ("fd5", "i16", 2, (256, 64)),
    ("fd3", "i16", 1, (100, 37)),
])
def test_resume_from_moments_is_exact(scheme, storage, flags, shape):
    from paper_1803_00437_gb300 import fdlbm as F
    nx, ny = shape
    cfg = F.LatticeConfig(nx, ny, scheme, s_xx=F.nu_to_s(0.15 if scheme == "fd9" else 0.02),
                          s_e=1.5, storage=storage, flags=flags,
                          storage_range=0.05 if storage == "i16" else 0.0)
    f = as_f32(inputs.random_fields(nx, ny, 0.02, seed=nx + ny, rho_amp=0.01))
    straight = _run(cfg, f, 70)
    checkpoint = _run(cfg, f, 30)
    resumed = _run(cfg, checkpoint, 40)
    for a, b in zip(straight, resumed):
        assert np.array_equal(a, b)


def test_resume_with_curved_walls_is_exact():
    from paper_1803_00437_gb300 import fdlbm as F
    N = 48
    walls = inputs.disk_walls(N, N, 18.0, reach=3)
    f = as_f32(inputs.stokes_disk_mode(N, N, 18.0, 1, 5.1356223, 1e-3))
    cfg = F.LatticeConfig(N, N, "fd5", s_xx=F.nu_to_s(0.05), s_e=1.5)
    straight = _run(cfg, f, 70, walls)
    resumed = _run(cfg, _run(cfg, f, 30, walls), 40, walls)
    for a, b in zip(straight, resumed):
        assert np.array_equal(a, b)


def test_mrt_resume_from_populations_is_exact():
    """The MRT state is its nine populations (fdlbm_get_populations /
    fdlbm_set_populations); resuming from them is exact, with walls and force
    too.  The other schemes refuse the call (their state is the moments)."""
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    for kw in ({}, dict(boundary="walls_y", wall_xi=0.5, force=(1e-6, 0.0))):
        cfg = F.LatticeConfig(96, 40, "mrt", s_xx=F.nu_to_s(0.02), s_e=1.5, **kw)
        f = as_f32(inputs.random_fields(96, 40, 0.02, seed=3, rho_amp=0.01))
        straight = _run(cfg, f, 70)
        lat = F.Lattice(cfg)
        lat.init(*[torch.from_numpy(np.ascontiguousarray(a)).to(lat.device) for a in f])
        lat.step(30)
        pops = lat.populations().clone()
        lat2 = F.Lattice(cfg)
        lat2.set_populations(pops)
        lat2.step(40)
        resumed = [t.cpu().numpy() for t in lat2.moments()]
        for a, b in zip(straight, resumed):
            assert np.array_equal(a, b)
    with pytest.raises(F.FdlbmError) as e:
        F.Lattice(F.LatticeConfig(64, 48, "fd5")).populations()
    assert e.value.status == F.ERR_UNSUPPORTED
