"""Failure detection on the GPU without a fault: a bounded device wait is
made to run out (a barrier whose arrival nothing provides), the kernel
records FDLBM_ERR_TIMEOUT in the handle's status word and returns, and the
host reads it at the next synchronisation -- the same path a step kernel
takes when a bulk copy does not land in time.  The context stays usable:
the lattice keeps stepping and matches a fresh run afterwards."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import as_f32, gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build
    build.build()


def test_expired_wait_is_reported_and_cleared():
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    f = as_f32(inputs.random_fields(256, 40, 0.01, seed=5, rho_amp=0.002))
    cfg = F.LatticeConfig(256, 40, "fd5", s_xx=F.nu_to_s(0.02), s_e=1.5)
    lat = F.Lattice(cfg)
    lat.init(*[torch.from_numpy(a).cuda() for a in f])
    lat.step(3)
    lat.selftest_wait_timeout(1000)
    with pytest.raises(F.FdlbmError) as ei:
        lat.sync()
    assert ei.value.status == F.ERR_TIMEOUT
    lat.sync()  # reported once, then cleared
    # through a reduction as well
    lat.selftest_wait_timeout(1000)
    with pytest.raises(F.FdlbmError) as ei:
        lat.reduce("mass")
    assert ei.value.status == F.ERR_TIMEOUT
    assert np.isfinite(lat.reduce("mass")[0])
    # the device is still usable and the state unaffected
    lat.step(4)
    got = [t.cpu().numpy().astype(np.float64) for t in lat.moments()]
    lat.sync()
    ref, _ = gpu_run(cfg, f, 7)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    with pytest.raises(F.FdlbmError):
        lat.selftest_wait_timeout(-1)
