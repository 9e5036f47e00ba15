"""fdlbm_reduce_fields_static: the reductions for callers that cannot
allocate device memory (no handle, no workspace; the partial sums live in a
fixed array inside the library).  Checked through the C ABI against
fdlbm_reduce on the same lattice, on two calls in a row.  Kept in the last
collected test file so that a run stopping at the first failure has run
every other test first."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lattice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build, fdlbm as F, inputs
    build.build()
    lat = F.Lattice(F.LatticeConfig(264, 200, "fd5", s_xx=F.nu_to_s(0.02), s_e=1.5))
    modes = inputs.random_modes(264, 200, 8, 5e-3, seed=21)
    d, ux, uy = inputs.transverse_modes(264, 200, modes)
    d = inputs.random_fields(264, 200, 0.0, seed=22, rho_amp=1e-3)[0]
    lat.init(*[torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda() for a in (d, ux, uy)])
    lat.step(50)
    fields = lat.moments()
    lat.sync()
    return lat, fields, modes[0]


def _same(static, ref):
    # FP64 sums over the same values in another order: rounding only
    return np.allclose(static, ref, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("what", ["mass", "momentum", "energy", "mode", "maxabs"])
def test_static_reduce_matches_workspace_reduce_twice(lattice, what):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    lat, fields, mode = lattice
    args = (mode.m, mode.n) if what == "mode" else None
    ref = lat.reduce(what, args)
    for _ in range(2):  # the second call reuses the array left by the first
        out = F.reduce_fields_static(*fields, what, args).cpu().numpy()
        torch.cuda.synchronize()
        assert out[3] == 0.0
        assert _same(out[:len(ref)], ref), (what, out, ref)


def test_static_reduce_rejects_oversized_and_bad_arguments(lattice):
    import ctypes
    from paper_1803_00437_gb300 import fdlbm as F
    lib = F.load_library()
    lat, fields, _ = lattice
    p = [ctypes.c_void_p(t.data_ptr()) for t in fields]
    out = ctypes.c_void_p(fields[0].data_ptr())  # never written: rejected before any launch
    too_big = (1 << 15) + 1  # (2^15 + 1)^2 > 2^30 nodes
    assert lib.fdlbm_reduce_fields_static(*p, too_big, too_big, 0, None, out, None) == F.ERR_INVALID
    assert lib.fdlbm_reduce_fields_static(*p, 0, 4, 0, None, out, None) == F.ERR_INVALID
    assert lib.fdlbm_reduce_fields_static(*p, 264, 200, 9, None, out, None) == F.ERR_INVALID
    assert lib.fdlbm_reduce_fields_static(*p, 264, 200, 3, None, out, None) == F.ERR_INVALID
