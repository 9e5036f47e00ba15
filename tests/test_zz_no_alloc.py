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


def _magnitude(fields, what, mode):
    """Sum of the magnitudes of the summed terms (the scale of a sum's
    rounding error, whatever the cancellation in the result)."""
    d, ux, uy = (t.cpu().numpy().astype(np.float64) for t in fields)
    rho = 1.0 + d
    if what == "mass":
        return np.abs(d).sum()
    if what == "momentum":
        return (rho * (np.abs(ux) + np.abs(uy))).sum()
    if what == "energy":
        return (0.5 * rho * (ux ** 2 + uy ** 2)).sum()
    if what == "mode":
        return np.hypot(ux, uy).mean()
    return 0.0


def _same(static, ref, magnitude):
    # Both sums carry at least 48 significant bits per partial (FP64 terms,
    # or compensated FP32 chunks added in FP64) and differ in order only:
    # agreement to 1e-13 of the summed magnitudes (2^-44 ~ 5.7e-14), exact
    # for the maxima.
    return np.all(np.abs(static - ref) <= 1e-13 * magnitude + 1e-15)


@pytest.mark.parametrize("what", ["mass", "momentum", "energy", "mode", "maxabs"])
def test_static_reduce_matches_workspace_reduce_twice(lattice, what):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    lat, fields, mode = lattice
    args = (mode.m, mode.n) if what == "mode" else None
    ref = lat.reduce(what, args)
    mag = _magnitude(fields, what, mode)
    for _ in range(2):  # the second call reuses the array left by the first
        out = F.reduce_fields_static(*fields, what, args).cpu().numpy()
        torch.cuda.synchronize()
        assert out[3] == 0.0
        assert _same(out[:len(ref)], ref, mag), (what, out, ref, mag)


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
