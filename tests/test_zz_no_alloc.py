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


def test_static_reduce_after_a_larger_call(lattice):
    """Every call shares the library's partial-sum array and it keeps the
    last call's contents: a small lattice reduced after a large one (which
    filled all 1024 blocks' partials) must read only its own partials."""
    import torch
    from paper_1803_00437_gb300 import fdlbm as F, inputs
    big = [torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda()
           for a in inputs.random_fields(640, 512, 0.3, seed=23, rho_amp=0.5)]
    small_np = [np.asarray(a, dtype=np.float64)
                for a in inputs.random_fields(40, 40, 0.02, seed=24, rho_amp=0.01)]
    small = [torch.from_numpy(a.astype(np.float32)).cuda() for a in small_np]
    d, ux, uy = (a.astype(np.float32).astype(np.float64) for a in small_np)
    rho = 1.0 + d
    expect = {"mass": [d.sum()], "momentum": [(rho * ux).sum(), (rho * uy).sum()],
              "energy": [(0.5 * rho * (ux ** 2 + uy ** 2)).sum()],
              "maxabs": [np.hypot(ux, uy).max(), np.abs(d).max()]}
    mags = {"mass": np.abs(d).sum(), "momentum": (rho * (np.abs(ux) + np.abs(uy))).sum(),
            "energy": expect["energy"][0], "maxabs": 0.0}
    for what, ref in expect.items():
        F.reduce_fields_static(*big, what)  # 640 x 512 nodes fill every block
        out = F.reduce_fields_static(*small, what).cpu().numpy()
        torch.cuda.synchronize()
        assert out[3] == 0.0
        assert _same(out[:len(ref)], np.array(ref), mags[what]), (what, out, ref)


def test_static_reduce_rejects_memory_off_the_device(lattice):
    """Pointers that are not memory of the current device (here page-locked
    host memory) are rejected before anything is enqueued."""
    import ctypes
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    lib = F.load_library()
    lat, fields, _ = lattice
    host = torch.zeros(264 * 200, dtype=torch.float32).pin_memory()
    dev = [ctypes.c_void_p(t.data_ptr()) for t in fields]
    hp = ctypes.c_void_p(host.data_ptr())
    out_dev = torch.zeros(4, dtype=torch.float64, device=fields[0].device)
    od = ctypes.c_void_p(out_dev.data_ptr())
    assert lib.fdlbm_reduce_fields_static(hp, dev[1], dev[2], 264, 200, 0, None, od,
                                          None) == F.ERR_INVALID
    out_host = torch.zeros(4, dtype=torch.float64).pin_memory()
    assert lib.fdlbm_reduce_fields_static(*dev, 264, 200, 0, None,
                                          ctypes.c_void_p(out_host.data_ptr()),
                                          None) == F.ERR_INVALID
    torch.cuda.synchronize()
    assert np.all(out_host.numpy() == 0.0) and np.all(out_dev.cpu().numpy() == 0.0)
