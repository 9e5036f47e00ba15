"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function that include/fdlbm.h declares; its host-only entry points
validate parameters."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdlbm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_00437_gb300 import build, fdlbm
    build.build()
    return fdlbm.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("fdlbm.h") + _declared("fdlbm_walls.h") + _declared("fdlbm_populations.h")
    assert len(names) >= 17 and "fdlbm_set_walls" in names
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_size_validates(lib):
    from paper_1803_00437_gb300 import fdlbm as F
    ok = F.LatticeConfig(64, 48, "fd5")
    n = F.workspace_size(ok)
    # two FP32 states of 3 planes with 256-byte row pitch, plus staging
    assert n >= 2 * 3 * 64 * 48 * 4 + 3 * 64 * 48 * 4
    bad = [F.LatticeConfig(0, 4), F.LatticeConfig(4, 4, s_xx=2.0), F.LatticeConfig(4, 4, s_e=0.0),
           F.LatticeConfig(4, 4, "mrt", storage="f16"),
           F.LatticeConfig(4, 1, boundary="walls_y"),
           F.LatticeConfig(4, 4, "mrt", boundary="walls_y", wall_xi=0.3),
           F.LatticeConfig(4, 4, boundary="walls_y", wall_xi=0.0),
           F.LatticeConfig(256, 64, "fd9", flags=F.FLAG_STREAM)]
    for cfg in bad:
        assert F.workspace_size(cfg) == 0, cfg
    f32 = F.workspace_size(F.LatticeConfig(512, 48, "fd5"))
    f16 = F.workspace_size(F.LatticeConfig(512, 48, "fd5", storage="f16"))
    assert f32 - f16 == 2 * 3 * 512 * 48 * 2
    mrt = F.workspace_size(F.LatticeConfig(64, 48, "mrt"))
    assert mrt > n
    # nine points: same state as the other FD-LBM stencils, walls and force allowed
    assert F.workspace_size(F.LatticeConfig(64, 48, "fd9")) == n
    assert F.workspace_size(F.LatticeConfig(64, 48, "fd9", boundary="walls_y", wall_xi=0.5,
                                            force=(1e-5, 0.0))) == n


def test_status_strings_and_null_handles(lib):
    from paper_1803_00437_gb300 import fdlbm as F
    assert F.status_string(0) == "FDLBM_OK"
    assert F.status_string(-5) == "FDLBM_ERR_DIVERGED"
    assert lib.fdlbm_step(None, 1) == F.ERR_INVALID
    assert lib.fdlbm_launch_count(None) == -1
    assert lib.fdlbm_batch_set_narrow_strips(None, 1) == F.ERR_INVALID
    assert lib.fdlbm_batch_set_segment_rows(None, 64) == F.ERR_INVALID
    assert lib.fdlbm_create(None, None, 0, None, None) == F.ERR_INVALID
    out = ctypes.c_void_p()
    p = F.LatticeConfig(8, 8).params()
    assert lib.fdlbm_create(ctypes.byref(p), None, 0, None, ctypes.byref(out)) == F.ERR_INVALID


def test_built_for_sm103a():
    """The build passes -gencode arch=compute_103a,code=sm_103a to nvcc."""
    from paper_1803_00437_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_missing_library_raises(tmp_path):
    """The binding has no CPU fallback: without the built library it raises."""
    from paper_1803_00437_gb300 import fdlbm
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.load_library(str(tmp_path / "libfdlbm.so"))


def test_no_gpu_no_lattice():
    """Without a GPU, creating a lattice or a batch fails instead of running
    anywhere else."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1803_00437_gb300 import fdlbm as F
    with pytest.raises((RuntimeError, AssertionError, F.FdlbmError)):
        F.Lattice(F.LatticeConfig(64, 64, "fd5"))
    with pytest.raises((RuntimeError, AssertionError, F.FdlbmError)):
        F.Batch("fd5", max_lattices=4, max_side=64, arena_bytes=1 << 20)


_DECL = re.compile(r"^(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fdlbm_[a-z0-9_]+)\s*\(")


def undocumented(lines):
    """Declarations of fdlbm_* functions not preceded by a comment.  Macros,
    blank lines and continuation lines may sit in between; a declaration may
    share the comment of the one before it when their names agree in their
    first three parts (fdlbm_batch_set_grid after fdlbm_batch_set_segment_rows)."""
    out = []
    for i, ln in enumerate(lines):
        m = _DECL.match(ln)
        if not m or ln.lstrip().startswith(("*", "/*", "#")):
            continue
        name = m.group(1)
        j = i - 1
        while j >= 0:
            prev = lines[j]
            pm = _DECL.match(prev)
            if prev.startswith("#define") or not prev.strip() or (
                    prev.startswith(" ") and prev.rstrip().endswith(");")):
                j -= 1
            elif pm and pm.group(1).split("_")[:3] == name.split("_")[:3]:
                j -= 1
            else:
                break
        if j < 0 or not lines[j].rstrip().endswith("*/"):
            out.append(name)
    return out


@pytest.mark.parametrize("header", ["fdlbm.h", "fdlbm_walls.h", "fdlbm_populations.h"])
def test_every_declaration_is_documented(header):
    """Each entry point of the C ABI follows a comment that states what it
    does."""
    lines = open(os.path.join(ROOT, "include", header)).read().split("\n")
    assert undocumented(lines) == []


def test_mrt_s_q_sentinel(lib):
    """MRT's s_q: FDLBM_S_Q_QUARTIC (0) leaves the rate to the library (the
    quartic condition, Eq. sigsig); other values must lie in (0, 2)."""
    from paper_1803_00437_gb300 import fdlbm as F
    assert F.S_Q_QUARTIC == 0.0
    assert F.workspace_size(F.LatticeConfig(64, 48, "mrt")) > 0  # s_q None -> sentinel
    assert F.workspace_size(F.LatticeConfig(64, 48, "mrt", s_q=0.0)) > 0
    assert F.workspace_size(F.LatticeConfig(64, 48, "mrt", s_q=1.2)) > 0
    for bad in (-0.5, 2.0, 2.5):
        assert F.workspace_size(F.LatticeConfig(64, 48, "mrt", s_q=bad)) == 0, bad


def test_fixed_point_storage_parameters(lib):
    """FDLBM_STORAGE_I16 needs a finite storage_range > 0, is FD-LBM only,
    and stores 2 bytes per field like FP16."""
    from paper_1803_00437_gb300 import fdlbm as F
    f16 = F.workspace_size(F.LatticeConfig(512, 48, "fd5", storage="f16"))
    assert F.workspace_size(F.LatticeConfig(512, 48, "fd5", storage="i16",
                                            storage_range=0.02)) == f16
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        assert F.workspace_size(F.LatticeConfig(512, 48, "fd5", storage="i16",
                                                storage_range=bad)) == 0, bad
    assert F.workspace_size(F.LatticeConfig(64, 48, "mrt", storage="i16",
                                            storage_range=0.02)) == 0
    assert F.status_string(F.ERR_RANGE) == "FDLBM_ERR_RANGE"
