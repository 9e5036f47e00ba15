"""The streaming step's launch plan (fdlbm_stream_plan, host logic, no GPU):
row segments of equal length that cover the lattice, CTA counts, the picks
measured best on GB300, and the documented cost model
    (segment rows + c) (items / resident CTAs + a),
c = 0.5 + 2R (2 for LW-ACM) and a = 0.2, except LW-ACM with FP32 storage
(c = 0.5, a = 0.4)."""
import ctypes
import math

import pytest

from paper_1803_00437_gb300 import fdlbm as F

RESIDENT = 152 * 8  # GB300: 152 SMs x 8 two-warp CTAs at 128 registers


def model_pick(nx, ny, scheme, storage, resident):
    R = {"fd3": 1, "fd5": 2, "lwacm": 0}[scheme]
    near_memory = R == 0 and storage == "f32"
    c = 0.5 if near_memory else (2.0 if R == 0 else 0.5 + 2 * R)
    a = 0.4 if near_memory else 0.2
    strips = math.ceil(math.ceil(nx / 120) / 2)
    best = None
    for n in range(1, (ny + 15) // 16 + 1):
        s = math.ceil(ny / n)
        if math.ceil(ny / s) != n:
            continue
        cost = (s + c) * (strips * n / resident + a)
        if best is None or cost < best[0]:
            best = (cost, s, n)
    return best[1], best[2]


@pytest.mark.parametrize("scheme,storage", [("fd5", "f32"), ("fd3", "f32"), ("lwacm", "f32"),
                                            ("fd5", "f16"), ("lwacm", "bf16"), ("fd5", "i16")])
def test_segments_cover_the_rows_and_follow_the_model(scheme, storage):
    for nx in (256, 264, 1000, 4096, 8192, 12000):
        for ny in (1, 7, 16, 17, 40, 100, 1000, 4096, 8192, 16384):
            for resident in (152, RESIDENT, 2 * RESIDENT):
                p = F.stream_plan(nx, ny, scheme, storage, resident)
                rows, nsegs = p["seg_rows"], p["nsegs"]
                assert rows >= 1 and nsegs >= 1
                assert nsegs * rows >= ny > (nsegs - 1) * rows  # equal segments, none empty
                assert nsegs <= max(1, (ny + 15) // 16)
                assert p["strips"] == math.ceil(math.ceil(nx / 120) / 2)
                assert p["ctas"] == p["strips"] * nsegs
                assert (rows, nsegs) == model_pick(nx, ny, scheme, storage, resident)


def test_picks_measured_on_gb300():
    """8192^2 segment sweeps (GLUPS, CUDA events): FD-5 within 1 % of its best
    at 104-171 segments, LW-ACM best at 512 (16-row) segments; 16384^2 FD-5
    within 1 % at 105-220 segments."""
    p = F.stream_plan(8192, 8192, "fd5", "f32", RESIDENT)
    assert (p["seg_rows"], p["nsegs"], p["ctas"]) == (64, 128, 4480)
    assert 104 <= p["nsegs"] <= 171
    p = F.stream_plan(8192, 8192, "lwacm", "f32", RESIDENT)
    assert (p["seg_rows"], p["nsegs"]) == (16, 512)
    assert 105 <= F.stream_plan(16384, 16384, "fd5", "f32", RESIDENT)["nsegs"] <= 220
    # one wave of long segments, the plan that measured 7 % slower on 8192^2
    assert F.stream_plan(8192, 8192, "fd5", "f32", RESIDENT)["nsegs"] != 34


def test_invalid_arguments():
    lib = F.load_library()
    out = (ctypes.c_int32 * 4)()
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 0, RESIDENT, None) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(8192, 8192, 100, 0, RESIDENT, out) == F.ERR_INVALID  # MRT
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 7, RESIDENT, out) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(0, 8192, 5, 0, RESIDENT, out) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 0, 0, out) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 0, RESIDENT, out) == F.OK
