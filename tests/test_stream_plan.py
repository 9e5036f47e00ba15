"""The streaming step's launch plan (fdlbm_stream_plan, host logic, no GPU):
row segments that cover the lattice, CTA counts, the documented cost model
and its picks measured on GB300, and the candidate list the autotuner times.

Model (row-times of one resident CTA): equal segments of s rows cost
    (s + c) (items / resident + a),
c = 0.5 + 2R (2 for LW-ACM) and a = 0.2, except LW-ACM with FP32 storage
(c = 0.5, a = 0.4).  The finite-difference steps may instead take nb long
segments of B rows per strip, nb = k resident / strips for k = 1, 2, 3, and
the rest in segments of t rows (t in 16, 24, 32, 48, 64), costing
    strips (nb (B + c) + nt (t + c)) / resident + a (t + c),
with B the longest multiple of 8 (at least 2 t) whose tail work per resident
CTA, strips nt (t + c) / resident, is at least 0.22 (B + c)."""
import ctypes
import math

import pytest

from paper_1803_00437_gb300 import fdlbm as F

RESIDENT = 152 * 8  # GB300: 152 SMs x 8 two-warp CTAs at 128 registers
TAILS = (16, 24, 32, 48, 64)


def model(nx, scheme, storage, resident):
    R = {"fd3": 1, "fd5": 2, "lwacm": 0}[scheme]
    near_memory = R == 0 and storage == "f32"
    c = 0.5 if near_memory else (2.0 if R == 0 else 0.5 + 2 * R)
    a = 0.4 if near_memory else 0.2
    strips = math.ceil(math.ceil(nx / 120) / 2)
    return R, c, a, strips


def model_pick(nx, ny, scheme, storage, resident):
    """(seg_rows, nsegs, tail_rows, ntail) of the model's plan."""
    R, c, a, P = model(nx, scheme, storage, resident)
    best = None
    for n in range(1, (ny + 15) // 16 + 1):
        s = math.ceil(ny / n)
        if math.ceil(ny / s) != n:
            continue
        cost = (s + c) * (P * n / resident + a)
        if best is None or cost < best[0]:
            best = (cost, (s, n, s, 0))
    if R > 0:
        for k in (1, 2, 3):
            nb = int(k * resident / P)
            if nb < 1:
                continue
            for t in TAILS:
                if nb * 2 * t >= ny:
                    continue
                B = ((ny - t) // nb) & ~7
                while B >= 2 * t:
                    nt = math.ceil((ny - nb * B) / t)
                    if P * nt * (t + c) / resident >= 0.22 * (B + c):
                        break
                    B -= 8
                if B < 2 * t:
                    continue
                nt = math.ceil((ny - nb * B) / t)
                cost = P * (nb * (B + c) + nt * (t + c)) / resident + a * (t + c)
                if cost < best[0]:
                    best = (cost, (B, nb, t, nt))
    return best[1]


def check_cover(p, ny):
    rows, nsegs, trows, ntail = p["seg_rows"], p["nsegs"], p["tail_rows"], p["ntail"]
    assert rows >= 1 and nsegs >= 1 and trows >= 1 and ntail >= 0
    if ntail == 0:  # equal segments, none empty
        assert nsegs * rows >= ny > (nsegs - 1) * rows
    else:  # long segments, then short ones covering the rest, none empty
        rest = ny - nsegs * rows
        assert rest > 0
        assert ntail * trows >= rest > (ntail - 1) * trows
        assert rows >= 2 * trows and rows % 8 == 0


@pytest.mark.parametrize("scheme,storage", [("fd5", "f32"), ("fd3", "f32"), ("lwacm", "f32"),
                                            ("fd5", "f16"), ("lwacm", "bf16"), ("fd5", "i16")])
def test_segments_cover_the_rows_and_follow_the_model(scheme, storage):
    for nx in (256, 264, 1000, 4096, 8192, 12000):
        for ny in (1, 7, 16, 17, 40, 100, 1000, 4096, 8192, 16384):
            for resident in (152, RESIDENT, 2 * RESIDENT):
                p = F.stream_plan(nx, ny, scheme, storage, resident)
                check_cover(p, ny)
                assert p["strips"] == math.ceil(math.ceil(nx / 120) / 2)
                assert p["ctas"] == p["strips"] * (p["nsegs"] + p["ntail"])
                got = (p["seg_rows"], p["nsegs"], p["tail_rows"], p["ntail"])
                assert got == model_pick(nx, ny, scheme, storage, resident)
                if scheme == "lwacm":
                    assert p["ntail"] == 0  # LW-ACM keeps equal segments


def test_picks_measured_on_gb300():
    """Step times measured on GB300 (GLUPS, CUDA events): 8192^2 FD-5 with
    equal 64-row segments 205.1, with 34 segments of 200 rows then 24- or
    32-row ones 212.1 / 213.7; LW-ACM best with equal 16-row segments (275.0,
    230.7 with 34 of 200 then 16); 16384^2 FD-5 equal 120-row segments 221.7,
    35 of about 400 rows then 32-48 rows 227-229."""
    p = F.stream_plan(8192, 8192, "fd5", "f32", RESIDENT)
    assert (p["seg_rows"], p["nsegs"]) == (200, 34) and p["tail_rows"] in (24, 32)
    p = F.stream_plan(8192, 8192, "lwacm", "f32", RESIDENT)
    assert (p["seg_rows"], p["nsegs"], p["ntail"]) == (16, 512, 0)
    p = F.stream_plan(16384, 16384, "fd5", "f32", RESIDENT)
    assert p["nsegs"] == 35 and 392 <= p["seg_rows"] <= 432 and 32 <= p["tail_rows"] <= 48


def test_candidates_start_with_the_model_plan_and_are_valid():
    for nx, ny, scheme, storage in [(8192, 8192, "fd5", "f32"), (16384, 16384, "fd5", "f32"),
                                    (4096, 4096, "fd3", "f16"), (8192, 8192, "lwacm", "f32"),
                                    (1000, 40, "fd5", "f32"), (256, 16, "fd5", "i16")]:
        p = F.stream_plan(nx, ny, scheme, storage, RESIDENT)
        c = F.stream_plan_candidates(nx, ny, scheme, storage, RESIDENT, 64)
        assert 1 <= len(c) <= 64 and len(set(c)) == len(c)
        assert c[0] == (p["seg_rows"], p["nsegs"], p["tail_rows"])
        for B, nb, t in c:
            assert B >= 1 and nb >= 1 and t >= 1
            if nb * B >= ny:  # equal segments
                assert t == B and (nb - 1) * B < ny
            else:
                assert B >= 2 * t and B % 8 == 0
        assert F.stream_plan_candidates(nx, ny, scheme, storage, RESIDENT, 3) == c[:3]
    # the plans measured best on 8192^2 and 16384^2 are among those timed
    c = F.stream_plan_candidates(8192, 8192, "fd5", "f32", RESIDENT, 32)
    assert (200, 34, 32) in c and (200, 34, 24) in c
    c = F.stream_plan_candidates(16384, 16384, "fd5", "f32", RESIDENT, 64)
    assert (408, 35, 48) in c or (392, 35, 48) in c


def test_invalid_arguments():
    lib = F.load_library()
    out = (ctypes.c_int32 * 6)()
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 0, RESIDENT, None) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(8192, 8192, 100, 0, RESIDENT, out) == F.ERR_INVALID  # MRT
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 7, RESIDENT, out) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(0, 8192, 5, 0, RESIDENT, out) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 0, 0, out) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan(8192, 8192, 5, 0, RESIDENT, out) == F.OK
    cand = (ctypes.c_int32 * 12)()
    n = ctypes.c_int32()
    assert lib.fdlbm_stream_plan_candidates(8192, 8192, 5, 0, RESIDENT, cand, 0,
                                            ctypes.byref(n)) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan_candidates(8192, 8192, 5, 0, RESIDENT, cand, 4,
                                            None) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan_candidates(8192, 8192, 5, 0, RESIDENT, None, 4,
                                            ctypes.byref(n)) == F.ERR_INVALID
    assert lib.fdlbm_stream_plan_candidates(8192, 8192, 5, 0, RESIDENT, cand, 4,
                                            ctypes.byref(n)) == F.OK and n.value == 4
    assert lib.fdlbm_set_stream_plan(None, 64, 2, 16) == F.ERR_INVALID
    assert lib.fdlbm_get_stream_plan(None, out) == F.ERR_INVALID
