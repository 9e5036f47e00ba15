"""The oracle's pins would catch a plausible mistake: each test plants one
mistake in a copy of the oracle's source (on the CPU), builds it, and checks
that at least one pin (Table 1 via the Jacobian, the closed-form shear
wave, the Poiseuille curvature, the damping of sound in a mean flow)
rejects the mutant while the unmodified oracle passes them all."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import linear
from paper_1803_00437_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fdlbm_ref.c")

MUTANTS = {
    # sign of the strain-rate term of theta_XY (the paper's misprint)
    "theta_xy_sign": ("(1.0 / 3.0) * (dx_Jy + dy_Jx)", "(1.0 / 3.0) * (dx_Jy - dy_Jx)"),
    # a Jx row of M without its minus signs (as printed)
    "m_row_sign": ("    {0, 1, 0, -1, 0, 1, -1, -1, 1},", "    {0, 1, 0, 1, 0, 1, 1, -1, 1},"),
    # five-point weight 3/4 -> 2/3
    "fd5_weight": ("return 0.75 * (FQ(i + di, j + dj)", "return (2.0 / 3.0) * (FQ(i + di, j + dj)"),
    # propagation in the wrong direction in the FD-LBM step
    "stream_direction": ("                    const int si = wrap(i - CX[a], nx);\n                    int sj = j - CY[a];\n                    if (!walls) sj = wrap(sj, ny);\n                    f[a] = fstar",
                         "                    const int si = wrap(i + CX[a], nx);\n                    int sj = j + CY[a];\n                    if (!walls) sj = wrap(sj, ny);\n                    f[a] = fstar"),
    # second half of the force dropped
    "half_force": ("m[1] = Jx + 0.5 * p->force_x;", "m[1] = Jx;"),
    # terms of theta that vanish at rest and only a mean flow sees
    "theta_e_v2": ("(2.0 + 6.0 * (vx * vx + vy * vy)) * (dx_Jx + dy_Jy)",
                   "(2.0 + 0.0 * (vx * vx + vy * vy)) * (dx_Jx + dy_Jy)"),
    "theta_e_rho": ("2.0 * (vx * drx + vy * dry);", "4.0 * (vx * drx + vy * dry);"),
    "theta_xx_rho": ("(2.0 / 3.0) * (vx * drx - vy * dry)", "(1.0 / 3.0) * (vx * drx - vy * dry)"),
    "theta_xx_flux": ("2.0 * (vx * (dx_Pxx + dy_Pxy) - vy * (dx_Pxy + dy_Pyy))",
                      "1.0 * (vx * (dx_Pxx + dy_Pxy) - vy * (dx_Pxy + dy_Pyy))"),
}

# the nine-point stencil and the curved-wall closure, checked by their own pins
NINE_WALL_MUTANTS = {
    # nine points: corner weight 1/4 -> 1/2 along x
    "fd9_corner_weight": ("                return FQ(i + 1, j) - FQ(i - 1, j) -\n                       0.25 * (",
                          "                return FQ(i + 1, j) - FQ(i - 1, j) -\n                       0.5 * ("),
    # curved walls: always extrapolate from the first fluid node
    "wall_reference_node": ("const int tref = (xi >= 0.5) ? d : d + 1;", "const int tref = d;"),
    # curved walls: density of the node along the line one step too far
    "wall_density_node": ("    *r = F->rho[first];", "    *r = F->rho[ref];"),
}

# the density of the channel's virtual rows, checked by the standing sound wave
WALL_DENSITY_MUTANTS = {
    # copied from the second fluid row instead of the first, at both walls
    "channel_density_second_row": (
        "        jrho = 0;\n    } else {\n        ywall = (double)(ny - 1) + xi;\n"
        "        jref = (xi >= 0.5) ? ny - 1 : ny - 2;\n        jrho = ny - 1;",
        "        jrho = 1;\n    } else {\n        ywall = (double)(ny - 1) + xi;\n"
        "        jref = (xi >= 0.5) ? ny - 1 : ny - 2;\n        jrho = ny - 2;"),
    # copied from the second fluid row at the lower wall only
    "channel_density_second_row_lower": ("        jrho = 0;\n", "        jrho = 1;\n"),
    # virtual rows at the rest density
    "channel_density_at_rest": ("    *r = F->rho[(int64_t)jrho * nx + i];", "    *r = 1.0;"),
}

# LW-ACM (Sec. 1-b), checked by its own pins
LW_MUTANTS = {
    # odd part taken at the upstream node instead of the node the link points to
    "lw_upstream": ("const int64_t d = (int64_t)wrap(j + CY[a], ny) * nx + wrap(i + CX[a], nx);",
                    "const int64_t d = (int64_t)wrap(j - CY[a], ny) * nx + wrap(i - CX[a], nx);"),
    # Theta = 1 - 2 nu / c_s^2 with c_s^2 = 2/3 instead of 1/3
    "lw_theta": ("return 1.0 - 6.0 * nu;", "return 1.0 - 3.0 * nu;"),
    # equilibrium without its quadratic term
    "lw_quadratic": ("1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2", "1.0 + 3.0 * cu - 1.5 * u2"),
    # even part instead of the odd part
    "lw_even_part": ("return 0.5 * (lw_feq(a, r, vx, vy) - lw_feq(a, r, -vx, -vy));",
                     "return 0.5 * (lw_feq(a, r, vx, vy) + lw_feq(a, r, -vx, -vy));"),
}


def _build(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    d = tmp / name
    d.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "fdlbm_ref.h"), d)
    (d / "fdlbm_ref.c").write_text(src.replace(old, new, 1))
    lib = d / "lib.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                    "-o", str(lib), str(d / "fdlbm_ref.c"), "-lm"], check=True)
    return str(lib)


def _pins_pass(ref):
    """The pins, evaluated with the oracle module `ref` (its library path set)."""
    failures = []
    # 1. Jacobian of the step == symbol H(k) (pinned by Table 1), FD-5, 6x5 grid
    p = ref.params(6, 5, 5, 1.7, 1.4)
    X, Y = np.meshgrid(np.arange(6), np.arange(5))
    h = 1e-6
    for (m, n) in ((1, 0), (1, 2), (2, 1)):
        kx, ky = 2 * np.pi * m / 6, 2 * np.pi * n / 5
        ph = np.exp(1j * (kx * X + ky * Y))
        B = np.zeros((3, 3), complex)
        for c in range(3):
            cols = []
            for part in (ph.real, ph.imag):
                o = []
                for sg in (1, -1):
                    st = [np.ones((5, 6)), np.zeros((5, 6)), np.zeros((5, 6))]
                    st[c] = st[c] + sg * h * part
                    o.append(np.array(ref.fd_run(p, *st, 1)))
                cols.append((o[0] - o[1]) / (2 * h))
            r = cols[0] + 1j * cols[1]
            B[:, c] = (r * np.conj(ph)).mean(axis=(1, 2))
        if np.abs(B - linear.H_fd(5, kx, ky, 1.7, 1.4)).max() > 1e-8:
            failures.append("jacobian")
            break
    # 2. closed-form shear wave, three points
    N, A, s = 32, 0.01, 1 / (3 * 0.02 + 0.5)
    d, ux, uy = inputs.shear_wave(N, N, A, m=0, n=1, phase=np.pi / 2)
    k = 2 * np.pi / N
    r, x, yv = ref.fd_run(ref.params(N, N, 3, s, 1.5), 1 + d, ux, uy, 100)
    z = 1 - (1 - np.cos(k)) / 3 + (1 - 1 / s) / 3 * np.sin(k) ** 2
    yy = np.arange(N)[:, None] * np.ones((1, N))
    if np.abs(x - A * z ** 100 * np.sin(k * yy)).max() > 1e-12 * A:
        failures.append("shear")
    # 3. Poiseuille curvature F / (2 nu), five points
    nu, N = 0.1, 16
    F = 8 * nu * 0.05 / (N ** 2)
    pc = ref.params(4, N, 5, 1 / (3 * nu + 0.5), 1.5, boundary=1, wall_xi=0.5, force=(F, 0.0))
    zf = np.zeros((N, 4))
    r, x, yv = ref.fd_run(pc, 1 + zf, zf, zf, 4000)
    u = x[:, 0]
    yy = np.arange(N)
    curv = -np.polyfit(yy[4:12], u[4:12], 2)[0]
    if abs(curv / (F / (2 * nu)) - 1) > 2e-5:
        failures.append("poiseuille")
    # 4. sound damping in a mean flow against its hand-derived rates, five points
    import test_oracle_closed_forms as C
    nu, s_e, V = 0.01, 1.5, 0.1
    ps = ref.params(256, 1, 5, 1 / (3 * nu + 0.5), s_e)
    e0 = C.sound_rates_in_mean_flow(nu, s_e, 0.0)[0]
    (_, g0m), _, (_, g0p) = C._sound_modes(ref, ps, 0.0)
    (_, gm), _, (_, gp) = C._sound_modes(ref, ps, V)
    em, ep = C.sound_rates_in_mean_flow(nu, s_e, V)
    if max(abs((gm - g0m) - (em - e0)), abs((gp - g0p) - (ep - e0))) > 1.5e-3 * e0:
        failures.append("mean_flow_sound")
    return failures


@pytest.fixture()
def oracle_at(tmp_path):
    from oracle import ref

    def load(path):
        ref._lib = None
        ref.LIB = path
        return ref

    yield load
    ref._lib = None
    ref.LIB = os.path.join(ROOT, "oracle", "libfdlbm_ref.so")


def _lw_pins_pass(ref):
    """The LW-ACM pins (see test_oracle_lwacm): printed H(k), sound, nu(v),
    conservation."""
    import test_oracle_lwacm as T
    failures = []
    B, k, _ = T._jacobian(ref, 64, 4, 1, 0, 0.02)
    if np.abs(B - T._printed_H(k, 0.02)).max() > k ** 3:
        failures.append("printed_H")
    B, k, _ = T._jacobian(ref, 128, 4, 1, 0, 0.02, V=(0.1, 0.0))
    w, vecs = np.linalg.eig(B)
    shear = w[np.argmax(np.abs(vecs[2, :]))]
    if abs(-np.log(abs(shear)) / ((0.02 - 0.005) * k * k) - 1) > 0.02:
        failures.append("nu_of_v")
    p = ref.params(24, 20, ref.LWACM, T._s(0.02))
    d, ux, uy = inputs.random_fields(24, 20, 0.02, seed=6, rho_amp=0.01)
    r, x, y = ref.lwacm_run(p, 1 + d, ux, uy, 50)
    if abs(r.sum() - (1 + d).sum()) > 1e-10 or abs((r * x).sum() - ((1 + d) * ux).sum()) > 1e-10:
        failures.append("conservation")
    return failures


def test_unmodified_oracle_passes_the_pins(oracle_at):
    from oracle import ref
    ref.build()
    assert _pins_pass(oracle_at(os.path.join(ROOT, "oracle", "libfdlbm_ref.so"))) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, oracle_at, name):
    old, new = MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    failures = _pins_pass(oracle_at(lib))
    assert failures, f"mutant {name} passed every pin"


def test_unmodified_lwacm_oracle_passes_its_pins(oracle_at):
    from oracle import ref
    ref.build()
    assert _lw_pins_pass(oracle_at(os.path.join(ROOT, "oracle", "libfdlbm_ref.so"))) == []


@pytest.mark.parametrize("name", sorted(LW_MUTANTS))
def test_planted_lwacm_mistake_is_caught(tmp_path, oracle_at, name):
    old, new = LW_MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    failures = _lw_pins_pass(oracle_at(lib))
    assert failures, f"mutant {name} passed every pin"


def _nine_wall_pins_pass(ref):
    """Pins of the nine-point stencil (the Jacobian of one step equals the
    symbol H(k), which Table 1 pins) and of the curved-wall closure (a
    straight channel written as a wall table equals the channel closure,
    whose own code the Poiseuille pins cover)."""
    failures = []
    p = ref.params(6, 5, 9, 1.7, 1.4)
    X, Y = np.meshgrid(np.arange(6), np.arange(5))
    h = 1e-6
    for (m, n) in ((1, 0), (1, 2), (2, 1)):
        kx, ky = 2 * np.pi * m / 6, 2 * np.pi * n / 5
        ph = np.exp(1j * (kx * X + ky * Y))
        B = np.zeros((3, 3), complex)
        for c in range(3):
            cols = []
            for part in (ph.real, ph.imag):
                o = []
                for sg in (1, -1):
                    st = [np.ones((5, 6)), np.zeros((5, 6)), np.zeros((5, 6))]
                    st[c] = st[c] + sg * h * part
                    o.append(np.array(ref.fd_run(p, *st, 1)))
                cols.append((o[0] - o[1]) / (2 * h))
            r = cols[0] + 1j * cols[1]
            B[:, c] = (r * np.conj(ph)).mean(axis=(1, 2))
        if np.abs(B - linear.H_fd(9, kx, ky, 1.7, 1.4)).max() > 1e-8:
            failures.append("jacobian9")
            break
    nx, nyf, reach = 12, 10, 3
    for xi in (0.25, 0.8):
        walls = inputs.channel_walls(nx, nyf, xi, reach)
        d, ux, uy = inputs.random_fields(nx, nyf, 0.02, seed=4, rho_amp=0.01)
        pw = ref.params(nx, nyf, 5, 1.7, 1.4, boundary=ref.WALLS_Y, wall_xi=xi)
        r1, x1, y1 = ref.run(pw, 1 + d, ux, uy, 10)
        pad = lambda a, v: np.vstack([np.full((reach, nx), v), a, np.full((reach, nx), v)])
        pp = ref.params(nx, nyf + 2 * reach, 5, 1.7, 1.4)
        r2, x2, y2 = ref.fd_run_walls(pp, walls, pad(1 + d, 1.0), pad(ux, 0.0), pad(uy, 0.0), 10)
        fl = slice(reach, reach + nyf)
        if max(np.abs(r2[fl] - r1).max(), np.abs(x2[fl] - x1).max()) > 1e-14:
            failures.append(f"channel_table_xi{xi}")
    return failures


def test_unmodified_oracle_passes_the_nine_point_and_wall_pins(oracle_at):
    from oracle import ref
    ref.build()
    assert _nine_wall_pins_pass(oracle_at(os.path.join(ROOT, "oracle", "libfdlbm_ref.so"))) == []


@pytest.mark.parametrize("name", sorted(NINE_WALL_MUTANTS))
def test_planted_nine_point_or_wall_mistake_is_caught(tmp_path, oracle_at, name):
    old, new = NINE_WALL_MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    failures = _nine_wall_pins_pass(oracle_at(lib))
    assert failures, f"mutant {name} passed every pin"


def _wall_density_pins_pass(ref):
    """The standing sound wave between walls at xi = 1/2 (see
    test_oracle_closed_forms.test_standing_sound_wave_between_walls): walls
    at -1/2 and ny - 1/2 to second order, for both stencils."""
    import test_oracle_closed_forms as C
    failures = []
    for stencil in (3, 5):
        gaps = {ny: C.acoustic_wall_gap(ref, stencil, ny) for ny in (24, 48)}
        scaled = np.array([g * ny * ny for ny, g in gaps.items()])
        if not (np.all(scaled > 0) and np.all(scaled < 1.0)
                and scaled.max() / scaled.min() - 1 < 0.01):
            failures.append(f"standing_wave_fd{stencil}")
    return failures


def test_unmodified_oracle_passes_the_wall_density_pin(oracle_at):
    from oracle import ref
    ref.build()
    assert _wall_density_pins_pass(oracle_at(os.path.join(ROOT, "oracle", "libfdlbm_ref.so"))) == []


@pytest.mark.parametrize("name", sorted(WALL_DENSITY_MUTANTS))
def test_planted_wall_density_mistake_is_caught(tmp_path, oracle_at, name):
    old, new = WALL_DENSITY_MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    failures = _wall_density_pins_pass(oracle_at(lib))
    assert failures, f"mutant {name} passed every pin"
