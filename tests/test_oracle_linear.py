"""Pins of the oracle's linear behaviour.

- The numpy amplification matrices H(k) (Eq. iteration) reproduce the
  hyperviscosities printed in Table 1, the shear viscosity
  nu = (1/s_xx - 1/2)/3 and sound speed 1/sqrt(3) of Sec. 1-a, and the
  isotropy of the MRT hyperviscosity under the quartic condition (Eq. sigsig).
- The brute-force Jacobian of the C oracle's step on tiny periodic grids
  equals H(k) entry by entry, for every wave vector of the grid, so the
  oracle's linear part is pinned by the same printed numbers.
"""
import os

import numpy as np
import pytest

from oracle import linear

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_hyperviscosity.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


@pytest.mark.parametrize("col,stencil", [(1, "3"), (2, "5"), (3, "9")])
def test_table1_hyperviscosity(col, stencil):
    """Table 1 (Sec. 3-a): nu_2 vs angle at s_xx = 1.85, to the printed digits."""
    tab = _table1()
    for row in tab:
        angle, printed = row[0], row[col]
        nu0, nu2 = linear.viscosity_expansion(stencil, np.deg2rad(angle), 1.85)
        decimals = 4 if abs(printed) == 0.0196 else 5
        assert abs(nu2 - printed) <= 0.5 * 10.0 ** (-decimals) + 1e-9, (stencil, angle, nu2)


@pytest.mark.parametrize("stencil", ["3", "5"])
def test_hyperviscosity_closed_forms(stencil):
    """Sec. 2 closed forms of nu_2 for the 3- and 5-point stencils, with the
    anisotropic term's sign fixed by Table 1 (+ sign)."""
    for s_xx in (1.2, 1.5, 1.85, 1.95):
        sig = 1.0 / s_xx - 0.5
        for phi in np.deg2rad([0.0, 13.0, 26.6, 45.0, 71.0]):
            c2 = np.cos(phi) ** 2
            aniso = c2 - c2 ** 2
            if stencil == "3":
                expect = (2 * sig - 3) * (2 * sig - 1) / 72 + (8 * sig - 3) / 36 * aniso
            else:
                expect = sig * (2 * sig - 1) / 36 + sig / 18 * aniso
            _, nu2 = linear.viscosity_expansion(stencil, phi, s_xx)
            assert abs(nu2 - expect) < 1e-7, (s_xx, phi, nu2, expect)


@pytest.mark.parametrize("scheme", ["3", "5", "9", "mrt"])
def test_shear_viscosity_and_sound_speed(scheme):
    """Sec. 1-a: nu = (1/s_xx - 1/2)/3 and c_s = 1/sqrt(3) (same for FD-LBM, Sec. 2)."""
    for s_xx in (1.3, 1.7, 1.9):
        nu0, _ = linear.viscosity_expansion(scheme, 0.3, s_xx, 1.5, 1.1, 1.4)
        assert abs(nu0 - (1 / s_xx - 0.5) / 3) < 1e-9
    k = 1e-3
    if scheme == "mrt":
        H = linear.H_mrt(k, 0.0, 1.7, 1.5, 1.1, 1.4)
    else:
        H = linear.H_fd(int(scheme), k, 0.0, 1.7, 1.5)
    z = np.linalg.eigvals(H)
    speeds = sorted(abs(np.angle(zz)) / k for zz in z if abs(zz) > 0.99)
    assert abs(speeds[-1] - 1 / np.sqrt(3)) < 1e-6


def test_sound_damping_bulk_viscosity():
    """Sec. 1-a: bulk viscosity zeta = (1/s_e - 1/2)/3; sound is damped at
    (nu + zeta)/2 k^2 in the long-wave limit, for FD-LBM and MRT alike."""
    k = 2e-3
    for s_e in (1.2, 1.5, 1.8):
        nu, zeta = (1 / 1.7 - 0.5) / 3, (1 / s_e - 0.5) / 3
        for H in (linear.H_fd(5, k, 0.0, 1.7, s_e), linear.H_mrt(k, 0.0, 1.7, s_e, 1.1, s_e)):
            z = [zz for zz in np.linalg.eigvals(H)
                 if abs(zz) > 0.9 and abs(np.angle(zz)) > 0.5 * k / np.sqrt(3)]
            assert len(z) == 2
            for zz in z:
                assert abs(-np.log(abs(zz)) / k ** 2 - (nu + zeta) / 2) < 1e-5


def test_quartic_condition_isotropic_mrt():
    """Eq. sigsig: (1/s_xx - 1/2)(1/s_q - 1/2) = 1/6 makes the MRT shear
    hyperviscosity isotropic; s_q = 0.9282 at nu = 1/sqrt(108) (Sec. 3-b)."""
    nu = 1 / np.sqrt(108)
    s_xx = 1 / (3 * nu + 0.5)
    s_q = 1 / (1 / (6 * (1 / s_xx - 0.5)) + 0.5)
    assert abs(s_q - 0.9282) < 5e-5
    nu2 = [linear.viscosity_expansion("mrt", np.deg2rad(a), s_xx, 1.5, s_q, 1.5)[1]
           for a in (0.0, 26.6, 45.0)]
    assert max(nu2) - min(nu2) < 1e-6
    nu2_off = [linear.viscosity_expansion("mrt", np.deg2rad(a), s_xx, 1.5, 1.3, 1.5)[1]
               for a in (0.0, 45.0)]
    assert abs(nu2_off[0] - nu2_off[1]) > 1e-3


def test_nine_point_unstable_along_diagonal():
    """Sec. 3-a: the nine-point stencil is linearly unstable in the {1,1}
    direction at nu_0 = 0.01; the three- and five-point stencils are stable."""
    s_xx = 1 / (3 * 0.01 + 0.5)
    diag = [np.max(np.abs(np.linalg.eigvals(linear.H_fd(9, k, k, s_xx, 1.5))))
            for k in np.linspace(0.05, np.pi / 1.0, 60)]
    assert max(diag) > 1.0 + 1e-6
    for st in (3, 5):
        assert linear.max_abs_z(str(st), s_xx, 1.5, n=24) <= 1.0 + 1e-12


def _jacobian_blocks(ref, p, ncomp, run_step, base_state, h=1e-6):
    """Fourier blocks of the oracle's one-step Jacobian around a uniform state.

    For each grid wave vector k the complex plane waves e_c exp(i k.x) are
    pushed through the central-difference linearisation and projected back
    on exp(i k.x); off-k leakage is returned too."""
    nx, ny = p.nx, p.ny
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    blocks, leak = {}, 0.0
    for m in range(nx):
        for n in range(ny):
            kx, ky = 2 * np.pi * m / nx, 2 * np.pi * n / ny
            ph = np.exp(1j * (kx * X + ky * Y))
            B = np.zeros((ncomp, ncomp), dtype=complex)
            for c in range(ncomp):
                resp = []
                for part in (ph.real, ph.imag):
                    outs = []
                    for sgn in (1.0, -1.0):
                        st = [b.copy() for b in base_state]
                        st[c] = st[c] + sgn * h * part
                        outs.append(np.array(run_step(st)))
                    resp.append((outs[0] - outs[1]) / (2 * h))
                r = resp[0] + 1j * resp[1]
                proj = (r * np.conj(ph)).mean(axis=(1, 2))
                B[:, c] = proj
                leak = max(leak, float(np.abs(r - proj[:, None, None] * ph).max()))
            blocks[(kx, ky)] = B
    return blocks, leak


@pytest.mark.parametrize("stencil", [3, 5, 9])
def test_oracle_jacobian_equals_symbol_fd(oracle, stencil):
    """Linearised oracle step == H_fd(k) for all k of an 8x6 periodic grid."""
    p = oracle.params(8, 6, stencil, 1.7, 1.4)
    base = [np.ones((6, 8)), np.zeros((6, 8)), np.zeros((6, 8))]
    blocks, leak = _jacobian_blocks(oracle, p, 3, lambda st: oracle.fd_run(p, *st, 1), base)
    assert leak < 1e-8
    for (kx, ky), B in blocks.items():
        H = linear.H_fd(stencil, kx, ky, 1.7, 1.4)
        assert np.abs(B - H).max() < 1e-8, (kx, ky)


def test_oracle_jacobian_equals_symbol_mrt(oracle):
    """Linearised oracle MRT step == H_mrt(k) on populations, 6x5 grid."""
    p = oracle.params(6, 5, oracle.MRT, 1.6, 1.3, 1.1, 1.4)
    f0 = oracle.mrt_init(p, np.ones((5, 6)), np.zeros((5, 6)), np.zeros((5, 6)))
    base = [f0[a] for a in range(9)]
    blocks, leak = _jacobian_blocks(
        oracle, p, 9, lambda st: oracle.mrt_step(p, np.stack(st), 1), base)
    assert leak < 1e-8
    for (kx, ky), B in blocks.items():
        H = linear.H_mrt(kx, ky, 1.6, 1.3, 1.1, 1.4)
        assert np.abs(B - H).max() < 1e-8, (kx, ky)


def test_bessel_column_reading():
    """Tables 2-3 'Bessel' column: singlets are squared zeros of J_1 and the
    l-th doublet the squared first zero of J_{l+1} (reading of Sec. 3-b)."""
    special = pytest.importorskip("scipy.special")
    with open(os.path.join(GOLDEN, "bessel_stokes_rates.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    j1 = special.jn_zeros(1, 6)
    for kind, l, val in rows:
        l, val = int(l), float(val)
        a = j1[l - 1] if kind == "singlet" else special.jn_zeros(l + 1, 1)[0]
        assert abs(a * a - val) < 6e-4, (kind, l)
