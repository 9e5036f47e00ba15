"""Pins of the LW-ACM oracle (Sec. 1-b): the link-wise artificial
compressibility method that rebuilds every link from equilibria only,
f_a(x) = feq_a(x - c_a) + Theta (feo_a(x) - feo_a(x - c_a)), Theta = 1 - 6 nu.

What fixes it, independently of the oracle's code:
- the linear amplification matrix H(k) printed in Sec. 1-b (at v = 0, to
  second order in k) against the Jacobian of one oracle step on a grid;
- the sound speed c_s = sqrt(2 nu) and sound damping nu/2 + 1/12 stated there;
- the mean-flow shear viscosity nu(v) = nu - v^2/2 stated there, and the
  instability it implies for v > c_s;
- the Fig. 1 experiment of Sec. 3-a (191^2, wave vector (3, 2) 2 pi / 191,
  mean velocity along k): damping falls as V grows, at the rate nu(V) k^2;
- exact conservation of mass and momentum on a periodic lattice.
"""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs


def _s(nu):
    return 1.0 / (3.0 * nu + 0.5)


def _jacobian(oracle, nx, ny, m, n, nu, V=(0.0, 0.0), h=1e-7):
    """3x3 response of one step to a Fourier perturbation exp(i k.x) of
    (rho, Jx, Jy) about rho = 1, u = V (J = rho u: at linear order about a
    uniform state dJ = du + V drho)."""
    p = oracle.params(nx, ny, oracle.LWACM, _s(nu))
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    kx, ky = 2 * np.pi * m / nx, 2 * np.pi * n / ny
    ph = np.exp(1j * (kx * X + ky * Y))
    one = np.ones((ny, nx))
    B = np.zeros((3, 3), complex)
    for c in range(3):
        cols = []
        for part in (ph.real, ph.imag):
            out = []
            for sg in (1, -1):
                d = sg * h * part
                r = one + (d if c == 0 else 0)
                jx = V[0] * one + (d if c == 1 else 0)
                jy = V[1] * one + (d if c == 2 else 0)
                r1, u1, v1 = oracle.lwacm_run(p, r, jx / r, jy / r, 1)
                out.append(np.array([r1, r1 * u1, r1 * v1]))
            cols.append((out[0] - out[1]) / (2 * h))
        resp = cols[0] + 1j * cols[1]
        B[:, c] = (resp * np.conj(ph)).mean(axis=(1, 2))
    return B, kx, ky


def _printed_H(k, nu):
    """H(k) of Sec. 1-b at v = 0, wave vector along x, basis (rho, Jx, Jy)."""
    return np.array([[1 - k * k / 6, -6j * nu * k, 0],
                     [-1j * k / 3, 1 - 3 * nu * k * k, 0],
                     [0, 0, 1 - nu * k * k]])


def test_two_phase_step_equals_point_form(oracle):
    p = oracle.params(40, 30, oracle.LWACM, _s(0.03))
    d, ux, uy = inputs.random_fields(40, 30, 0.02, seed=5, rho_amp=0.01)
    r, x, y = oracle.lwacm_run(p, 1 + d, ux, uy, 1)
    pts = oracle.lwacm_step_points(p, 1 + d, ux, uy, np.arange(40 * 30))
    assert np.array_equal(pts[:, 0], r.ravel())
    assert np.array_equal(pts[:, 1], x.ravel())
    assert np.array_equal(pts[:, 2], y.ravel())


def test_mass_and_momentum_conserved(oracle):
    p = oracle.params(48, 40, oracle.LWACM, _s(0.02))
    d, ux, uy = inputs.random_fields(48, 40, 0.02, seed=6, rho_amp=0.01)
    r0 = 1 + d
    r, x, y = oracle.lwacm_run(p, r0, ux, uy, 300)
    assert abs(r.sum() - r0.sum()) <= 1e-12 * r0.sum()
    assert abs((r * x).sum() - (r0 * ux).sum()) <= 1e-12 * np.abs(r0 * ux).sum()
    assert abs((r * y).sum() - (r0 * uy).sum()) <= 1e-12 * np.abs(r0 * uy).sum()


@pytest.mark.parametrize("nu", [0.01, 0.05])
def test_linear_symbol_is_the_printed_H(oracle, nu):
    """The Jacobian of one step equals H(k) of Sec. 1-b up to third order in
    k: the gap shrinks eightfold when k halves."""
    gaps = []
    for m in (2, 1):
        B, kx, _ = _jacobian(oracle, 64, 4, m, 0, nu)
        gap = np.abs(B - _printed_H(kx, nu)).max()
        assert gap <= kx ** 3, (m, gap, kx ** 3)
        gaps.append(gap)
    assert 5.0 < gaps[0] / gaps[1] < 11.0, gaps


def test_sound_speed_and_damping(oracle):
    """Longitudinal pair of roots exp(+-i c_s k - Gamma_s k^2) with
    c_s = sqrt(2 nu) and Gamma_s = nu/2 + 1/12 (Sec. 1-b), at small k."""
    nu = 0.02
    B, k, _ = _jacobian(oracle, 128, 4, 1, 0, nu)
    z = np.linalg.eigvals(B[:2, :2])
    lz = np.log(z)
    cs = np.abs(lz.imag).max() / k
    gs = -lz.real.mean() / k ** 2
    assert abs(cs / np.sqrt(2 * nu) - 1) < 0.01, cs
    assert abs(gs / (nu / 2 + 1.0 / 12) - 1) < 0.02, gs


@pytest.mark.parametrize("V", [0.0, 0.05, 0.1])
def test_mean_flow_shear_viscosity(oracle, V):
    """Shear root about a uniform flow V along k: damping (nu - V^2/2) k^2
    per step (Sec. 1-b), to O(k^2)."""
    nu = 0.02
    B, k, _ = _jacobian(oracle, 128, 4, 1, 0, nu, V=(V, 0.0))
    z = np.linalg.eigvals(B)
    # the shear root: eigenvector along Jy
    w, vecs = np.linalg.eig(B)
    shear = w[np.argmax(np.abs(vecs[2, :]))]
    gamma = -np.log(abs(shear))
    assert abs(gamma / ((nu - V * V / 2) * k * k) - 1) < 0.02, (gamma, z)


def test_shear_waves_grow_above_the_sound_speed(oracle):
    """nu(v) < 0 for v > c_s = sqrt(2 nu): the shear root leaves the unit circle."""
    nu = 0.005
    B, k, _ = _jacobian(oracle, 64, 4, 1, 0, nu, V=(0.15, 0.0))
    w, vecs = np.linalg.eig(B)
    shear = w[np.argmax(np.abs(vecs[2, :]))]
    assert abs(shear) > 1.0


def test_fig1_damping_falls_as_mean_velocity_grows(oracle):
    """Sec. 3-a, Fig. 1: 191 x 191 periodic, shear wave of wave vector
    (3, 2) 2 pi / 191 carried by a mean velocity V parallel to k.  The
    amplitude of the wave decays at (nu - V^2/2) k^2 per step; the paper does
    not state nu for this figure, nu = 0.01 is used."""
    N, nu, A, steps = 191, 0.01, 1e-4, 400
    kx, ky = 2 * np.pi * 3 / N, 2 * np.pi * 2 / N
    k = np.hypot(kx, ky)
    X, Y = np.meshgrid(np.arange(N), np.arange(N))
    ph = kx * X + ky * Y
    p = oracle.params(N, N, oracle.LWACM, _s(nu))
    rates = []
    for V in (0.0, 0.04, 0.08):
        jx = -A * ky / k * np.cos(ph) + kx / k * V
        jy = A * kx / k * np.cos(ph) + ky / k * V
        r = np.ones((N, N))
        r1, u1, v1 = oracle.lwacm_run(p, r, jx, jy, steps)

        def amp(ux, uy):
            ut = (-ky * ux + kx * uy) / k
            return abs((ut * np.exp(-1j * ph)).mean())
        g = -np.log(amp(r1 * u1, r1 * v1) / amp(jx, jy)) / steps
        assert abs(g / ((nu - V * V / 2) * k * k) - 1) < 0.03, (V, g)
        rates.append(g)
    assert rates[0] > rates[1] > rates[2]
