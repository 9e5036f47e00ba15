"""Von Neumann (Fourier) analysis of the FD-LBM and MRT D2Q9 schemes.

TEST INFRASTRUCTURE ONLY (part of the oracle).

The amplification matrix H(k) of Eq. iteration, Phi^{n+1} = H Phi^n, built
directly from the definition of one time step in Fourier space (Sec. 1-b and
Sec. 2): a plane wave of small amplitude on the state at rest (rho = 1,
u = 0) is reconstructed / collided, mapped to populations by M^-1 and
propagated with the phase factor exp(-i k.c) of Eq. 2.  The dispersion
relation is det(H - z Id) = 0 (Eq. disp) and the attenuation rate of a mode
is Gamma = -log z.  Written independently of the C oracle; the tests check
that the brute-force Jacobian of the C oracle's step on tiny periodic grids
equals these matrices, and that these matrices reproduce the paper's
printed hyperviscosities (Table 1) and transport coefficients (Sec. 1-a).
"""
from __future__ import annotations

import numpy as np

# Velocity set and moment matrix, Sec. 1 (rows rho, Jx, Jy, E, XX, XY, qx, qy, eps)
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
             dtype=float)
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
], dtype=float)
MINV = np.linalg.inv(M)


def deriv_symbol(stencil: int, kx: float, ky: float):
    """Fourier symbols (Dx, Dy) of the finite differences of Sec. 2:
    the difference operator applied to exp(i k.x) returns D exp(i k.x)."""
    if stencil == 3:
        return 1j * np.sin(kx), 1j * np.sin(ky)
    if stencil == 5:
        return (1j * (1.5 * np.sin(kx) - 0.25 * np.sin(2 * kx)),
                1j * (1.5 * np.sin(ky) - 0.25 * np.sin(2 * ky)))
    if stencil == 9:
        # f(i+1,j) - f(i-1,j) - 1/4 [f(i+1,j+1) - f(i-1,j+1) - f(i-1,j-1) + f(i+1,j-1)]
        return (1j * np.sin(kx) * (2.0 - np.cos(ky)), 1j * np.sin(ky) * (2.0 - np.cos(kx)))
    raise ValueError("stencil must be 3, 5 or 9")


def streaming(kx: float, ky: float):
    """Phase factors of Eq. 2: f_a(x) <- f*_a(x - c_a)."""
    return np.exp(-1j * (C[:, 0] * kx + C[:, 1] * ky))


def H_fd(stencil: int, kx: float, ky: float, s_xx: float, s_e: float):
    """3x3 amplification matrix of FD-LBM on the state (d rho, d Jx, d Jy) at rest.

    Linearised reconstruction (Sec. 2) at rho = 1, u = 0: the equilibria give
    E = -2 rho, XX = XY = 0, q = -J, eps = rho, and the defects reduce to
    theta_E = 2 div u, theta_XX = 2/3 (dx ux - dy uy),
    theta_XY = 1/3 (dx uy + dy ux)."""
    Dx, Dy = deriv_symbol(stencil, kx, ky)
    S = streaming(kx, ky)
    H = np.zeros((3, 3), dtype=complex)
    for c in range(3):
        phi = np.zeros(3, dtype=complex)
        phi[c] = 1.0
        dr, jx, jy = phi
        th_E = 2.0 * (Dx * jx + Dy * jy)
        th_XX = (2.0 / 3.0) * (Dx * jx - Dy * jy)
        th_XY = (1.0 / 3.0) * (Dx * jy + Dy * jx)
        m = np.array([dr, jx, jy,
                      -2.0 * dr + (1.0 - 1.0 / s_e) * th_E,
                      (1.0 - 1.0 / s_xx) * th_XX,
                      (1.0 - 1.0 / s_xx) * th_XY,
                      -jx, -jy, dr], dtype=complex)
        f_new = S * (MINV @ m)
        H[:, c] = [f_new.sum(), (C[:, 0] * f_new).sum(), (C[:, 1] * f_new).sum()]
    return H


def H_mrt(kx: float, ky: float, s_xx: float, s_e: float, s_q: float, s_eps: float):
    """9x9 amplification matrix of MRT D2Q9 (Eq. 1, 2) on the populations."""
    rates = np.diag([0.0, 0.0, 0.0, s_e, s_xx, s_xx, s_q, s_q, s_eps])
    # linear equilibria of the moments at rest, as a function of the moments
    Eq = np.zeros((9, 9))
    Eq[0, 0] = Eq[1, 1] = Eq[2, 2] = 1.0
    Eq[3, 0] = -2.0
    Eq[6, 1] = -1.0
    Eq[7, 2] = -1.0
    Eq[8, 0] = 1.0
    collide = MINV @ (np.eye(9) + rates @ (Eq - np.eye(9))) @ M
    return np.diag(streaming(kx, ky)) @ collide


def shear_root(H: np.ndarray, kx: float, ky: float, projector=None):
    """The eigenvalue z of H that belongs to the transverse (shear) mode."""
    w, V = np.linalg.eig(H)
    k = np.hypot(kx, ky)
    t = np.array([-ky / k, kx / k])
    norms = np.linalg.norm(V, axis=0)
    if projector is not None:
        V = projector @ V
    overlap = np.abs(t[0] * V[1] + t[1] * V[2]) / norms
    return w[np.argmax(overlap)]


def _moment_projector():
    # populations -> (rho, Jx, Jy)
    return M[:3]


def shear_gamma(scheme: str, k: float, phi: float, s_xx: float, s_e: float = 1.5,
                s_q: float = 1.0, s_eps: float = 1.5) -> float:
    """Attenuation rate Gamma = -log z of the shear mode along angle phi."""
    kx, ky = k * np.cos(phi), k * np.sin(phi)
    if scheme == "mrt":
        z = shear_root(H_mrt(kx, ky, s_xx, s_e, s_q, s_eps), kx, ky, _moment_projector())
    else:
        z = shear_root(H_fd(int(scheme), kx, ky, s_xx, s_e), kx, ky)
    return float(-np.log(np.abs(z)))


def viscosity_expansion(scheme: str, phi: float, s_xx: float, s_e: float = 1.5,
                        s_q: float = 1.0, s_eps: float = 1.5, kmax: float = 0.08, npts: int = 8):
    """Least-squares fit Gamma(k) / k^2 = nu0 + nu2 k^2 + nu4 k^4 + nu6 k^6 at small k.

    Returns (nu0, nu2): the long-wave shear viscosity and the hyperviscosity of
    Sec. 2 (Gamma = nu0 k^2 + nu2 k^4)."""
    ks = np.linspace(kmax / npts, kmax, npts)
    g = np.array([shear_gamma(scheme, k, phi, s_xx, s_e, s_q, s_eps) for k in ks])
    A = np.stack([np.ones_like(ks), ks ** 2, ks ** 4, ks ** 6], axis=1)
    coef, *_ = np.linalg.lstsq(A, g / ks ** 2, rcond=None)
    return float(coef[0]), float(coef[1])


def max_abs_z(scheme: str, s_xx: float, s_e: float = 1.5, s_q: float = 1.0, s_eps: float = 1.5,
              n: int = 48) -> float:
    """max |z| over a grid of wave vectors in [-pi, pi]^2 (linear stability,
    Sec. 2: the full dispersion equation solved numerically for k up to pi)."""
    worst = 0.0
    for kx in np.linspace(-np.pi, np.pi, n + 1):
        for ky in np.linspace(-np.pi, np.pi, n + 1):
            if scheme == "mrt":
                H = H_mrt(kx, ky, s_xx, s_e, s_q, s_eps)
            else:
                H = H_fd(int(scheme), kx, ky, s_xx, s_e)
            worst = max(worst, float(np.max(np.abs(np.linalg.eigvals(H)))))
    return worst
