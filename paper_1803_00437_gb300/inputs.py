"""Seeded synthetic inputs for the D2Q9 lattices: shear waves, transverse
Fourier ("Stokes") modes on periodic lattices and a channel at rest.

This module holds none of the scheme's arithmetic.  It only draws wave
vectors, amplitudes and phases and evaluates the initial primitive fields
(rho - 1, ux, uy) in FP64.  Both the CUDA path and the CPU oracle take their
inputs from here, so that they start from the same values.

Initial shear wave (Sec. 3-a): rho = 1 and a velocity
    u = A cos(k.x + phase) * (-ky/k, kx/k) + V * (kx/k, ky/k)
with k = 2 pi (m / nx, n / ny) for integers (m, n); the paper prints
cos(kx x + kx y), read here as cos(kx x + ky y).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Mode:
    m: int          # wave number along x: kx = 2 pi m / nx
    n: int          # wave number along y: ky = 2 pi n / ny
    amp: float      # velocity amplitude A
    phase: float    # phase in radians


def seed_for(config_index: int) -> int:
    """Fixed seed per workload: config index * 1000 + 17."""
    return int(config_index) * 1000 + 17


def transverse_modes(nx: int, ny: int, modes, mean_velocity=(0.0, 0.0)):
    """Sum of transverse plane waves; returns (drho, ux, uy) FP64 [ny][nx].

    Evaluated separably (cos(a + b) = cos a cos b - sin a sin b) so that
    lattices of 1e8 nodes take seconds."""
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    ux = np.full((ny, nx), float(mean_velocity[0]))
    uy = np.full((ny, nx), float(mean_velocity[1]))
    for md in modes:
        kx = 2.0 * np.pi * md.m / nx
        ky = 2.0 * np.pi * md.n / ny
        k = np.hypot(kx, ky)
        if k == 0.0:
            raise ValueError("a transverse mode needs a non-zero wave vector")
        a = kx * x
        b = ky * y + md.phase
        wave = np.outer(np.cos(b), np.cos(a)) - np.outer(np.sin(b), np.sin(a))
        ux += (-md.amp * ky / k) * wave
        uy += (md.amp * kx / k) * wave
    drho = np.zeros((ny, nx))
    return drho, ux, uy


def shear_wave(nx: int, ny: int, amp: float, m: int = 0, n: int = 1, phase: float = 0.0,
               mean_speed: float = 0.0):
    """One transverse wave with an optional uniform flow parallel to k."""
    kx = 2.0 * np.pi * m / nx
    ky = 2.0 * np.pi * n / ny
    k = np.hypot(kx, ky)
    V = (mean_speed * kx / k, mean_speed * ky / k)
    return transverse_modes(nx, ny, [Mode(m, n, amp, phase)], V)


def random_modes(nx: int, ny: int, n_modes: int, amp: float, seed: int, max_index: int = 32,
                 multiple_of: int = 1):
    """n_modes transverse modes with (m, n) drawn uniformly in
    |m|, |n| <= min(max_index, side / 4) (not both zero) and phase ~ U[0, 2 pi).
    With multiple_of > 1 the wave numbers are multiples of it (the field is
    then periodic with period side / multiple_of)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lim_x = max(1, min(max_index, nx // 4) // multiple_of)
    lim_y = max(1, min(max_index, ny // 4) // multiple_of)
    modes = []
    while len(modes) < n_modes:
        m = int(rng.integers(-lim_x, lim_x + 1)) * multiple_of
        n = int(rng.integers(-lim_y, lim_y + 1)) * multiple_of
        if m == 0 and n == 0:
            continue
        modes.append(Mode(m, n, float(amp), float(rng.uniform(0.0, 2.0 * np.pi))))
    return modes


def random_fields(nx: int, ny: int, amp: float, seed: int, rho_amp: float = 0.0):
    """Unstructured seeded noise (tests of the data path, not physics):
    drho ~ rho_amp * U[-1, 1], u ~ amp * U[-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    drho = rho_amp * rng.uniform(-1.0, 1.0, (ny, nx))
    ux = amp * rng.uniform(-1.0, 1.0, (ny, nx))
    uy = amp * rng.uniform(-1.0, 1.0, (ny, nx))
    return drho, ux, uy


def channel_at_rest(nx: int, ny: int):
    """Poiseuille channel start (Sec. 3-c): rho = 1, u = 0."""
    z = np.zeros((ny, nx))
    return z.copy(), z.copy(), z.copy()


def batch_lattices(count: int, seed: int, side_range=(32, 512), nu_range=(0.002, 0.1),
                   amp: float = 1e-3):
    """Independent periodic square lattices: side ~ U{lo..hi}, nu ~ U[lo, hi],
    each one transverse mode of random wave vector (|m|, |n| <= side / 4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        L = int(rng.integers(side_range[0], side_range[1] + 1))
        nu = float(rng.uniform(nu_range[0], nu_range[1]))
        lim = max(1, min(32, L // 4))
        while True:
            m = int(rng.integers(-lim, lim + 1))
            n = int(rng.integers(-lim, lim + 1))
            if m or n:
                break
        out.append((L, nu, Mode(m, n, amp, float(rng.uniform(0.0, 2.0 * np.pi)))))
    return out


# ---- curved walls (Sec. 3-b) ---------------------------------------------------------------

# D2Q9 links (Sec. 1): link a = 0..8 -> (cx, cy)
LINKS = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))


@dataclass(frozen=True)
class Walls:
    """Wall geometry of a lattice with solid regions, as the closure reads it.

    kind[j, i]: 0 fluid, 1 virtual (a solid node listed below), 2 unused
    (never read by the scheme).  Virtual node t sits at node[t] = j * nx + i;
    link[t] (1..8) is the lattice link along which the straight line from it
    reaches the fluid, and xi[t] the distance, in link lengths, from the first
    fluid node on that line back to the wall (0 < xi <= 1)."""
    kind: np.ndarray
    node: np.ndarray
    link: np.ndarray
    xi: np.ndarray


def disk_walls(nx: int, ny: int, radius: float, centre=None, reach: int = 3) -> Walls:
    """A disk of the given radius (lattice units) centred at `centre`
    (default: the middle of the lattice).  Nodes strictly inside are fluid;
    solid nodes within Chebyshev distance `reach` of a fluid node are virtual.
    For a virtual node the link is the one best aligned with the inward
    normal (the direction from the node to the centre): largest c.n / |c|.
    Walking from the node along it, the first fluid node is d links away and
    the circle crosses the line at t_w in (d - 1, d); xi = d - t_w."""
    cx0, cy0 = ((nx - 1) / 2.0, (ny - 1) / 2.0) if centre is None else centre
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    fluid = np.hypot(x - cx0, y - cy0) < radius
    if fluid[0, :].any() or fluid[-1, :].any() or fluid[:, 0].any() or fluid[:, -1].any():
        raise ValueError("the disk must not touch the lattice's edges")
    near = np.zeros_like(fluid)
    for dy in range(-reach, reach + 1):
        for dx in range(-reach, reach + 1):
            near |= np.roll(np.roll(fluid, dy, axis=0), dx, axis=1)
    virtual = near & ~fluid
    kind = np.where(fluid, 0, np.where(virtual, 1, 2)).astype(np.uint8)
    nodes, links, xis = [], [], []
    for j, i in zip(*np.nonzero(virtual)):
        n = np.array([cx0 - i, cy0 - j])
        n /= np.linalg.norm(n)
        a = max(range(1, 9), key=lambda b: (LINKS[b][0] * n[0] + LINKS[b][1] * n[1])
                / np.hypot(*LINKS[b]))
        ex, ey = LINKS[a]
        d = 1
        while not fluid[j + d * ey, i + d * ex]:
            d += 1
        # |(i, j) + t (ex, ey) - centre| = radius, smaller root
        qa = ex * ex + ey * ey
        qb = 2.0 * ((i - cx0) * ex + (j - cy0) * ey)
        qc = (i - cx0) ** 2 + (j - cy0) ** 2 - radius * radius
        tw = (-qb - np.sqrt(qb * qb - 4.0 * qa * qc)) / (2.0 * qa)
        xi = d - tw
        if not (0.0 < xi <= 1.0) or not fluid[j + (d + 1) * ey, i + (d + 1) * ex]:
            raise ValueError("disk too small for the closure's two fluid nodes")
        nodes.append(j * nx + i)
        links.append(a)
        xis.append(xi)
    return Walls(kind, np.array(nodes, np.int64), np.array(links, np.int8),
                 np.array(xis, np.float64))


def channel_walls(nx: int, ny_fluid: int, xi: float, reach: int = 3) -> Walls:
    """The channel of Sec. 3-c on a periodic lattice of ny_fluid + 2 reach
    rows: `reach` virtual rows below and above the fluid rows, whose lines
    reach the fluid along +y and -y, the walls xi below the first and above
    the last fluid row."""
    ny = ny_fluid + 2 * reach
    kind = np.zeros((ny, nx), np.uint8)
    kind[:reach] = 1
    kind[reach + ny_fluid:] = 1
    nodes, links = [], []
    for j in list(range(reach)) + list(range(reach + ny_fluid, ny)):
        for i in range(nx):
            nodes.append(j * nx + i)
            links.append(2 if j < reach else 4)
    return Walls(kind, np.array(nodes, np.int64), np.array(links, np.int8),
                 np.full(len(nodes), float(xi)))


def stokes_disk_mode(nx: int, ny: int, radius: float, m: int, a: float, amp: float,
                     centre=None):
    """Stokes mode of a disk (Sec. 3-b): stream function
    psi = [J_m(a r / R) - J_m(a) (r / R)^m] cos(m theta), with a a zero of
    J_1 for m = 0 (singlets) or of J_{m+1} for m > 0 (doublets), so that u = 0
    on r = R.  u_r = (1/r) d psi / d theta, u_theta = -d psi / dr, scaled to
    max |u| = amp over the fluid; zero outside.  Returns (drho, ux, uy)."""
    from scipy.special import jv
    cx0, cy0 = ((nx - 1) / 2.0, (ny - 1) / 2.0) if centre is None else centre
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    X, Y = x - cx0, y - cy0
    r = np.hypot(X, Y)
    th = np.arctan2(Y, X)
    s = a * r / radius
    dpsi_dr = a / radius * 0.5 * (jv(m - 1, s) - jv(m + 1, s))
    if m > 0:
        dpsi_dr = dpsi_dr - jv(m, a) * m * r ** (m - 1) / radius ** m
    radial = jv(m, s) - jv(m, a) * (r / radius) ** m
    ur = -m * radial * np.sin(m * th) / np.maximum(r, 1e-300)
    ut = -dpsi_dr * np.cos(m * th)
    ux = ur * np.cos(th) - ut * np.sin(th)
    uy = ur * np.sin(th) + ut * np.cos(th)
    fluid = r < radius
    scale = amp / np.hypot(ux, uy)[fluid].max()
    ux = np.where(fluid, ux * scale, 0.0)
    uy = np.where(fluid, uy * scale, 0.0)
    return np.zeros((ny, nx)), ux, uy
