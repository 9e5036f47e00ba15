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
