"""Pins of the oracle's curved-wall closure (Sec. 3-b): virtual nodes
outside the fluid take u linearly extrapolated to zero at the wall along a
lattice link, from the first fluid node when the wall is at least half a
link away from it and from the second otherwise, and rho of the first.

- A straight channel written as a wall table reproduces the channel closure
  of Sec. 3-c (its own code path, pinned by the Poiseuille tests) to
  rounding.
- Stokes modes in a disk of radius 29.9 (Sec. 3-b, Table 2, nu_0 = 0.05)
  decay at nu a^2 / R^2, a a zero of J_1 (singlets) or J_{m+1} (doublets,
  scipy's Bessel zeros): within 0.4 % with five points, as Table 2 prints
  for that stencil, while three points err upward and more for higher
  modes, as Table 2 also prints.
- Reading an unused node is an error, not a silent value."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs


def _s(nu):
    return 1.0 / (3.0 * nu + 0.5)


@pytest.mark.parametrize("stencil", [3, 5, 9])
@pytest.mark.parametrize("xi", [0.25, 0.5, 0.8, 1.0])
def test_channel_table_equals_channel_closure(oracle, stencil, xi):
    nx, nyf, reach = 12, 10, 3
    walls = inputs.channel_walls(nx, nyf, xi, reach)
    d, ux, uy = inputs.random_fields(nx, nyf, 0.02, seed=4, rho_amp=0.01)
    force = (1e-5, 0.0)
    pw = oracle.params(nx, nyf, stencil, 1.7, 1.4, boundary=oracle.WALLS_Y, wall_xi=xi,
                       force=force)
    r1, x1, y1 = oracle.run(pw, 1 + d, ux, uy, 20)

    def pad(a, fill):
        return np.vstack([np.full((reach, nx), fill), a, np.full((reach, nx), fill)])

    pp = oracle.params(nx, nyf + 2 * reach, stencil, 1.7, 1.4, force=force)
    r2, x2, y2 = oracle.fd_run_walls(pp, walls, pad(1 + d, 1.0), pad(ux, 0.0), pad(uy, 0.0), 20)
    fl = slice(reach, reach + nyf)
    for a, b in ((r2[fl], r1), (x2[fl], x1), (y2[fl], y1)):
        assert np.abs(a - b).max() <= 1e-14


def disk_rate(oracle, stencil, nu, m, a, N=68, radius=29.9):
    """Decay rate of the Stokes mode (m, a) in the disk, from the projection
    of u on the initial mode over the fluid after n/2 and n steps."""
    walls = inputs.disk_walls(N, N, radius, reach=3)
    fluid = walls.kind == 0
    d, ux0, uy0 = inputs.stokes_disk_mode(N, N, radius, m, a, 1e-4)
    p = oracle.params(N, N, stencil, _s(nu), 1.5)
    n = int(2.0 / (nu * a * a / radius ** 2))
    r, x, y = oracle.fd_run_walls(p, walls, 1 + d, ux0, uy0, n // 2)
    a1 = ((x * ux0 + y * uy0)[fluid]).sum()
    r, x, y = oracle.fd_run_walls(p, walls, r, x, y, n - n // 2)
    a2 = ((x * ux0 + y * uy0)[fluid]).sum()
    return -np.log(a2 / a1) / (n - n // 2) * radius ** 2 / nu


def test_disk_stokes_modes():
    from scipy.special import jn_zeros
    from oracle import ref as oracle
    nu = 0.05
    modes = [(0, jn_zeros(1, 2)[0]), (0, jn_zeros(1, 2)[1]), (1, jn_zeros(2, 1)[0])]
    err5 = [disk_rate(oracle, 5, nu, m, a) / a ** 2 - 1 for m, a in modes]
    err3 = [disk_rate(oracle, 3, nu, m, a) / a ** 2 - 1 for m, a in modes]
    print("five points", np.round(err5, 5), "three points", np.round(err3, 5))
    assert max(abs(e) for e in err5) <= 0.004
    assert all(e > 0.004 for e in err3) and err3[1] > err3[0]


def test_reading_an_unused_node_is_an_error(oracle):
    """A wall table one node deep leaves the five-point stencil reading
    unused nodes."""
    N = 40
    walls = inputs.disk_walls(N, N, 15.0, reach=1)
    d, ux, uy = inputs.stokes_disk_mode(N, N, 15.0, 0, 3.8317, 1e-4)
    with pytest.raises(RuntimeError):
        oracle.fd_run_walls(oracle.params(N, N, 5, 1.7, 1.5), walls, 1 + d, ux, uy, 1)


def printed_tables_2_3():
    """Rows (table, kind, l, bessel, fd3, fd5) of Tables 2 and 3 as printed."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "tables2_3_stokes_disk.txt")
    rows = []
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            t, kind, l, b, e3, e5 = ln.split()
            rows.append((int(t), kind, int(l), float(b), float(e3), float(e5)))
    return rows


def test_bessel_column_is_the_mode_set():
    """The Bessel column of Tables 2 and 3 is a^2 for the singlets l = 1..6
    (a the l-th zero of J_1, stream function J_0) and for the doublets
    m = 1..11 (a the first zero of J_{m+1}, stream function J_m cos(m theta)):
    the modes that stokes_disk_mode builds.  Printed to 4-5 decimals."""
    from scipy.special import jn_zeros
    for t, kind, l, bessel, _, _ in printed_tables_2_3():
        a = jn_zeros(1, l)[l - 1] if kind == "singlet" else jn_zeros(l + 1, 1)[0]
        assert abs(a * a - bessel) <= 1e-4, (t, kind, l, a * a, bessel)
