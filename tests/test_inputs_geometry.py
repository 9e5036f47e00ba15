"""The wall geometry and Stokes modes of the input generator (Sec. 3-b),
checked against their definitions: the disk's wall table describes the
circle, and the modes satisfy the no-slip condition and incompressibility
that define them."""
import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs


@pytest.mark.parametrize("N,radius,reach", [(68, 29.9, 3), (40, 15.0, 2), (41, 17.3, 3)])
def test_disk_wall_table_describes_the_circle(N, radius, reach):
    w = inputs.disk_walls(N, N, radius, reach=reach)
    c = (N - 1) / 2.0
    y, x = np.mgrid[0:N, 0:N].astype(float)
    r = np.hypot(x - c, y - c)
    assert np.array_equal(w.kind == 0, r < radius)
    # virtual nodes: solid, within the reach of a fluid node, listed once
    assert len(np.unique(w.node)) == len(w.node) == int((w.kind == 1).sum())
    assert np.all(w.kind.ravel()[w.node] == 1)
    for n, a, xi in zip(w.node, w.link, w.xi):
        j, i = divmod(int(n), N)
        ex, ey = inputs.LINKS[a]
        d = 1
        while w.kind[j + d * ey, i + d * ex] != 0:
            d += 1
        assert d <= reach + 1 and 0.0 < xi <= 1.0
        # the wall sits xi links before the first fluid node on the line
        tw = d - xi
        assert abs(np.hypot(i + tw * ex - c, j + tw * ey - c) - radius) < 1e-9
        # the link is the one best aligned with the inward normal
        nrm = np.array([c - i, c - j]) / np.hypot(c - i, c - j)
        score = [(inputs.LINKS[b][0] * nrm[0] + inputs.LINKS[b][1] * nrm[1])
                 / np.hypot(*inputs.LINKS[b]) for b in range(1, 9)]
        assert score[a - 1] >= max(score) - 1e-12
    # no unused node within the reach of the fluid
    fluid = w.kind == 0
    for dy in range(-reach, reach + 1):
        for dx in range(-reach, reach + 1):
            near = np.roll(np.roll(fluid, dy, 0), dx, 1)
            assert not np.any(near & (w.kind == 2))


def test_channel_wall_table():
    w = inputs.channel_walls(8, 10, 0.3, reach=3)
    assert w.kind.shape == (16, 8)
    assert np.all(w.kind[3:13] == 0) and np.all(w.kind[:3] == 1) and np.all(w.kind[13:] == 1)
    rows = w.node // 8
    assert np.all(w.link[rows < 3] == 2) and np.all(w.link[rows >= 13] == 4)
    assert np.all(w.xi == 0.3)


@pytest.mark.parametrize("m,zero", [(0, (1, 1)), (0, (1, 3)), (1, (2, 1)), (3, (4, 1))])
def test_stokes_modes_no_slip_and_divergence_free(m, zero):
    """u vanishes on r = R (a is a zero of J_1 for m = 0, of J_{m+1} for
    m > 0) and is divergence-free: near the wall |u| falls linearly, and the
    centred discrete divergence in the interior is O(h^2) of |u| / R."""
    from scipy.special import jn_zeros
    N, R = 161, 75.0
    a = jn_zeros(zero[0], zero[1])[-1]
    d, ux, uy = inputs.stokes_disk_mode(N, N, R, m, a, 1.0)
    c = (N - 1) / 2.0
    y, x = np.mgrid[0:N, 0:N].astype(float)
    r = np.hypot(x - c, y - c)
    assert np.abs(d).max() == 0.0
    speed = np.hypot(ux, uy)
    shell = (r < R) & (r > R - 1.0)
    assert speed[shell].max() < 4.0 * a * 1.0 / R  # |u| <= |u'| * distance, |u'| ~ a / R
    inner = r < R - 3.0
    div = 0.5 * (np.roll(ux, -1, 1) - np.roll(ux, 1, 1)) + 0.5 * (np.roll(uy, -1, 0) - np.roll(uy, 1, 0))
    assert np.abs(div[inner]).max() < 0.05 * (a / R) ** 2
