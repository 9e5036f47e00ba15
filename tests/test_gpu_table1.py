"""Table 1 (Sec. 3-a) measured on the streaming FD-LBM kernel: the shear
hyperviscosity nu_2 of the three- and five-point stencils at s_xx = 1.85,
along 0, 26.6 and 45 degrees, from the decay of single transverse waves.

Each wave u = A e_perp cos(k.x) (A = 1e-4, rho = 1) runs on a 256 x ny
periodic lattice (the streaming kernel's shape) with (m, n) chosen so that
|k| spans 0.1 ... 0.35 along the angle; its amplitude is the FP64 projection
of u.e_perp on exp(i k.x), taken after steps // 5 steps and after `steps`
steps (a decay of e^-1.5), and Gamma = -log(a2 / a1) / (steps - steps // 5).

Checks:
- every Gamma equals the shear root of the step's Fourier symbol H(k)
  (oracle.linear) to 2e-5 relative.  Taking the rate between two times
  biases it by under 1e-7 (the initial wave is the shear eigenvector to
  that order), so the bound covers FP32 rounding only;
- nu_2 from a least-squares fit Gamma / k^2 - nu_0 = nu_2 k^2 + nu_4 k^4 +
  nu_6 k^6 (nu_0 = (1/s_xx - 1/2)/3, Sec. 1-a) equals the symbol's nu_2 to
  5e-5.  A relative error e in the rates moves the fit by at most 1.7 e;
- and the value printed in Table 1 to 1e-4.  That bound includes the
  printed rounding and the 2e-5 between 26.6 degrees and the lattice's
  atan(1/2) = 26.565 degrees.

The nine-point column is not measured: at s_xx = 1.85 that stencil is
linearly unstable (Sec. 3-a), so a decay cannot be followed for thousands of
steps (test_gpu_fd9 measures its growth instead)."""
import os

import numpy as np
import pytest

from paper_1803_00437_gb300 import inputs
from parity_util import as_f32

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
S_XX, NX, AMP = 1.85, 256, 1e-4
# (m, n, ny): wave vector 2 pi (m / 256, n / ny) along the angle
SETS = {
    0.0: [(4, 0, 16), (6, 0, 16), (8, 0, 16), (11, 0, 16), (14, 0, 16)],
    26.6: [(4, 1, 128), (6, 3, 256), (8, 1, 64), (10, 5, 256), (12, 3, 128)],
    45.0: [(3, 3, 256), (4, 1, 64), (5, 5, 256), (6, 3, 128), (8, 1, 32), (10, 5, 128)],
}


def _printed(angle, stencil):
    rows = [ln.split() for ln in open(os.path.join(ROOT, "tests", "golden",
                                                   "table1_hyperviscosity.txt"))
            if ln.strip() and not ln.startswith("#")]
    col = {"fd3": 1, "fd5": 2}[stencil]
    return next(float(r[col]) for r in rows if abs(float(r[0]) - angle) < 1e-9)


def _gpu_rate(scheme, m, n, ny, steps):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    cfg = F.LatticeConfig(NX, ny, scheme, s_xx=S_XX, s_e=1.5, flags=F.FLAG_STREAM)
    lat = F.Lattice(cfg)
    f = as_f32(inputs.shear_wave(NX, ny, AMP, m=m, n=n))
    lat.init(*[torch.from_numpy(np.ascontiguousarray(a)).to(lat.device) for a in f])
    n1 = steps // 5
    lat.step(n1)
    a1 = float(np.hypot(*lat.reduce("mode", [m, n])))
    lat.step(steps - n1)
    a2 = float(np.hypot(*lat.reduce("mode", [m, n])))
    lat.close()
    return -np.log(a2 / a1) / (steps - n1)


@pytest.mark.parametrize("angle", sorted(SETS))
@pytest.mark.parametrize("stencil", ["fd3", "fd5"])
def test_table1_on_the_streaming_kernel(stencil, angle):
    from oracle import linear
    nu0 = (1 / S_XX - 0.5) / 3
    ks, rates, phi = [], [], 0.0
    for m, n, ny in SETS[angle]:
        kx, ky = 2 * np.pi * m / NX, 2 * np.pi * n / ny
        k, phi = np.hypot(kx, ky), np.arctan2(ky, kx)
        steps = int(1.5 / (nu0 * k * k))
        g = _gpu_rate(stencil, m, n, ny, steps)
        g_sym = linear.shear_gamma(stencil[-1], k, phi, S_XX)
        print(f"{stencil} {angle:4.1f} deg  k {k:.4f}  Gamma GPU {g:.9e}  symbol {g_sym:.9e}  "
              f"rel {g / g_sym - 1:+.2e}")
        assert abs(g / g_sym - 1) <= 2e-5, (k, g, g_sym)
        ks.append(k)
        rates.append(g)
    ks, rates = np.array(ks), np.array(rates)
    A = np.stack([ks ** 2, ks ** 4, ks ** 6], axis=1)
    nu2 = float(np.linalg.lstsq(A, rates / ks ** 2 - nu0, rcond=None)[0][0])
    nu2_sym = linear.viscosity_expansion(stencil[-1], phi, S_XX)[1]
    printed = _printed(angle, stencil)
    print(f"{stencil} {angle:4.1f} deg  nu_2 GPU {nu2:.6f}  symbol {nu2_sym:.6f}  "
          f"Table 1 {printed:.5f}")
    assert abs(nu2 - nu2_sym) <= 5e-5
    assert abs(nu2 - printed) <= 1e-4
