"""Helpers shared by the GPU parity tests: run the CUDA library and the FP64
oracle from the same seeded inputs and compare element by element."""
import numpy as np

from paper_1803_00437_gb300 import inputs

SCHEME_TO_ORACLE = {"fd3": 3, "fd5": 5, "fd9": 9, "mrt": 100, "lwacm": 200}
BOUNDARY_TO_ORACLE = {"periodic": 0, "walls_y": 1}


def as_f32(fields):
    """Round the FP64 inputs to FP32 once; both sides start from these."""
    return tuple(np.asarray(f, dtype=np.float32) for f in fields)


def gpu_run(cfg, fields32, nsteps, stream=None):
    import torch
    from paper_1803_00437_gb300 import fdlbm as F
    lat = F.Lattice(cfg, stream=stream)
    dev = [torch.from_numpy(np.ascontiguousarray(f)).to(lat.device) for f in fields32]
    lat.init(*dev)
    lat.step(nsteps)
    out = [t.cpu().numpy().astype(np.float64) for t in lat.moments()]
    torch.cuda.synchronize()
    return out, lat


def quartic_s_q(s_xx):
    """Eq. sigsig (Sec. 3-b): (1/s_xx - 1/2)(1/s_q - 1/2) = 1/6, the rate the
    library takes for MRT when s_q is left to it (FDLBM_S_Q_QUARTIC)."""
    return 1.0 / (1.0 / (6.0 * (1.0 / s_xx - 0.5)) + 0.5)


def oracle_params(oracle, cfg):
    s_q = cfg.s_q if cfg.s_q is not None else quartic_s_q(cfg.s_xx)
    return oracle.params(cfg.nx, cfg.ny, SCHEME_TO_ORACLE[cfg.scheme], cfg.s_xx, cfg.s_e, s_q,
                         cfg.s_eps, boundary=BOUNDARY_TO_ORACLE[cfg.boundary],
                         wall_xi=cfg.wall_xi, force=cfg.force)


def oracle_run(oracle, cfg, fields32, nsteps):
    d, x, y = (f.astype(np.float64) for f in fields32)
    p = oracle_params(oracle, cfg)
    r, ux, uy = oracle.run(p, 1.0 + d, x, y, nsteps)
    return [r - 1.0, ux, uy]


def max_err(gpu, ref, scale):
    return max(float(np.abs(g - r).max()) for g, r in zip(gpu, ref)) / scale


def amplitude(fields):
    return max(float(np.abs(fields[1]).max()), float(np.abs(fields[2]).max()))
