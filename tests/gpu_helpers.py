"""Shared helpers of the GPU tests: config <-> oracle parameters, cached
oracle solves. Imports the oracle (test infrastructure) and the binding."""
import functools

import numpy as np

from oracle import henry as H
from paper_2403_17018_gb300 import binding as hb
from paper_2403_17018_gb300.inputs import xi_batch


def oracle_physics(cfg) -> H.Physics:
    return H.Physics(rho0=cfg.rho0, rho1=cfg.rho1, mu=cfg.mu, g=cfg.g, D=cfg.D, K0=cfg.K0,
                     phi0=cfg.phi0, q0=cfg.q0, Lx=cfg.Lx, Ly=cfg.Ly,
                     field_model=cfg.field_model)


def oracle_grid(cfg, level) -> H.Grid:
    return H.Grid(nx=cfg.nx0 << level, ny=cfg.ny0 << level, nt=cfg.nt0 << level, T=cfg.T)


@functools.lru_cache(maxsize=None)
def _oracle_solve_cached(key):
    (nx0, ny0, nt0, T, level, xi_t, phys_t) = key
    ph = H.Physics(*phys_t)
    g = H.Grid(nx=nx0 << level, ny=ny0 << level, nt=nt0 << level, T=T)
    r = H.solve(g, ph, np.array(xi_t))
    return r["p"], r["c"], H.qoi(g, ph, r["fields"], r["c"])


def oracle_solve(cfg, level, xi):
    """(p, c, q) of the oracle for one sample (cached by value)."""
    ph = oracle_physics(cfg)
    phys_t = (ph.rho0, ph.rho1, ph.mu, ph.g, ph.D, ph.K0, ph.phi0, ph.q0, ph.Lx, ph.Ly,
              ph.field_model)
    key = (cfg.nx0, cfg.ny0, cfg.nt0, cfg.T, level, tuple(float(v) for v in xi), phys_t)
    return _oracle_solve_cached(key)


def tight_config(**kw):
    """Config whose Newton tolerance sits well below the parity bar."""
    base = dict(newton_rtol=1e-12, newton_atol=3e-13, newton_maxit=60, newton_stag_tol=1e-11)
    base.update(kw)
    return hb.default_config(**base)


def xi_cuda(level, first, count, n_xi=3):
    import torch
    return torch.from_numpy(xi_batch(level, first, count, n_xi=n_xi)).cuda()
