"""Discrete adjoint of a QoI through the implicit Euler time stepping
(test infrastructure only).

With R^n(u^n, u^{n-1}; theta) = 0 the residual of step n (oracle.henry)
and Q = Q(u^r), the Lagrangian Q - sum_n lam_n^T R^n gives
    J_r^T lam_r = dQ/du^r,
    J_n^T lam_n = -(dR^{n+1}/du^n)^T lam_{n+1},   n = r-1, ..., 1,
    dQ/dtheta   = -sum_n (dR^n/dtheta)^T lam_n,
J_n = dR^n/du^n. Every partial derivative here is a complex-step
derivative of the oracle's residual, fields or QoI integrand, so nothing is
shared with a hand-derived adjoint. Parameters: xi (through the random
fields) and a per-cell log-permeability perturbation theta.

QoIs: "Q_S" = int c rho dx (section 4, Eq. integral_s) and "toe" =
int c (Lx - x) dx.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from oracle import henry as H

_H = 1e-30


def qoi_integrand(name, grid, phys, c):
    """Per-cell integrand of the QoI (sum over cells = Q)."""
    hx, hy = grid.lengths(phys)
    V = hx * hy
    if name == "Q_S":
        rho = phys.rho0 + (phys.rho1 - phys.rho0) * c
        return c * rho * V
    if name == "toe":
        x, _ = H.cell_centres(grid, phys)
        return c * (phys.Lx - x)[None, :] * V
    raise ValueError(name)


def qoi_value(name, grid, phys, c):
    return float(np.sum(qoi_integrand(name, grid, phys, c)))


def _step_fields(grid, phys, f, n):
    """Fields of step n (1-based): with the paper's model the inflow carries
    the recharge factor (1 + sin(pi t / 40)) at t = n tau (as oracle.henry.solve)."""
    if phys.field_model != 1:
        return f
    fac = 1.0 + np.sin(np.pi * n * grid.tau / 40.0)
    return H.Fields(phi=f.phi, K=f.K, qin=f.qin * fac)


def adjoint(grid, phys, xi, qoi="Q_S", logk=None):
    """Returns dict(q, dq_dxi [n_xi], dq_dlogk [ny, nx], lam (per step))."""
    xi = np.asarray(xi, dtype=float)
    ny, nx = grid.ny, grid.nx
    lk = np.zeros((ny, nx)) if logk is None else np.asarray(logk, dtype=float)
    fwd = H.solve(grid, phys, xi, lk, keep_states=True)
    f = fwd["fields"]
    states = fwd["states"]
    r = grid.nt
    # dQ/du^r: only c enters the QoI
    gc = qoi_integrand(qoi, grid, phys, states[r][1] + 1j * _H).imag / _H
    rhs = H.interleave(np.zeros((ny, nx)), gc)
    jj, ii = np.mgrid[0:ny, 0:nx]
    colour = (ii + 2 * jj) % 5
    dq_dxi = np.zeros(xi.shape[0])
    dq_dlogk = np.zeros((ny, nx))
    lams = {}
    lam_next = None
    for n in range(r, 0, -1):
        p_n, c_n = states[n]
        c_prev = states[n - 1][1]
        if n < r:
            # -(dR^{n+1}/du^n)^T lam_{n+1}: R^{n+1} sees u^n through c_old only,
            # cell by cell (diagonal), so one complex step gives it
            p1, c1 = states[n + 1]
            Rp, Rc = H.residual(grid, phys, _step_fields(grid, phys, f, n + 1), p1, c1,
                                c_n + 1j * _H)
            dp, dc = Rp.imag / _H, Rc.imag / _H
            lp, lc = lam_next[0::2].reshape(ny, nx), lam_next[1::2].reshape(ny, nx)
            rhs = H.interleave(np.zeros((ny, nx)), -(dp * lp + dc * lc))
        Jn = H.jacobian(grid, phys, _step_fields(grid, phys, f, n), p_n, c_n, c_prev)
        lam = spla.spsolve(Jn.T.tocsc(), rhs)
        lams[n] = lam
        lp, lc = lam[0::2].reshape(ny, nx), lam[1::2].reshape(ny, nx)
        # xi: complex step through the fields
        for j in range(xi.shape[0]):
            xz = xi.astype(complex)
            xz[j] += 1j * _H
            fz = _step_fields(grid, phys, H.fields(grid, phys, xz, lk), n)
            Rp, Rc = H.residual(grid, phys, fz, p_n, c_n, c_prev)
            dq_dxi[j] -= np.sum(lp * Rp.imag / _H + lc * Rc.imag / _H)
        # per-cell log K: coloured complex steps (theta_P reaches the
        # residual of P and its four neighbours only)
        for col in range(5):
            mask = colour == col
            fz = _step_fields(grid, phys, H.fields(grid, phys, xi, lk + 1j * _H * mask), n)
            Rp, Rc = H.residual(grid, phys, fz, p_n, c_n, c_prev)
            w = lp * Rp.imag / _H + lc * Rc.imag / _H          # lam_Q dR_Q / dtheta_P
            Pj, Pi = np.nonzero(mask)
            acc = np.zeros(Pj.shape[0])
            for dj, di in ((0, 0), (0, -1), (0, 1), (-1, 0), (1, 0)):
                Qj, Qi = Pj + dj, Pi + di
                ok = (Qj >= 0) & (Qj < ny) & (Qi >= 0) & (Qi < nx)
                acc[ok] += w[Qj[ok], Qi[ok]]
            dq_dlogk[Pj, Pi] -= acc
        lam_next = lam
    return {"q": qoi_value(qoi, grid, phys, states[r][1]), "dq_dxi": dq_dxi,
            "dq_dlogk": dq_dlogk, "lam": lams}


def forward_qoi(grid, phys, xi, qoi="Q_S", logk=None):
    r = H.solve(grid, phys, np.asarray(xi, dtype=float), logk)
    return qoi_value(qoi, grid, phys, r["c"])
