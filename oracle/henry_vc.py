"""Vertex-centred variant of the FP64 oracle (test infrastructure only).

Paper section 2.3: the deterministic solver discretises Eqs. 1-2 with a
vertex-centred finite-volume scheme and partial upwinding of the convective
terms, first order in h + tau in practice (Eq. 1st_ord_conv). The paper
gives neither the scheme's formulas nor its upwind weights (they are
ug4's); this variant is this project's reading of them:

  * nodes (x_i, y_j) = (i hx, j hy), i = 0..nx, j = 0..ny of the level grid;
    the control volume of a node is its box [x_i - hx/2, x_i + hx/2] x
    [y_j - hy/2, y_j + hy/2] clipped to the domain; the box face between two
    neighbouring nodes is made of the two half-segments that lie in the two
    cells it crosses (one at the boundary);
  * the random field is evaluated at integration points, as the paper
    describes ("directly evaluated at the integration points"): at the
    midpoint of every face segment for the face coefficients, at the centre
    of every quarter-cell of a box for its storage;
  * fluxes between two nodes by two-point differences: volumetric flux
    Q = -T (p_U - p_L + rho_bar g d e_y), T = sum over segments K A_s/(mu d),
    diffusive conductance Dc = sum over segments phi A_s D / d, rho_bar the
    mean of the two nodes' densities;
  * partial upwind: the advected rho and rho c of a face are
    w a_L + (1 - w) a_U with w = (1 + alpha sgn(Q)) / 2 and the exponentially
    fitted weight alpha = coth(Pe/2) - 2/Pe of the face Peclet number
    Pe = |Q| / Dc (Allen and Southwell 1955, Il'in 1969): central as Pe -> 0,
    full upwind as Pe -> infinity, and nodally exact for one-dimensional
    steady advection-diffusion with constant coefficients;
  * boundary conditions as section 2.1 states them: the right column x = Lx
    is Dirichlet, p = rho1 g (Ly - y), c = 1 (boundary data, not unknowns);
    the left column has c = 0 (a Dirichlet row, scaled by V phi0 rho0 /
    tau) and the fresh-water mass inflow rho0 q_in through its box face; top
    and bottom are closed.

Unknowns: p and c at the nodes i = 0..nx-1, j = 0..ny, arrays [ny+1, nx].
Jacobians by complex step and Newton with sparse LU, as in oracle.henry.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import henry as H

_CS_H = 1e-30


@dataclass
class VFields:
    """Coefficients of the vertex-centred scheme on the unknown nodes."""
    vphi: np.ndarray   # [ny+1, nx] integral of phi over each box
    vol: np.ndarray    # [ny+1, nx] box areas
    tx: np.ndarray     # [ny+1, nx] T of the face to the east neighbour (i = nx-1: to x = Lx)
    dx: np.ndarray     # [ny+1, nx] diffusive conductance of that face
    ty: np.ndarray     # [ny, nx] T of the face to the north neighbour
    dy: np.ndarray     # [ny, nx]
    qin: np.ndarray    # [ny+1] fresh-water inflow through each left box face [m^2/s]
    vphi_r: np.ndarray  # [ny+1] box integral of phi of the Dirichlet column (QoIs)


def nodes(grid: H.Grid, phys: H.Physics):
    hx, hy = grid.lengths(phys)
    return np.arange(grid.nx + 1) * hx, np.arange(grid.ny + 1) * hy


def _segments(n, h, L):
    """Per node k = 0..n of a 1-D node row: the two half-segments of its box,
    as (lower, upper) midpoints and lengths (0 where clipped)."""
    x = np.arange(n + 1) * h
    lo_len = np.where(np.arange(n + 1) > 0, h / 2, 0.0)
    hi_len = np.where(np.arange(n + 1) < n, h / 2, 0.0)
    return x - h / 4, lo_len, x + h / 4, hi_len


def vfields(grid: H.Grid, phys: H.Physics, xi) -> VFields:
    xi = np.asarray(xi)
    nx, ny = grid.nx, grid.ny
    hx, hy = grid.lengths(phys)
    xs_lo, xl_lo, xs_hi, xl_hi = _segments(nx, hx, phys.Lx)
    ys_lo, yl_lo, ys_hi, yl_hi = _segments(ny, hy, phys.Ly)

    def f(X, Y):
        return H.field_at(phys, xi, X, Y)

    # storage: four quarter-cells per box, phi at each quarter's centre
    vphi = np.zeros((ny + 1, nx + 1), dtype=np.result_type(xi, float))
    vol = np.zeros((ny + 1, nx + 1))
    for xc, xl in ((xs_lo, xl_lo), (xs_hi, xl_hi)):
        for yc, yl in ((ys_lo, yl_lo), (ys_hi, yl_hi)):
            X, Y = np.meshgrid(xc, yc)
            A = np.outer(yl, xl)
            vphi = vphi + f(X, Y)[0] * A
            vol = vol + A
    # east faces of nodes i = 0..nx-1: x = x_i + hx/2, segments below and above y_j
    xf = (np.arange(nx) + 0.5) * hx
    tx = np.zeros((ny + 1, nx), dtype=vphi.dtype)
    dxc = np.zeros((ny + 1, nx), dtype=vphi.dtype)
    for yc, yl in ((ys_lo, yl_lo), (ys_hi, yl_hi)):
        X, Y = np.meshgrid(xf, yc)
        phi, K = f(X, Y)
        tx = tx + K * yl[:, None] / (phys.mu * hx)
        dxc = dxc + phi * yl[:, None] * phys.D / hx
    # north faces of rows j = 0..ny-1 (nodes i = 0..nx-1): y = y_j + hy/2
    yf = (np.arange(ny) + 0.5) * hy
    ty = np.zeros((ny, nx), dtype=vphi.dtype)
    dyc = np.zeros((ny, nx), dtype=vphi.dtype)
    for xc, xl in ((xs_lo[:nx], xl_lo[:nx]), (xs_hi[:nx], xl_hi[:nx])):
        X, Y = np.meshgrid(xc, yf)
        phi, K = f(X, Y)
        ty = ty + K * xl[None, :] / (phys.mu * hy)
        dyc = dyc + phi * xl[None, :] * phys.D / hy
    # inflow through the left box faces: q_in at the segment midpoints
    qin = H.inflow_at(phys, xi, ys_lo) * yl_lo + H.inflow_at(phys, xi, ys_hi) * yl_hi
    return VFields(vphi=vphi[:, :nx], vol=vol[:, :nx], tx=tx, dx=dxc, ty=ty, dy=dyc, qin=qin,
                   vphi_r=vphi[:, nx])


def fitted_alpha(Pe):
    """alpha(Pe) = coth(Pe/2) - 2/Pe for Pe >= 0 (alpha(0) = 0). Below
    Pe = 1e-2 its Taylor series Pe/6 - Pe^3/360 + Pe^5/15120 - Pe^7/604800
    (the direct form loses digits to cancellation there; the next term is
    below 1e-25). Complex arguments are allowed (complex step)."""
    Pe = np.asarray(Pe)
    small = np.abs(np.real(Pe)) < 1e-2
    Ps = np.where(small, Pe, 0.0)
    P2 = Ps * Ps
    series = Ps * (1.0 / 6 - P2 * (1.0 / 360 - P2 * (1.0 / 15120 - P2 / 604800)))
    Pl = np.where(small, 1.0, Pe)
    direct = 1.0 / np.tanh(0.5 * Pl) - 2.0 / Pl
    return np.where(small, series, direct)


def _adv_weight(Q, Dc):
    """w of the partial upwind value w a_L + (1 - w) a_U. The sign of Q
    decides on its real part (frozen under complex-step differentiation);
    without diffusion (Dc = 0) the weight is full upwind."""
    s = np.where(np.real(Q) >= 0, 1.0, -1.0)
    diff = np.real(Dc) > 0
    Pe = Q * s / np.where(diff, Dc, 1.0)
    alpha = np.where(diff, fitted_alpha(Pe), 1.0)
    return 0.5 * (1.0 + alpha * s)


def _face(phys, Q_or_none, T, Dc, pL, cL, pU, cU, gd):
    """Mass and salt flux from L to U through one face (arrays)."""
    drho = phys.rho1 - phys.rho0
    rL = phys.rho0 + drho * cL
    rU = phys.rho0 + drho * cU
    rbar = 0.5 * (rL + rU)
    Q = -T * (pU - pL + rbar * gd) if Q_or_none is None else Q_or_none
    w = _adv_weight(Q, Dc)
    Fm = Q * (w * rL + (1.0 - w) * rU)
    Fs = Q * (w * rL * cL + (1.0 - w) * rU * cU) - Dc * rbar * (cU - cL)
    return Q, Fm, Fs


def right_pressure(grid, phys):
    _, y = nodes(grid, phys)
    return phys.rho1 * phys.g * (phys.Ly - y)


def face_fluxes(grid, phys, vf: VFields, p, c):
    """Mass and salt fluxes through every box face (east faces [ny+1, nx],
    the last column to the Dirichlet column; north faces [ny, nx]; left
    inflow [ny+1])."""
    hx, hy = grid.lengths(phys)
    pR = right_pressure(grid, phys)[:, None]
    pE = np.concatenate([p[:, 1:], pR + 0.0 * p[:, :1]], axis=1)
    cE = np.concatenate([c[:, 1:], 1.0 + 0.0 * c[:, :1]], axis=1)
    Qx, Fmx, Fsx = _face(phys, None, vf.tx, vf.dx, p, c, pE, cE, 0.0)
    Qy, Fmy, Fsy = _face(phys, None, vf.ty, vf.dy, p[:-1], c[:-1], p[1:], c[1:], phys.g * hy)
    return {"Qx": Qx, "mass_x": Fmx, "salt_x": Fsx, "Qy": Qy, "mass_y": Fmy, "salt_y": Fsy,
            "mass_left": -phys.rho0 * vf.qin}


def residual(grid, phys, vf: VFields, p, c, c_old):
    """(R_p, R_c), each [ny+1, nx]: box balances of Eqs. 1-2 over one
    implicit Euler step; the left column's R_c is the Dirichlet row
    (V phi0 rho0 / tau) c."""
    tau = grid.tau
    drho = phys.rho1 - phys.rho0
    rho = phys.rho0 + drho * c
    rho_o = phys.rho0 + drho * c_old
    dt = np.result_type(p, c, c_old, vf.vphi, vf.tx)
    Rp = (vf.vphi * (rho - rho_o) / tau).astype(dt)
    Rc = (vf.vphi * (rho * c - rho_o * c_old) / tau).astype(dt)
    F = face_fluxes(grid, phys, vf, p, c)
    Rp = Rp + F["mass_x"]
    Rp[:, 1:] -= F["mass_x"][:, :-1]
    Rc = Rc + F["salt_x"]
    Rc[:, 1:] -= F["salt_x"][:, :-1]
    Rp[:-1] += F["mass_y"]
    Rp[1:] -= F["mass_y"]
    Rc[:-1] += F["salt_y"]
    Rc[1:] -= F["salt_y"]
    Rp[:, 0] += F["mass_left"]
    Rc[:, 0] = vf.vol[:, 0] * phys.phi0 * phys.rho0 / tau * c[:, 0]
    return Rp, Rc


def jacobian(grid, phys, vf, p, c, c_old):
    """Exact Jacobian by complex step, interleaved unknowns (as oracle.henry)."""
    ny1, nx = p.shape
    jj, ii = np.mgrid[0:ny1, 0:nx]
    colour = (ii + 2 * jj) % 5
    rows, cols, vals = [], [], []
    for col in range(5):
        mask = colour == col
        Pj, Pi = np.nonzero(mask)
        for var in (0, 1):
            pz = p.astype(complex)
            cz = c.astype(complex)
            if var == 0:
                pz = pz + 1j * _CS_H * mask
            else:
                cz = cz + 1j * _CS_H * mask
            Rp, Rc = residual(grid, phys, vf, pz, cz, c_old)
            dRp, dRc = Rp.imag / _CS_H, Rc.imag / _CS_H
            for dj, di in H._STENCIL:
                Qj, Qi = Pj + dj, Pi + di
                ok = (Qj >= 0) & (Qj < ny1) & (Qi >= 0) & (Qi < nx)
                pc = Pj[ok] * nx + Pi[ok]
                qc = Qj[ok] * nx + Qi[ok]
                rows += [2 * qc, 2 * qc + 1]
                cols += [2 * pc + var, 2 * pc + var]
                vals += [dRp[Qj[ok], Qi[ok]], dRc[Qj[ok], Qi[ok]]]
    n = 2 * nx * ny1
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def initial_state(grid, phys):
    """c = 0; Newton guess p = seawater hydrostatics at the nodes."""
    pR = right_pressure(grid, phys)
    return np.repeat(pR[:, None], grid.nx, axis=1), np.zeros((grid.ny + 1, grid.nx))


def newton_step(grid, phys, vf, p, c, c_old, maxit=30, tol_c=1e-12, tol_p_rel=1e-12):
    """One implicit step by Newton from (p, c): stops when the update is
    below tol_c in c and tol_p_rel times the seawater pressure scale rho1 g
    Ly (at least 1 Pa, so that gravity-free cases stop too)."""
    p = p.copy()
    c = c.copy()
    pscale = max(phys.rho1 * phys.g * phys.Ly, 1.0)
    for it in range(1, maxit + 1):
        Rp, Rc = residual(grid, phys, vf, p, c, c_old)
        J = jacobian(grid, phys, vf, p, c, c_old)
        d = spla.spsolve(J, -H.interleave(Rp, Rc))
        dp = d[0::2].reshape(p.shape)
        dc = d[1::2].reshape(c.shape)
        p += dp
        c += dc
        if np.max(np.abs(dc)) <= tol_c and np.max(np.abs(dp)) <= tol_p_rel * pscale:
            return p, c, it
    raise RuntimeError("vertex-centred oracle Newton did not converge")


def solve(grid, phys, xi, c0=None, p0=None, keep_states=False):
    """Implicit Euler time loop from c = 0 (or c0). With the paper's field
    model the inflow of step n carries (1 + sin(pi t / 40)) at t = n tau, as
    in oracle.henry.solve."""
    import dataclasses
    import math
    vf = vfields(grid, phys, xi)
    p, c = initial_state(grid, phys)
    if c0 is not None:
        c = np.array(c0, dtype=float)
    if p0 is not None:
        p = np.array(p0, dtype=float)
    its = []
    states = [(p.copy(), c.copy())] if keep_states else None
    for n in range(grid.nt):
        vn = vf
        if phys.field_model == 1:
            t = (n + 1) * grid.tau
            vn = dataclasses.replace(vf, qin=vf.qin * (1.0 + math.sin(math.pi * t / 40.0)))
        p, c, it = newton_step(grid, phys, vn, p, c, c.copy())
        its.append(it)
        if keep_states:
            states.append((p.copy(), c.copy()))
    return {"p": p, "c": c, "its": its, "vfields": vf, "states": states}


def full_nodes(grid, phys, c):
    """Nodal c on every node [ny+1, nx+1] (the Dirichlet column c = 1 added)."""
    return np.concatenate([c, np.ones((grid.ny + 1, 1))], axis=1)


def qoi(grid, phys, vf: VFields, c):
    """The 22 QoIs of oracle.henry.qoi with c a nodal field: integrals by the
    box rule (c constant on each box, the Dirichlet column included), point
    values by bilinear interpolation of the nodal values."""
    hx, hy = grid.lengths(phys)
    cf = full_nodes(grid, phys, c)
    x, y = nodes(grid, phys)
    xl = np.clip(x - hx / 2, 0.0, phys.Lx)
    xr = np.clip(x + hx / 2, 0.0, phys.Lx)
    yb = np.clip(y - hy / 2, 0.0, phys.Ly)
    yt = np.clip(y + hy / 2, 0.0, phys.Ly)
    V = np.outer(yt - yb, xr - xl)
    vphi = np.concatenate([vf.vphi, vf.vphi_r[:, None]], axis=1)
    rho = phys.rho0 + (phys.rho1 - phys.rho0) * cf
    out = [np.sum(V * cf * rho), np.sum(vphi * rho * cf), np.sum(V * cf * (phys.Lx - x)[None, :])]
    for px, py in H.OBS_POINTS:
        i0 = int(min(max(np.floor(px / hx), 0), grid.nx - 1))
        j0 = int(min(max(np.floor(py / hy), 0), grid.ny - 1))
        tx = px / hx - i0
        ty = py / hy - j0
        out.append((1 - tx) * (1 - ty) * cf[j0, i0] + tx * (1 - ty) * cf[j0, i0 + 1]
                   + (1 - tx) * ty * cf[j0 + 1, i0] + tx * ty * cf[j0 + 1, i0 + 1])
    out.append(float(np.sum(V * (cf <= H.FRESH_C))))
    for px, py in H.POINTS15:
        ox = np.clip(np.minimum(xr, px + H.BOX_HALF) - np.maximum(xl, px - H.BOX_HALF), 0.0, None)
        oy = np.clip(np.minimum(yt, py + H.BOX_HALF) - np.maximum(yb, py - H.BOX_HALF), 0.0, None)
        out.append(float(np.sum(cf * rho * oy[:, None] * ox[None, :])))
    return np.array(out)
