"""Plain FP64 oracle of the deterministic Henry solve (test infrastructure only).

What it computes (paper section 2):
  mass of the liquid phase     d_t(phi rho) + div(rho q) = 0           (Eq. 1)
  mass of salt                 d_t(phi rho c) + div(rho c q - rho D grad c) = 0  (Eq. 2)
  Darcy velocity               q = -K/mu (grad p - rho g), g = (0, -9.8)  (Eq. 3)
  linear density               rho(c) = rho0 + (rho1 - rho0) c, mu const  (Eq. 4)
  molecular diffusion          D_tensor = phi D I                        (Eq. 5)
  initial state c = 0; right side c = 1, p hydrostatic seawater; left side
  c = 0 with a prescribed freshwater mass inflow; top and bottom no flow
  (section 2.1, boundary conditions).
Discretisation (the readings listed here are this project's, the paper uses a
vertex-centred scheme in ug4): cell-centred finite volumes on [0,Lx]x[0,Ly]
(y upward; the paper's [0,2]x[-1,0] shifted by +1), implicit Euler with a
fixed step tau (section 2.3), Newton on the coupled (p, c) system
(section 2.3).

  * face permeability and porosity: harmonic means of the two cells;
  * face density in gravity and diffusion: arithmetic mean of rho(c);
  * advected rho and rho*c: full upwind by the sign of the face flux q_f,
    `q_f >= 0` takes the cell on the negative side;
  * left side: fixed mass inflow rho0 * q_in(y) per unit length, no advected
    salt, diffusive Dirichlet c = 0 at distance hx/2;
  * right side: Dirichlet p = rho1 g (Ly - y) at distance hx/2; advected
    values upwinded with c = 1 (rho = rho1) on inflow; diffusive Dirichlet
    c = 1 at distance hx/2;
  * boundary faces use the cell's own K and phi and the mean of the cell's
    and the boundary's rho.

Linear solves use scipy's sparse LU (a library primitive); the Jacobian is
exact, obtained by complex-step differentiation of the residual with a
5-colour distance-2 colouring of the 5-point stencil, so it shares nothing
with a hand-derived Jacobian.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------
# Parameters (Table 1 of the paper; gravity from Eq. 3)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Physics:
    rho0: float = 1000.0          # pure water density [kg/m^3], Table 1
    rho1: float = 1024.99         # brine density [kg/m^3], Table 1
    mu: float = 1e-3              # viscosity [kg/(m s)], Table 1
    g: float = 9.8                # gravity magnitude [m/s^2], Eq. 3
    D: float = 18.8571e-6         # diffusion coefficient [m^2/s], Table 1
    K0: float = 1.020408e-9       # reference permeability [m^2], Table 1
    phi0: float = 0.35            # mean porosity, Table 1
    q0: float = 6.6e-5            # freshwater inflow [m/s] (6.6e-2 kg/s / rho0)
    Lx: float = 2.0
    Ly: float = 1.0
    field_model: int = 0          # 0: smooth 3/6-variable fields; 1: the paper's
                                  # Eq. poro_2levels + Kozeny-Carman + recharge

    @property
    def kappa_kc(self) -> float:
        """Kozeny-Carman scaling (Eq. e_perm_Kozeny_Carman) chosen so that the
        mean porosity gives the reference permeability: K0 (1 - phi0^2) / phi0^3
        (Table 1 lists kappa_KC = 2.088415e-8 m^2 beside K0 and phi0)."""
        return self.K0 * (1.0 - self.phi0 ** 2) / self.phi0 ** 3


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nt: int          # number of implicit Euler steps
    T: float         # final time [s]

    def lengths(self, phys: "Physics"):
        return phys.Lx / self.nx, phys.Ly / self.ny

    @property
    def tau(self) -> float:
        return self.T / self.nt


def level_grid(level: int, nx0: int = 32, ny0: int = 16, nt0: int = 24,
               T: float = 43200.0) -> Grid:
    """MLMC level l: h and tau halve per level (nx = nx0 2^l, r = nt0 2^l)."""
    f = 1 << level
    return Grid(nx=nx0 * f, ny=ny0 * f, nt=nt0 * f, T=T)


# Observation points: the paper's points 3, 9 and 15 (Eq. 12points),
# (1.40,-0.95), (1.65,-0.75), (1.90,-0.50), shifted into y in [0, 1].
OBS_POINTS = ((1.40, 0.05), (1.65, 0.25), (1.90, 0.50))

# The paper's 15 points (Eq. 12points) in the frame y in [0, 1], and the
# freshwater threshold of Eq. integral_fw.
POINTS15 = tuple((x, y) for y in (0.05, 0.25, 0.50) for x in (0.90, 1.15, 1.40, 1.65, 1.90))
BOX_HALF = 0.1
FRESH_C = 0.012178

QOI_NAMES = ("Q_S", "salt_mass", "toe", "c_x3", "c_x9", "c_x15", "Q_FW") + tuple(
    f"Q_{i + 1}" for i in range(15))
NQ = len(QOI_NAMES)


def cell_centres(grid: Grid, phys: Physics):
    hx, hy = grid.lengths(phys)
    x = (np.arange(grid.nx) + 0.5) * hx
    y = (np.arange(grid.ny) + 0.5) * hy
    return x, y


# ----------------------------------------------------------------------------
# Random fields (the paper's model is Eq. poro_2levels; the smooth three-
# and six-variable fields below are this workload's stand-in for it)
# ----------------------------------------------------------------------------
@dataclass
class Fields:
    phi: np.ndarray      # [ny, nx] porosity at cell centres
    K: np.ndarray        # [ny, nx] permeability at cell centres
    qin: np.ndarray      # [ny] left-side inflow velocity per row [m/s]


def field_at(phys: Physics, xi, X, Y, logk=None):
    """Porosity and permeability of the random field at points (X, Y) (any
    array shape, frame y in [0, Ly]); see `fields` for the formulas."""
    if phys.field_model == 1:
        Yp = Y - phys.Ly
        C0 = np.where(Yp < -0.8, 1.2 * (1.0 + 0.2 * xi[0]), 1.0 + 0.0 * xi[0])
        C1 = 1.0 + 0.15 * (xi[1] * np.cos(np.pi * X / 2) - xi[1] * np.sin(2 * np.pi * Yp)
                           + xi[0] * np.cos(2 * np.pi * X))
        C2 = 1.0 + 0.2 * (xi[0] * np.sin(64 * np.pi * X) + xi[1] * np.sin(32 * np.pi * Yp))
        phi = phys.phi0 * C0 * C1 * C2
        K = phys.kappa_kc * phi ** 3 / (1.0 - phi ** 2)
        if logk is not None:
            K = K * np.exp(logk)
        return phi, K
    a = 0.1 * xi[0] * np.cos(np.pi * X / 2) * np.sin(np.pi * Y)
    b = 0.5 * xi[1] * np.sin(np.pi * X / 2) * np.cos(np.pi * Y)
    if xi.shape[0] >= 6:
        a = a + 0.05 * xi[3] * np.cos(np.pi * X) * np.sin(2 * np.pi * Y)
        b = b + 0.05 * xi[4] * np.sin(np.pi * X) * np.cos(2 * np.pi * Y)
    if logk is not None:
        b = b + logk
    return phys.phi0 * (1.0 + a), phys.K0 * np.exp(b)


def inflow_at(phys: Physics, xi, y):
    """Left-side inflow velocity q_in at heights y (the base of Eq.
    e_recharge_of_param for field model 1)."""
    if phys.field_model == 1:
        return phys.q0 * (1.0 + 0.5 * xi[2]) + 0.0 * y
    qf = 1.0 + 0.1 * xi[2] + 0.0 * y
    if xi.shape[0] >= 6:
        qf = qf + 0.05 * xi[5] * np.cos(np.pi * y)
    return phys.q0 * qf


def fields(grid: Grid, phys: Physics, xi, logk=None) -> Fields:
    """field_model 0 (the configs' smooth fields):
    phi = phi0 (1 + 0.1 xi1 cos(pi x/2) sin(pi y) [+ 0.05 xi4 cos(pi x) sin(2 pi y)])
    K   = K0 exp(0.5 xi2 sin(pi x/2) cos(pi y) [+ 0.05 xi5 sin(pi x) cos(2 pi y)] + theta)
    q_in = q0 (1 + 0.1 xi3 [+ 0.05 xi6 cos(pi y)])
    field_model 1 (the paper's, Eq. poro_2levels with y_p = y - Ly in its frame):
    phi = phi0 C0 C1 C2, C0 = 1.2 (1 + 0.2 xi1) for y_p < -0.8 else 1,
      C1 = 1 + 0.15 (xi2 cos(pi x/2) - xi2 sin(2 pi y_p) + xi1 cos(2 pi x)),
      C2 = 1 + 0.2 (xi1 sin(64 pi x) + xi2 sin(32 pi y_p));
    K = kappa_KC phi^3 / (1 - phi^2) exp(theta) (Eq. e_perm_Kozeny_Carman);
    q_in = q0 (1 + 0.5 xi3), the base of Eq. e_recharge_of_param (its time
    factor is applied per step by `solve`).
    Evaluated at cell centres of this grid (the paper evaluates its fields at
    integration points rather than from a precomputed raster, section
    "Uncertain porosity and recharge"). `xi` may be complex (complex step).
    """
    xi = np.asarray(xi)
    x, y = cell_centres(grid, phys)
    X, Y = np.meshgrid(x, y)
    phi, K = field_at(phys, xi, X, Y, logk)
    return Fields(phi=phi, K=K, qin=inflow_at(phys, xi, y))


# ----------------------------------------------------------------------------
# Fluxes and residual (Eqs. 1-5 integrated over each cell, implicit Euler)
# ----------------------------------------------------------------------------
def _upwind(q, a_neg, a_pos):
    """Value carried by face flux q: from the cell on the negative side if
    q >= 0, else from the positive side. Only the real part decides, so the
    switch is frozen under complex-step differentiation."""
    return np.where(np.real(q) >= 0, a_neg, a_pos)


def face_fluxes(grid: Grid, phys: Physics, f: Fields, p, c):
    """Mass and salt fluxes [kg/(s m)] through every face, positive along +x
    (vertical faces) or +y (horizontal faces); boundary fluxes positive
    outward. Returns a dict of arrays."""
    hx, hy = grid.lengths(phys)
    rho = phys.rho0 + (phys.rho1 - phys.rho0) * c
    rc = rho * c
    out = {}
    # vertical faces between (j, i) and (j, i+1); area hy, distance hx
    KP, KN = f.K[:, :-1], f.K[:, 1:]
    Kf = 2.0 * KP * KN / (KP + KN)
    fP, fN = f.phi[:, :-1], f.phi[:, 1:]
    phif = 2.0 * fP * fN / (fP + fN)
    rbar = 0.5 * (rho[:, :-1] + rho[:, 1:])
    q = -(Kf / phys.mu) * (p[:, 1:] - p[:, :-1]) / hx
    out["mass_x"] = hy * q * _upwind(q, rho[:, :-1], rho[:, 1:])
    out["salt_x"] = hy * (q * _upwind(q, rc[:, :-1], rc[:, 1:])
                          - rbar * phif * phys.D * (c[:, 1:] - c[:, :-1]) / hx)
    out["q_x"] = q
    # horizontal faces between (j, i) and (j+1, i); area hx, distance hy
    KP, KN = f.K[:-1, :], f.K[1:, :]
    Kf = 2.0 * KP * KN / (KP + KN)
    fP, fN = f.phi[:-1, :], f.phi[1:, :]
    phif = 2.0 * fP * fN / (fP + fN)
    rbar = 0.5 * (rho[:-1, :] + rho[1:, :])
    # q.n = -K/mu (dp/dy - rho g.e_y) with g.e_y = -g
    q = -(Kf / phys.mu) * ((p[1:, :] - p[:-1, :]) / hy + rbar * phys.g)
    out["mass_y"] = hx * q * _upwind(q, rho[:-1, :], rho[1:, :])
    out["salt_y"] = hx * (q * _upwind(q, rc[:-1, :], rc[1:, :])
                          - rbar * phif * phys.D * (c[1:, :] - c[:-1, :]) / hy)
    out["q_y"] = q
    # left side x = 0, outward normal -x: prescribed freshwater inflow
    cP, rP, phP = c[:, 0], rho[:, 0], f.phi[:, 0]
    out["mass_left"] = -hy * phys.rho0 * f.qin + 0.0 * cP
    rb = 0.5 * (rP + phys.rho0)
    out["salt_left"] = -hy * rb * phP * phys.D * (0.0 - cP) / (0.5 * hx)
    # right side x = Lx, outward normal +x: hydrostatic seawater
    _, y = cell_centres(grid, phys)
    pb = phys.rho1 * phys.g * (phys.Ly - y)
    cP, rP, phP, KP = c[:, -1], rho[:, -1], f.phi[:, -1], f.K[:, -1]
    q = -(KP / phys.mu) * (pb - p[:, -1]) / (0.5 * hx)
    rb = 0.5 * (rP + phys.rho1)
    out["mass_right"] = hy * q * _upwind(q, rP, phys.rho1 + 0.0 * rP)
    out["salt_right"] = hy * (q * _upwind(q, rP * cP, phys.rho1 * 1.0 + 0.0 * rP)
                              - rb * phP * phys.D * (1.0 - cP) / (0.5 * hx))
    out["q_right"] = q
    return out


def residual(grid: Grid, phys: Physics, f: Fields, p, c, c_old):
    """Implicit-Euler finite-volume residual (R_p, R_c), each [ny, nx]:
    R = V (m(u) - m(u_old)) / tau + sum of outward face fluxes."""
    hx, hy = grid.lengths(phys)
    V = hx * hy
    tau = grid.tau
    rho = phys.rho0 + (phys.rho1 - phys.rho0) * c
    rho_o = phys.rho0 + (phys.rho1 - phys.rho0) * c_old
    dt = np.result_type(p, c, c_old, f.phi, f.K, f.qin)
    Rp = (V * f.phi * (rho - rho_o) / tau).astype(dt)
    Rc = (V * f.phi * (rho * c - rho_o * c_old) / tau).astype(dt)
    F = face_fluxes(grid, phys, f, p, c)
    Rp[:, :-1] += F["mass_x"]
    Rp[:, 1:] -= F["mass_x"]
    Rc[:, :-1] += F["salt_x"]
    Rc[:, 1:] -= F["salt_x"]
    Rp[:-1, :] += F["mass_y"]
    Rp[1:, :] -= F["mass_y"]
    Rc[:-1, :] += F["salt_y"]
    Rc[1:, :] -= F["salt_y"]
    Rp[:, 0] += F["mass_left"]
    Rc[:, 0] += F["salt_left"]
    Rp[:, -1] += F["mass_right"]
    Rc[:, -1] += F["salt_right"]
    return Rp, Rc


# ----------------------------------------------------------------------------
# Exact Jacobian by complex step, Newton with sparse LU
# ----------------------------------------------------------------------------
_CS_H = 1e-30
_STENCIL = ((0, 0), (0, -1), (0, 1), (-1, 0), (1, 0))


def interleave(a, b):
    """Unknown ordering of the oracle's linear systems: u[2*cell + var],
    var 0 = p, var 1 = c, cell = j*nx + i."""
    out = np.empty(2 * a.size, dtype=np.result_type(a, b))
    out[0::2] = a.ravel()
    out[1::2] = b.ravel()
    return out


def jacobian(grid: Grid, phys: Physics, f: Fields, p, c, c_old):
    """d(R_p, R_c)/d(p, c) as a sparse [2N, 2N] matrix (interleaved order).
    Complex-step derivative, exact to rounding; cells coloured by
    (i + 2j) mod 5 so that perturbed stencils never overlap."""
    ny, nx = grid.ny, grid.nx
    jj, ii = np.mgrid[0:ny, 0:nx]
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
            Rp, Rc = residual(grid, phys, f, pz, cz, c_old)
            dRp, dRc = Rp.imag / _CS_H, Rc.imag / _CS_H
            for dj, di in _STENCIL:
                Qj, Qi = Pj + dj, Pi + di
                ok = (Qj >= 0) & (Qj < ny) & (Qi >= 0) & (Qi < nx)
                pc = Pj[ok] * nx + Pi[ok]
                qc = Qj[ok] * nx + Qi[ok]
                rows += [2 * qc, 2 * qc + 1]
                cols += [2 * pc + var, 2 * pc + var]
                vals += [dRp[Qj[ok], Qi[ok]], dRc[Qj[ok], Qi[ok]]]
    n = 2 * nx * ny
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def hydrostatic_guess(grid: Grid, phys: Physics):
    """Initial Newton guess for p: seawater hydrostatics rho1 g (Ly - y)."""
    _, y = cell_centres(grid, phys)
    return np.repeat((phys.rho1 * phys.g * (phys.Ly - y))[:, None], grid.nx, axis=1)


def newton_step(grid: Grid, phys: Physics, f: Fields, p, c, c_old,
                maxit: int = 30, tol_c: float = 1e-12, tol_p_rel: float = 1e-12):
    """One implicit Euler step: Newton from (p, c) until the update is below
    tol_c in c and tol_p_rel * rho1 g Ly in p (quadratic convergence leaves
    the remaining error at rounding level). Returns (p, c, iterations)."""
    p = p.copy()
    c = c.copy()
    pscale = phys.rho1 * phys.g * phys.Ly
    for it in range(1, maxit + 1):
        Rp, Rc = residual(grid, phys, f, p, c, c_old)
        J = jacobian(grid, phys, f, p, c, c_old)
        d = spla.spsolve(J, -interleave(Rp, Rc))
        dp = d[0::2].reshape(p.shape)
        dc = d[1::2].reshape(c.shape)
        p += dp
        c += dc
        if np.max(np.abs(dc)) <= tol_c and np.max(np.abs(dp)) <= tol_p_rel * pscale:
            return p, c, it
    raise RuntimeError("oracle Newton did not converge")


def solve(grid: Grid, phys: Physics, xi, logk=None, c0=None, p0=None,
          keep_states: bool = False):
    """Run the implicit Euler time loop for grid.nt steps from c0 (default 0).
    Returns dict with p, c at T, Newton iterations per step and, if asked,
    every state (p^n, c^n), n = 0..nt."""
    f = fields(grid, phys, xi, logk)
    c = np.zeros((grid.ny, grid.nx)) if c0 is None else np.array(c0, dtype=float)
    p = hydrostatic_guess(grid, phys) if p0 is None else np.array(p0, dtype=float)
    its = []
    states = [(p.copy(), c.copy())] if keep_states else None
    for n in range(grid.nt):
        fn = f
        if phys.field_model == 1:
            # Eq. e_recharge_of_param: inflow times (1 + sin(pi t / 40)), t in
            # seconds, taken at the new time level t^(n+1) of the implicit step
            t = (n + 1) * grid.tau
            fn = Fields(phi=f.phi, K=f.K, qin=f.qin * (1.0 + math.sin(math.pi * t / 40.0)))
        p, c, it = newton_step(grid, phys, fn, p, c, c.copy())
        its.append(it)
        if keep_states:
            states.append((p.copy(), c.copy()))
    return {"p": p, "c": c, "its": its, "fields": f, "states": states}


# ----------------------------------------------------------------------------
# Quantities of interest (section 4, Eqs. integral_s and 12points)
# ----------------------------------------------------------------------------
def point_value(grid: Grid, phys: Physics, c, x, y):
    """Bilinear interpolation of cell-centred values, clamped to the
    outermost cell centres."""
    hx, hy = grid.lengths(phys)
    fx, fy = x / hx - 0.5, y / hy - 0.5
    i0 = int(min(max(math.floor(fx), 0), grid.nx - 2))
    j0 = int(min(max(math.floor(fy), 0), grid.ny - 2))
    tx = min(max(fx - i0, 0.0), 1.0)
    ty = min(max(fy - j0, 0.0), 1.0)
    return ((1 - tx) * (1 - ty) * c[j0, i0] + tx * (1 - ty) * c[j0, i0 + 1]
            + (1 - tx) * ty * c[j0 + 1, i0] + tx * ty * c[j0 + 1, i0 + 1])


def box_integral(grid: Grid, phys: Physics, g, x0, y0, half=BOX_HALF):
    """Integral of the cell-wise constant field g over the box
    [x0 - half, x0 + half] x [y0 - half, y0 + half] clipped to the domain:
    sum over cells of g times the area of the cell inside the box."""
    hx, hy = grid.lengths(phys)
    xl = np.arange(grid.nx) * hx
    yl = np.arange(grid.ny) * hy
    ox = np.clip(np.minimum(xl + hx, x0 + half) - np.maximum(xl, x0 - half), 0.0, None)
    oy = np.clip(np.minimum(yl + hy, y0 + half) - np.maximum(yl, y0 - half), 0.0, None)
    return float(np.sum(g * oy[:, None] * ox[None, :]))


def qoi(grid: Grid, phys: Physics, f: Fields, c):
    """[Q_S, salt mass, toe, c(x3), c(x9), c(x15), Q_FW, Q_1..Q_15]:
    Q_S = int c rho dx (Eq. integral_s), salt mass = int phi rho c dx (the
    conserved quantity of Eq. 2), toe = int c (Lx - x) dx, c at the three
    observation points, Q_FW = area where c <= 0.012178 (Eq. integral_fw),
    Q_i = int over the box of half-width 0.1 around point i of c rho dx
    (Eq. integral_box, points of Eq. 12points), with c constant per cell."""
    hx, hy = grid.lengths(phys)
    V = hx * hy
    rho = phys.rho0 + (phys.rho1 - phys.rho0) * c
    x, _ = cell_centres(grid, phys)
    out = [np.sum(c * rho) * V, np.sum(f.phi * rho * c) * V,
           np.sum(c * (phys.Lx - x)[None, :]) * V]
    out += [point_value(grid, phys, c, px, py) for px, py in OBS_POINTS]
    out.append(float(np.sum(c <= FRESH_C)) * V)
    out += [box_integral(grid, phys, c * rho, px, py) for px, py in POINTS15]
    return np.array(out)


def prolong_constant(c_coarse):
    """Piecewise-constant transfer of a coarse cell field to the grid refined
    by two in each direction (used for fine-minus-coarse field differences)."""
    return np.repeat(np.repeat(c_coarse, 2, axis=0), 2, axis=1)


def solve_batch(grid: Grid, phys: Physics, xis, logks=None):
    """Loop of independent solves; returns (q [B, NQ], c [B, ny, nx], p)."""
    qs, cs, ps = [], [], []
    for b in range(len(xis)):
        r = solve(grid, phys, xis[b], None if logks is None else logks[b])
        qs.append(qoi(grid, phys, r["fields"], r["c"]))
        cs.append(r["c"])
        ps.append(r["p"])
    return np.array(qs), np.array(cs), np.array(ps)
