"""Pins of the vertex-centred oracle variant (oracle/henry_vc.py) against
what the mathematics fixes, chosen so that a mistake in any part of it
fails one of them:
  diffusion closed form      -> storage, diffusive conductances, half boxes
                                on closed sides, Dirichlet nodes at x = 0, Lx
  steady advection-diffusion -> the exponentially fitted partial upwind
                                weight (nodally exact: the discrete profile IS
                                the exact exponential one), inflow, scatter
                                signs, right Dirichlet column
  uniform flow pressure      -> Darcy fluxes, face transmissibilities
  hydrostatic rest           -> gravity term and its face density
  salt balance               -> interior fluxes cancel over a union of boxes
  Jacobian vs differences    -> complex-step assembly
  grid convergence           -> order of the coupled scheme (Eq. 1st_ord_conv)
  fitted weight              -> series / direct branches, limits
"""
import math

import numpy as np
import pytest

from oracle import henry as H
from oracle import henry_vc as V
from paper_2403_17018_gb300.inputs import xi_batch


def test_fitted_weight_limits_and_branches():
    """alpha(Pe) = coth(Pe/2) - 2/Pe: alpha(0) = 0 (central), alpha -> 1
    (upwind), alpha ~ Pe/6 for small Pe; the series branch below 1e-2 meets
    the direct form at the switch and both agree with a high-precision
    evaluation (mpmath-free: the continued identity coth x - 1/x =
    sum 2 x / (x^2 + (k pi)^2))."""
    assert V.fitted_alpha(0.0) == 0.0
    assert V.fitted_alpha(1e4) == pytest.approx(1.0 - 2e-4, rel=1e-15)
    for P in (1e-6, 3e-3, 9.9e-3, 1.01e-2, 0.3, 2.0, 17.0):
        x = P / 2
        ref = sum(2 * x / (x * x + (k * math.pi) ** 2) for k in range(1, 200000))
        assert V.fitted_alpha(P) == pytest.approx(ref, rel=1e-5)     # tail of the sum ~1e-6
    # continuity at the switch, within the direct form's cancellation
    # error there (eps 2 / Pe = 4.4e-14)
    lo, hi = V.fitted_alpha(1e-2 * (1 - 1e-12)), V.fitted_alpha(1e-2)
    assert abs(lo - hi) <= 5e-14


@pytest.mark.parametrize("nx,ny", [(32, 16), (24, 6)])
def test_vc_diffusion_closed_form(nx, ny):
    """rho1 = rho0 and no inflow leave the fluid at rest, so c obeys
    d_t c = D lap c with c = 0 at the nodes x = 0 and c = 1 at x = Lx. x/2
    is the exact discrete steady state, and sin(pi x/2) cos(pi y) is an
    exact eigenvector of the vertex-centred operator (Dirichlet nodes in x,
    half boxes and closed sides in y) with eigenvalue
    D (4/hx^2 sin^2(pi hx/4) + 4/hy^2 sin^2(pi hy/2)); implicit Euler damps it
    by (1 + tau lambda)^-1 per step."""
    ph = H.Physics(rho1=1000.0, q0=0.0)
    g = H.Grid(nx, ny, 5, 5 * 1800.0)
    hx, hy = g.lengths(ph)
    x, y = V.nodes(g, ph)
    X, Y = np.meshgrid(x[:nx], y)
    A = 0.3
    mode = np.sin(np.pi * X / 2) * np.cos(np.pi * Y)
    xi = np.array([0.0, 0.8, -0.4])       # xi1 = 0: uniform porosity
    r = V.solve(g, ph, xi, c0=X / 2 + A * mode)
    lam = ph.D * (4 / hx**2 * math.sin(math.pi * hx / 4) ** 2
                  + 4 / hy**2 * math.sin(math.pi * hy / 2) ** 2)
    expect = X / 2 + A * mode * (1 + g.tau * lam) ** (-g.nt)
    assert np.max(np.abs(r["c"] - expect)) <= 1e-12
    assert np.max(np.abs(r["p"] - ph.rho0 * ph.g * (ph.Ly - Y))) <= 1e-9


@pytest.mark.parametrize("q0", [6.6e-5, 6.6e-4, 3e-3])
def test_vc_steady_advection_is_nodally_exact(q0):
    """Uniform phi and K, rho1 = rho0: the inflow drives the uniform flow q,
    p = rho0 g (Ly - y) + mu q / K (Lx - x) exactly, and the steady salt
    profile of the exponentially fitted scheme equals the exact solution of
    q c' = phi D c'', c(0) = 0, c(Lx) = 1, at every node:
    c = (exp(k (x - Lx)) - exp(-k Lx)) / (1 - exp(-k Lx)), k = q / (phi D).
    Cell Peclet numbers 0.66, 6.6 and 30 (nearly central to nearly upwind)."""
    ph = H.Physics(rho1=1000.0, q0=q0)
    g = H.Grid(32, 4, 2, 2e12)              # tau = 1e12 s: each step lands on the steady state
    xi3 = 0.6
    r = V.solve(g, ph, np.array([0.0, 0.0, xi3]))
    q = q0 * (1 + 0.1 * xi3)
    x, y = V.nodes(g, ph)
    X, Y = np.meshgrid(x[:g.nx], y)
    p_exact = ph.rho0 * ph.g * (ph.Ly - Y) + ph.mu * q / ph.K0 * (ph.Lx - X)
    assert np.max(np.abs(r["p"] - p_exact)) <= 1e-9 * np.max(np.abs(p_exact))
    k = q / (ph.phi0 * ph.D)
    c_exact = (np.exp(k * (x - ph.Lx)) - math.exp(-k * ph.Lx)) / (1 - math.exp(-k * ph.Lx))
    assert np.max(np.abs(r["c"] - c_exact[None, :g.nx])) <= 1e-11


def test_vc_hydrostatic_rest():
    """c = 1 and no inflow: seawater at rest. Every Darcy flux vanishes to
    rounding at the nodal hydrostatic pressure, and so do the mass residuals."""
    ph = H.Physics(q0=0.0)
    g = H.Grid(32, 16, 2, 3600.0)
    vf = V.vfields(g, ph, np.array([0.7, -0.9, 0.3]))
    x, y = V.nodes(g, ph)
    p = np.repeat((ph.rho1 * ph.g * (ph.Ly - y))[:, None], g.nx, axis=1)
    c = np.ones_like(p)
    F = V.face_fluxes(g, ph, vf, p, c)
    qscale = ph.K0 / ph.mu * ph.rho1 * ph.g
    assert np.max(np.abs(F["Qx"])) <= 1e-13 * qscale and np.max(np.abs(F["Qy"])) <= 1e-13 * qscale
    Rp, _ = V.residual(g, ph, vf, p, c, c)
    assert np.max(np.abs(Rp)) <= 1e-13 * qscale * ph.rho1


@pytest.mark.parametrize("n_xi", [3, 6])
def test_vc_salt_balance_over_the_interior_boxes(n_xi):
    """At a converged step, over the boxes of the nodes i >= 1 (the left
    column's salt equation is its Dirichlet row), the stored salt changes by
    -tau times the net outflow through the faces x = hx/2 and x = Lx - hx/2:
    every face between two of these boxes cancels."""
    ph = H.Physics()
    g = H.Grid(32, 16, 3, 3 * 1800.0)
    r = V.solve(g, ph, xi_batch(0, 5, 1, n_xi=n_xi)[0], keep_states=True)
    vf = r["vfields"]
    drho = ph.rho1 - ph.rho0
    for n in range(1, g.nt + 1):
        p, c = r["states"][n]
        co = r["states"][n - 1][1]
        F = V.face_fluxes(g, ph, vf, p, c)
        store = np.sum(vf.vphi[:, 1:] * ((ph.rho0 + drho * c) * c - (ph.rho0 + drho * co) * co)[:, 1:])
        out = np.sum(F["salt_x"][:, -1]) - np.sum(F["salt_x"][:, 0])
        scale = g.tau * ph.rho1 * ph.q0 * ph.Ly
        assert abs(store + g.tau * out) <= 1e-11 * scale


def test_vc_jacobian_matches_central_differences():
    ph = H.Physics()
    g = H.Grid(12, 6, 1, 1800.0)
    rng = np.random.default_rng(7)
    vf = V.vfields(g, ph, xi_batch(0, 3, 1)[0])
    p0, _ = V.initial_state(g, ph)
    p = p0 + 30 * rng.standard_normal(p0.shape)
    c = np.clip(rng.random(p0.shape), 0, 1)
    c_old = np.clip(c + 0.05 * rng.standard_normal(c.shape), 0, 1)
    J = V.jacobian(g, ph, vf, p, c, c_old).toarray()
    for col in rng.choice(J.shape[1], size=40, replace=False):
        cell, var = divmod(col, 2)
        j, i = divmod(cell, g.nx)
        h = 1e-3 if var == 0 else 1e-6
        pp, cp, pm, cm = p.copy(), c.copy(), p.copy(), c.copy()
        if var == 0:
            pp[j, i] += h
            pm[j, i] -= h
        else:
            cp[j, i] += h
            cm[j, i] -= h
        R1 = V.residual(g, ph, vf, pp, cp, c_old)
        R0 = V.residual(g, ph, vf, pm, cm, c_old)
        fd = H.interleave((R1[0] - R0[0]) / (2 * h), (R1[1] - R0[1]) / (2 * h))
        assert np.max(np.abs(fd - J[:, col])) <= 1e-6 * np.max(np.abs(J[:, col]))


def test_vc_grid_convergence_is_at_least_first_order():
    """Eq. 1st_ord_conv: h and tau halve per level; the nodes of level l are
    nodes of level l+1, so successive levels are compared at the common nodes.
    The distances ||c_l - c_(l+1)|| of levels 0-1 and 1-2 shrink by a factor
    of at least 1.6 (first order gives 2, second order 4)."""
    ph = H.Physics()
    xi = np.array([0.4, -0.3, 0.5])
    T = 4 * 1800.0
    cs = []
    for l in range(3):
        g = H.Grid(32 << l, 16 << l, 4 << l, T)
        cs.append(V.full_nodes(g, ph, V.solve(g, ph, xi)["c"]))
    d01 = np.max(np.abs(cs[0] - cs[1][::2, ::2]))
    d12 = np.max(np.abs(cs[1] - cs[2][::2, ::2]))
    assert d01 / d12 >= 1.6, (d01, d12)


def test_vc_qoi_of_known_fields():
    """c = 1 everywhere (nodes and the Dirichlet column): Q_S = rho1 |D| = 2
    rho1, the toe integral is |D| Lx / 2 = 2, the points read 1, Q_FW = 0 and
    every box integral is rho1 times the clipped box area."""
    ph = H.Physics()
    g = H.Grid(64, 32, 1, 1.0)
    vf = V.vfields(g, ph, np.zeros(3))
    q = V.qoi(g, ph, vf, np.ones((g.ny + 1, g.nx)))
    assert q[0] == pytest.approx(2 * ph.rho1, rel=1e-14)
    assert q[2] == pytest.approx(2.0, rel=1e-14)
    assert np.allclose(q[3:6], 1.0, rtol=1e-15) and q[6] == 0.0
    area = np.array([0.03] * 5 + [0.04] * 10)
    assert np.allclose(q[7:22], ph.rho1 * area, rtol=1e-13)


def test_vc_variable_density_diffusion_telescopes_to_the_continuum_profile():
    """No gravity (g = 0), no inflow: the fluid stays at rest and the steady
    salt profile carries a constant flux -rho(c) phi D c'. With the face
    density the mean of the two nodes', rho_bar (c_(i+1) - c_i) = G(c_(i+1))
    - G(c_i) for G(c) = rho0 c + (rho1 - rho0) c^2 / 2, so the discrete
    profile is the continuum one at every node: G(c_i) = G(1) x_i / Lx."""
    ph = H.Physics(g=0.0, q0=0.0)
    g = H.Grid(16, 2, 2, 2e12)
    r = V.solve(g, ph, np.array([0.0, 0.4, 0.0]))
    x, _ = V.nodes(g, ph)
    drho = ph.rho1 - ph.rho0
    Gx = (ph.rho0 + drho / 2) * x[:g.nx] / ph.Lx
    c_exact = (-ph.rho0 + np.sqrt(ph.rho0 ** 2 + 2 * drho * Gx)) / drho
    assert np.max(np.abs(r["c"] - c_exact[None, :])) <= 1e-12
    assert np.max(np.abs(r["p"])) <= 1e-9


def test_vc_upwind_density_without_diffusion():
    """D = 0 (full upwind by definition), no gravity, rho1 != rho0: fresh
    water enters on the left and the steady state is c = 0 at every unknown
    node; every face, the one to the seawater column included, carries the
    upwind (fresh) density, so the pressure is exactly the uniform-flow
    profile mu q / K (Lx - x)."""
    ph = H.Physics(g=0.0, D=0.0)
    g = H.Grid(16, 2, 2, 2e12)
    xi3 = 0.3
    r = V.solve(g, ph, np.array([0.0, 0.0, xi3]))
    q = ph.q0 * (1 + 0.1 * xi3)
    x, _ = V.nodes(g, ph)
    assert np.max(np.abs(r["c"])) <= 1e-14
    p_exact = ph.mu * q / ph.K0 * (ph.Lx - x[:g.nx])
    assert np.max(np.abs(r["p"] - p_exact[None, :])) <= 1e-10 * np.max(p_exact)


def test_vc_coefficients_are_integrals_of_the_field():
    """The storage of a box is the integral of phi over it and each face's
    conductances the integrals of K and phi along it (midpoint rule on the
    quarter cells and half segments, O(h^2)): against the exact integrals of
    the smooth field phi = phi0 (1 + 0.1 xi1 cos(pi x/2) sin(pi y)) and of
    K = K0 exp(0.5 xi2 sin(pi x/2) cos(pi y)) (the latter by a fine rule)."""
    ph = H.Physics()
    g = H.Grid(32, 16, 1, 1.0)
    hx, hy = g.lengths(ph)
    xi = np.array([0.9, -0.7, 0.0])
    vf = V.vfields(g, ph, xi)
    x, y = V.nodes(g, ph)
    xl, xr = np.clip(x - hx / 2, 0, ph.Lx), np.clip(x + hx / 2, 0, ph.Lx)
    yb, yt = np.clip(y - hy / 2, 0, ph.Ly), np.clip(y + hy / 2, 0, ph.Ly)
    Ix = (2 / np.pi) * (np.sin(np.pi * xr / 2) - np.sin(np.pi * xl / 2))
    Iy = (np.cos(np.pi * yb) - np.cos(np.pi * yt)) / np.pi
    exact = ph.phi0 * (np.outer(yt - yb, xr - xl) + 0.1 * xi[0] * np.outer(Iy, Ix))
    V_box = np.outer(yt - yb, xr - xl)
    assert np.max(np.abs(vf.vphi - exact[:, :g.nx]) / V_box[:, :g.nx]) <= 2e-4
    assert np.max(np.abs(vf.vphi_r - exact[:, g.nx]) / V_box[:, g.nx]) <= 2e-4
    # diffusive conductance of the east faces: D / hx * integral of phi along x = x_i + hx/2
    xf = (np.arange(g.nx) + 0.5) * hx
    dx_exact = ph.D / hx * ph.phi0 * ((yt - yb)[:, None]
                                     + 0.1 * xi[0] * np.outer(Iy, np.cos(np.pi * xf / 2)))
    assert np.max(np.abs(vf.dx - dx_exact) / (ph.D * ph.phi0)) <= 2e-4
    # transmissibility of the north faces: integral of K along y = y_j + hy/2, fine rule
    yf = (np.arange(g.ny) + 0.5) * hy
    s = (np.arange(400) + 0.5) / 400
    tyx = np.zeros((g.ny, g.nx))
    for i in range(g.nx):
        xs = xl[i] + (xr[i] - xl[i]) * s
        X, Y = np.meshgrid(xs, yf)
        Kv = ph.K0 * np.exp(0.5 * xi[1] * np.sin(np.pi * X / 2) * np.cos(np.pi * Y))
        tyx[:, i] = Kv.mean(axis=1) * (xr[i] - xl[i]) / (ph.mu * hy)
    assert np.max(np.abs(vf.ty - tyx) / tyx) <= 2e-4
