"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a different part of the discretisation so that a dropped
term, a wrong sign or index, or a swapped operand fails at least one of them:
  hydrostatic rest          -> gravity sign/magnitude, face density, right-side p
  diffusion closed form     -> diffusion term, tau, accumulation, Dirichlet c at
                               hx/2 on both sides, zero flux top/bottom
  uniform flow + advection  -> Darcy law in x, mu, K, inflow magnitude, right
                               p at hx/2, upwind direction and boundary upwinding
  salt/fluid balance        -> interior face fluxes cancel (scatter signs)
  Jacobian vs central FD    -> colouring and assembly of the exact Jacobian
  time order                -> first order of implicit Euler (section 2.3)
  grid convergence          -> h/tau scaling of every term of the coupled
                               problem (successive levels approach each other)
  allocation table          -> Eq. M_ell against the paper's printed numbers
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import henry as H
from oracle import mlmc as M
from paper_2403_17018_gb300.inputs import xi_batch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(nx, ny, nt, T):
    return H.Grid(nx=nx, ny=ny, nt=nt, T=T)


def test_hydrostatic_rest():
    """c = 1 everywhere and no inflow: seawater at rest. q = 0 on every face,
    the fluid-mass residual vanishes, and the salt residual vanishes except in
    the left column, where the only flux is diffusion towards c = 0."""
    ph = H.Physics(q0=0.0)
    g = _grid(32, 16, 2, 3600.0)
    xi = np.array([0.7, -0.9, 0.3])
    f = H.fields(g, ph, xi)
    c = np.ones((g.ny, g.nx))
    p = H.hydrostatic_guess(g, ph)
    F = H.face_fluxes(g, ph, f, p, c)
    # scale of the two cancelling terms in a vertical face flux
    qscale = ph.K0 / ph.mu * ph.rho1 * ph.g
    for k in ("q_x", "q_y", "q_right"):
        assert np.max(np.abs(F[k])) <= 1e-13 * qscale
    Rp, Rc = H.residual(g, ph, f, p, c, c)
    hx, hy = g.lengths(ph)
    rscale = hx * qscale * ph.rho1
    assert np.max(np.abs(Rp)) <= 1e-13 * rscale
    assert np.max(np.abs(Rc[:, 1:])) <= 1e-13 * rscale
    assert np.all(Rc[:, 0] > 0)
    # with rho1 = rho0 the fluid stays at rest while salt diffuses: Newton
    # from a disturbed pressure returns to hydrostatics
    ph2 = H.Physics(rho0=ph.rho1, q0=0.0)
    p_dist = p + 50.0 * np.sin(np.arange(g.nx))[None, :] * np.cos(np.arange(g.ny))[:, None]
    r = H.solve(g, ph2, xi, c0=c, p0=p_dist)
    assert np.max(np.abs(r["p"] - p)) <= 1e-10 * ph.rho1 * ph.g * ph.Ly


@pytest.mark.parametrize("nx,ny", [(32, 16), (24, 6)])
def test_diffusion_closed_form(nx, ny):
    """rho1 = rho0 and no inflow leave q = 0, so c obeys d_t c = D lap c with
    c = 0 at x = 0 and c = 1 at x = Lx. x/2 is the exact discrete steady
    state, and sin(pi x/2) cos(pi y) is an exact eigenvector of the
    cell-centred operator (Dirichlet at hx/2 in x, zero flux in y) with
    eigenvalue D (4/hx^2 sin^2(pi hx/4) + 4/hy^2 sin^2(pi hy/2)); implicit
    Euler damps it by (1 + tau lambda)^-1 per step."""
    ph = H.Physics(rho1=1000.0, q0=0.0)
    g = _grid(nx, ny, 5, 5 * 1800.0)
    hx, hy = g.lengths(ph)
    x, y = H.cell_centres(g, ph)
    X, Y = np.meshgrid(x, y)
    A = 0.3
    mode = np.sin(np.pi * X / 2) * np.cos(np.pi * Y)
    c0 = X / 2 + A * mode
    xi = np.array([0.0, 0.8, -0.4])   # xi1 = 0: uniform porosity
    r = H.solve(g, ph, xi, c0=c0)
    lam = ph.D * (4 / hx**2 * math.sin(math.pi * hx / 4) ** 2
                  + 4 / hy**2 * math.sin(math.pi * hy / 2) ** 2)
    expect = X / 2 + A * mode * (1 + g.tau * lam) ** (-g.nt)
    assert np.max(np.abs(r["c"] - expect)) <= 1e-12
    # pressure stays fresh-water hydrostatic (rho1 = rho0 here)
    assert np.max(np.abs(r["p"] - ph.rho0 * ph.g * (ph.Ly - Y))) <= 1e-9


def test_uniform_flow_and_steady_advection():
    """Uniform phi and K, rho1 = rho0: the left inflow drives a uniform flow
    q = q_in in +x, so p = rho0 g (Ly - y) + mu q / K (Lx - x) exactly.
    The steady salt profile of the upwind scheme satisfies, with cell Peclet
    a = q hx / (phi D) and constant scaled flux F:
      c_{i+1} = (1 + a) c_i - F,  c_0 = -F/2 (Dirichlet 0 at hx/2),
      F = (a + 2) c_{N-1} - 2       (outflow, Dirichlet 1 at hx/2)."""
    ph = H.Physics(rho1=1000.0)
    g = _grid(32, 4, 2, 2e12)   # tau = 1e12 s: each step lands on the steady state
    xi3 = 0.6
    xi = np.array([0.0, 0.0, xi3])
    r = H.solve(g, ph, xi)
    x, y = H.cell_centres(g, ph)
    X, Y = np.meshgrid(x, y)
    q = ph.q0 * (1 + 0.1 * xi3)
    p_exact = ph.rho0 * ph.g * (ph.Ly - Y) + ph.mu * q / ph.K0 * (ph.Lx - X)
    assert np.max(np.abs(r["p"] - p_exact)) <= 1e-9 * np.max(np.abs(p_exact))
    hx, _ = g.lengths(ph)
    a = q * hx / (ph.phi0 * ph.D)
    N = g.nx
    gN = 1 / a - (1 + a) ** (N - 1) * (0.5 + 1 / a)
    F = -2.0 / (1.0 - (a + 2) * gN)
    i = np.arange(N)
    c_exact = F * (1 / a - (1 + a) ** i * (0.5 + 1 / a))
    assert np.max(np.abs(r["c"] - c_exact[None, :])) <= 1e-10


@pytest.mark.parametrize("n_xi", [3, 6])
def test_salt_and_fluid_mass_balance(n_xi):
    """At a converged step the change of stored salt (fluid) mass equals
    -tau times the net boundary outflow: all interior fluxes cancel."""
    ph = H.Physics()
    g = _grid(32, 16, 3, 3 * 1800.0)
    xi = xi_batch(0, 5, 1, n_xi=n_xi)[0]
    r = H.solve(g, ph, xi, keep_states=True)
    f = r["fields"]
    hx, hy = g.lengths(ph)
    V = hx * hy
    for n in range(1, g.nt + 1):
        p_o, c_o = r["states"][n - 1]
        p, c = r["states"][n]
        rho = ph.rho0 + (ph.rho1 - ph.rho0) * c
        rho_o = ph.rho0 + (ph.rho1 - ph.rho0) * c_o
        F = H.face_fluxes(g, ph, f, p, c)
        out_salt = F["salt_left"].sum() + F["salt_right"].sum()
        out_mass = F["mass_left"].sum() + F["mass_right"].sum()
        dsalt = V * np.sum(f.phi * (rho * c - rho_o * c_o))
        dmass = V * np.sum(f.phi * (rho - rho_o))
        scale = g.tau * hy * ph.rho1 * ph.q0 * g.ny
        assert abs(dsalt + g.tau * out_salt) <= 1e-11 * scale
        assert abs(dmass + g.tau * out_mass) <= 1e-11 * scale


def test_jacobian_matches_central_differences():
    ph = H.Physics()
    g = _grid(16, 8, 1, 1800.0)
    rng = np.random.default_rng(3)
    xi = xi_batch(0, 11, 1)[0]
    f = H.fields(g, ph, xi, logk=0.1 * rng.standard_normal((g.ny, g.nx)))
    c = np.clip(rng.random((g.ny, g.nx)), 0, 1)
    c_old = np.clip(c + 0.05 * rng.standard_normal(c.shape), 0, 1)
    p = H.hydrostatic_guess(g, ph) + 30 * rng.standard_normal(c.shape)
    J = H.jacobian(g, ph, f, p, c, c_old).toarray()
    for col in rng.choice(2 * g.nx * g.ny, size=40, replace=False):
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
        Rp1, Rc1 = H.residual(g, ph, f, pp, cp, c_old)
        Rp0, Rc0 = H.residual(g, ph, f, pm, cm, c_old)
        fd = H.interleave((Rp1 - Rp0) / (2 * h), (Rc1 - Rc0) / (2 * h))
        scale = np.max(np.abs(J[:, col]))
        assert np.max(np.abs(fd - J[:, col])) <= 1e-6 * scale


def test_implicit_euler_first_order_in_time():
    """Against the continuum decay exp(-D (pi/2)^2 t) of the x-mode, halving
    h and tau together halves the error (order 1, section 2.3, Eq. 1st_ord_conv)."""
    ph = H.Physics(rho1=1000.0, q0=0.0)
    T = 6 * 3600.0
    errs = []
    for k in range(3):
        g = _grid(16 << k, 2, 4 << k, T)
        x, y = H.cell_centres(g, ph)
        X, _ = np.meshgrid(x, y)
        c0 = X / 2 + 0.5 * np.sin(np.pi * X / 2)
        r = H.solve(g, ph, np.array([0.0, 0.0, 0.0]), c0=c0)
        exact = X / 2 + 0.5 * np.sin(np.pi * X / 2) * math.exp(-ph.D * (math.pi / 2) ** 2 * T)
        errs.append(np.max(np.abs(r["c"] - exact)))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    for q in ratios:
        assert 1.8 < q < 2.2, ratios


def test_observation_points_are_the_papers_points_3_9_15():
    """Eq. 12points lists x_3=(1.40,-0.95), x_9=(1.65,-0.75), x_15=(1.90,-0.50)
    in the paper's frame y in [-1, 0]."""
    paper = [(1.40, -0.95), (1.65, -0.75), (1.90, -0.50)]
    assert [(x, round(y - 1.0, 12) + 0.0) for x, y in H.OBS_POINTS] == \
        [(x, y) for x, y in paper] or all(
            abs(a[0] - b[0]) < 1e-12 and abs(a[1] - 1.0 - b[1]) < 1e-12
            for a, b in zip(H.OBS_POINTS, paper))


def test_point_value_is_exact_for_bilinear_fields():
    ph = H.Physics()
    g = _grid(32, 16, 1, 1.0)
    x, y = H.cell_centres(g, ph)
    X, Y = np.meshgrid(x, y)
    c = 0.2 + 0.3 * X - 0.7 * Y + 0.11 * X * Y
    for px, py in H.OBS_POINTS + ((0.5, 0.5),):
        assert abs(H.point_value(g, ph, c, px, py) - (0.2 + 0.3 * px - 0.7 * py + 0.11 * px * py)) < 1e-13


def test_qoi_integrals_of_known_fields():
    ph = H.Physics()
    g = _grid(32, 16, 1, 1.0)
    f = H.fields(g, ph, np.zeros(3))
    c = np.ones((g.ny, g.nx))
    q = H.qoi(g, ph, f, c)
    area = ph.Lx * ph.Ly
    assert abs(q[0] - ph.rho1 * area) < 1e-9               # int c rho
    assert abs(q[1] - ph.phi0 * ph.rho1 * area) < 1e-9     # int phi rho c
    assert abs(q[2] - ph.Ly * ph.Lx ** 2 / 2) < 1e-12       # int (Lx - x)


def test_allocation_reproduces_the_papers_table():
    with open(os.path.join(GOLDEN, "allocation_table.json")) as fh:
        tab = json.load(fh)
    for eps2, row in tab["rows"].items():
        m = M.allocation(tab["V"], tab["s"], math.sqrt(float(eps2)), var_budget_fraction=1.0)
        assert list(m) == row, (eps2, list(m), row)


def test_allocation_meets_variance_budget_at_minimal_cost():
    """With real-valued m_l from Eq. M_ell, Var Y = eps^2/2 exactly and the
    cost equals Eq. total_cost_MLMC; any other split of the same variance
    costs more (Lagrange optimality, Eq. zero_deriv)."""
    rng = np.random.default_rng(0)
    V = rng.random(5) * 1e-3
    s = 2.0 ** (3 * np.arange(5)) * (1 + rng.random(5))
    eps = 1e-2
    tot = np.sum(np.sqrt(V * s))
    m = 2 / eps**2 * np.sqrt(V / s) * tot
    assert abs(np.sum(V / m) - eps**2 / 2) < 1e-12 * eps**2
    assert abs(np.sum(m * s) - M.optimal_cost(V, s, eps)) < 1e-9 * np.sum(m * s)
    for _ in range(20):
        w = m * np.exp(0.3 * rng.standard_normal(5))
        w *= np.sum(V / w) / (eps**2 / 2)      # rescale to the same variance
        assert np.sum(w * s) >= np.sum(m * s) * (1 - 1e-12)


def test_cost_theorem_exponents_match_test_b4():
    with open(os.path.join(GOLDEN, "cost_theorem.json")) as fh:
        t = json.load(fh)
    e = M.cost_exponent(t["alpha"], t["beta"], t["gamma"], t["d_hat"])
    assert round(e, 2) == t["mlmc_exponent_printed"]
    mc = 2 + t["d_hat"] * t["gamma"] / t["alpha"]
    assert round(mc, 1) == t["mc_exponent_printed"]


def test_two_pass_statistics_closed_form():
    """Samples 1..n: mean (n+1)/2, unbiased variance n(n+1)/12."""
    n = 101
    a = np.arange(1, n + 1, dtype=float)[:, None] * np.array([[1.0, -2.0]])
    st = M.level_stats(a)
    assert np.allclose(st["mean_f"], [(n + 1) / 2, -(n + 1)], rtol=0, atol=1e-12)
    assert np.allclose(st["var_f"], [n * (n + 1) / 12, 4 * n * (n + 1) / 12], rtol=1e-14)
    st2 = M.level_stats(a, a - 1.0)
    assert np.allclose(st2["mean_d"], 1.0) and np.allclose(st2["var_d"], 0.0, atol=1e-20)


def test_telescoping_sum_equals_finest_level_mean():
    """Eq. EgL with the same samples on every level: the sum of level-mean
    differences telescopes to the finest level's mean."""
    rng = np.random.default_rng(1)
    g = [rng.random((64, 3)) for _ in range(4)]
    means = [g[0].mean(0)] + [(g[l] - g[l - 1]).mean(0) for l in range(1, 4)]
    Y, _ = M.estimator(means, np.zeros((4, 3)), np.ones(4))
    assert np.allclose(Y, g[3].mean(0), atol=1e-14)


def test_fit_rate_recovers_geometric_decay():
    lev = np.arange(4)
    vals = 3.0 * 2.0 ** (-1.7 * lev)
    rate, zeta = M.fit_rate(lev, vals, base=2.0)
    assert abs(rate - 1.7) < 1e-12 and abs(zeta - math.log2(3.0)) < 1e-12


def test_grid_convergence_order_of_the_coupled_problem():
    """Observed convergence of the full density-driven problem (section 2.3,
    first order in h and tau together): on levels 0, 1, 2 with tau halved
    with h (4, 8, 16 steps of 1800/2^l s) and one xi, the distance between
    successive levels, || c_l - R c_{l+1} ||_2 with R the average over the
    four children, shrinks by about 2 per level. A wrong scaling of a flux
    or of the accumulation with h or tau stops the differences from
    decaying like this."""
    ph = H.Physics()
    xi = np.array([0.3, -0.5, 0.7])
    cs = []
    for level in range(3):
        g = _grid(32 << level, 16 << level, 4 << level, 4 * 1800.0)
        cs.append(H.solve(g, ph, xi)["c"])

    def R(c):
        return 0.25 * (c[0::2, 0::2] + c[1::2, 0::2] + c[0::2, 1::2] + c[1::2, 1::2])

    d = [math.sqrt(np.mean((cs[l] - R(cs[l + 1])) ** 2)) for l in range(2)]
    assert 1.5 < d[0] / d[1] < 2.5, d
    # and P0-prolongated coarse minus fine shrinks too (the MLMC field
    # correction of the level pairs tends to zero)
    P0 = [H.prolong_constant(cs[l]) - cs[l + 1] for l in range(2)]
    assert math.sqrt(np.mean(P0[1] ** 2)) < math.sqrt(np.mean(P0[0] ** 2))


@pytest.mark.parametrize("a,eps,E0", [(0.3, 1e-3, 1.0), (0.05, 2e-3, 0.52), (2.0, 1e-2, 336.0)])
def test_num_levels_is_the_smallest_level_meeting_the_bias_bound(a, eps, E0):
    """Eq. num_levels with the weak-error model of Eq. weak_error_model: for
    corrections E Y_l = a 2^-l (first order in h, the paper's alpha = 1/2 in
    its log_4 convention) the bias of level L is the tail sum over the finer
    corrections, a 2^-L. The fitted (alpha, c1) and the chosen L must agree
    with that tail, summed term by term, and with the smallest L meeting
    |bias| <= eps E0 / sqrt(2), found by brute force."""
    levels = [1, 2, 3, 4]
    alpha, c1 = M.weak_error_constants(levels, [a * 2.0 ** -l for l in levels])
    assert abs(alpha - 0.5) < 1e-12
    for L in (0, 3, 7):
        tail = sum(a * 2.0 ** -k for k in range(L + 1, L + 200))
        assert abs(c1 * 4.0 ** (-alpha * L) - tail) <= 1e-12 * tail
    brute = next(L for L in range(200)
                 if sum(a * 2.0 ** -k for k in range(L + 1, L + 200)) <= eps * E0 / math.sqrt(2.0))
    assert M.num_levels(eps, E0, c1, alpha) == brute


# ---------------------------------------------------------------------------
# the paper's own workload: Eq. poro_2levels, Eq. e_perm_Kozeny_Carman,
# Eq. e_recharge_of_param, Eqs. integral_fw and integral_box
# ---------------------------------------------------------------------------
def test_kozeny_carman_scaling_is_table_1s():
    """Table 1 lists kappa_KC = 2.088415e-8 m^2 beside K0 = 1.020408e-9 and
    phi0 = 0.35: the Kozeny-Carman law through the mean porosity gives K0."""
    ph = H.Physics(field_model=1)
    assert ph.kappa_kc == pytest.approx(2.088415e-8, rel=5e-7)


def test_paper_porosity_layers_at_xi_zero():
    """xi = 0: C1 = C2 = 1, so phi = 0.35 above y_p = -0.8 and 0.35 * 1.2 in
    the lower layer (y < 0.2 in this frame), and K = K0 where phi = phi0."""
    ph = H.Physics(field_model=1)
    g = _grid(40, 20, 1, 1.0)
    f = H.fields(g, ph, np.zeros(3))
    _, y = H.cell_centres(g, ph)
    low = y < 0.2
    assert np.allclose(f.phi[low], 0.42, rtol=1e-15) and np.allclose(f.phi[~low], 0.35, rtol=1e-15)
    assert np.allclose(f.K[~low], ph.K0, rtol=1e-14)
    assert np.allclose(f.qin, ph.q0, rtol=1e-15)
    f3 = H.fields(g, ph, np.array([0.0, 0.0, 1.0]))
    assert np.allclose(f3.qin, 1.5 * ph.q0, rtol=1e-15)


def _unit_dft(v, axis):
    """DFT over the last (or given) axis scaled so that a sampled
    cos(2 pi k s) at s_i = (i + 1/2) / N has coefficient exp(i pi k / N) at
    bin k (and sin(2 pi k s) the coefficient -i exp(i pi k / N)): the
    half-cell phase is removed, so a cosine term reads as a real number and
    a sine term as an imaginary one."""
    N = v.shape[axis]
    X = np.fft.fft(v, axis=axis) / (N / 2)
    k = np.arange(N)
    shape = [1] * v.ndim
    shape[axis] = N
    return X * np.exp(-1j * np.pi * k / N).reshape(shape)


def test_paper_porosity_layer_factor_c0():
    """Eq. poro_2levels_C: with xi2 = 0 the oscillating factors C1, C2
    depend on x only and average to one over a period (cos 2 pi x, sin 64 pi x
    and their product are orthogonal to the constant on [0, 1), also on the
    midpoint grid), so the x-average of each row over [0, 1) is
    0.35 C0(xi1): 0.35 * 1.2 (1 + 0.2 xi1) below y_p = -0.8 (y < 0.2 in this
    frame) and 0.35 above. A flipped sign, a swapped layer test or the
    commented draft's threshold (-0.75) fails."""
    ph = H.Physics(field_model=1)
    g = _grid(256, 40, 1, 1.0)              # 128 cells per metre, rows every 0.025 m
    _, y = H.cell_centres(g, ph)
    for a in (0.7, -0.45):
        f = H.fields(g, ph, np.array([a, 0.0, 0.3]))
        mean = f.phi[:, :128].mean(axis=1)
        want = np.where(y < 0.2, 0.35 * 1.2 * (1.0 + 0.2 * a), 0.35)
        assert np.allclose(mean, want, rtol=1e-14, atol=0)


def test_paper_porosity_x_spectrum_of_the_xi1_terms():
    """Eq. poro_2levels with xi = (a, 0, 0): phi / (0.35 C0) = (1 + 0.15 a
    cos 2 pi x)(1 + 0.2 a sin 64 pi x), independent of y inside a layer and
    of period 1 in x. Its spectrum over one period has exactly five lines:
    1 (bin 0); 0.15 a, a cosine at 1 cycle/m; 0.2 a, a sine at 32 cycles/m;
    and the product 0.03 a^2 cos 2 pi x sin 64 pi x = 0.015 a^2 (sin 62 pi x
    + sin 66 pi x), sines at 31 and 33 cycles/m. A swapped coordinate, a
    wrong frequency, a sine for a cosine or a flipped sign fails."""
    ph = H.Physics(field_model=1)
    g = _grid(256, 40, 1, 1.0)
    _, y = H.cell_centres(g, ph)
    a = 0.8
    f = H.fields(g, ph, np.array([a, 0.0, 0.0]))
    C0 = np.where(y < 0.2, 1.2 * (1.0 + 0.2 * a), 1.0)
    r = f.phi / (0.35 * C0[:, None])
    assert np.allclose(r, r[:1], rtol=1e-15, atol=0)                     # no y dependence
    assert np.allclose(r[:, :128], r[:, 128:], rtol=1e-14, atol=0)       # period 1 in x
    X = _unit_dft(r[0, :128], axis=0)
    want = np.zeros(128, dtype=complex)
    want[0] = 2.0                      # the constant 1 (bin 0 counts it twice)
    want[1] = 0.15 * a
    want[32] = -1j * 0.2 * a
    want[31] = want[33] = -1j * 0.015 * a * a
    assert np.allclose(X[:64], want[:64], rtol=0, atol=1e-13)


def test_paper_porosity_y_spectrum_of_the_xi2_terms():
    """Eq. poro_2levels with xi = (0, b, 0): C0 does not depend on xi, so
    phi(xi) / phi(0) = C1 C2 = (1 + 0.15 b (cos(pi x/2) - sin 2 pi y_p))
    (1 + 0.2 b sin 32 pi y_p), y_p = y - 1. Over y in [0, 1) at a column x
    the spectrum has exactly: bin 0, 1 + 0.15 b cos(pi x/2); a sine at 1
    cycle/m with coefficient -0.15 b; a sine at 16 cycles/m with coefficient
    0.2 b (1 + 0.15 b cos(pi x/2)); and the product -0.03 b^2 sin 2 pi y sin
    32 pi y = -0.015 b^2 (cos 30 pi y - cos 34 pi y), cosines at 15 and 17
    cycles/m. The columns x and 2 - x differ only in the sign of cos(pi x/2)."""
    ph = H.Physics(field_model=1)
    g = _grid(20, 128, 1, 1.0)
    x, _ = H.cell_centres(g, ph)
    b = -0.6
    r = H.fields(g, ph, np.array([0.0, b, 0.0])).phi / H.fields(g, ph, np.zeros(3)).phi
    X = _unit_dft(r, axis=0)                       # [bin, column]
    for i in range(g.nx):
        cx = np.cos(np.pi * x[i] / 2)
        want = np.zeros(64, dtype=complex)
        want[0] = 2.0 * (1.0 + 0.15 * b * cx)
        want[1] = -1j * (-0.15 * b)
        want[16] = -1j * 0.2 * b * (1.0 + 0.15 * b * cx)
        want[15] = -0.015 * b * b
        want[17] = 0.015 * b * b
        assert np.allclose(X[:64, i], want, rtol=0, atol=1e-13), i
    # mirror columns: the sum removes the cos(pi x/2) term
    s = r + r[:, ::-1]
    assert np.allclose(s, s[:, :1], rtol=1e-14, atol=0)


def test_box_integrals_and_fresh_water_area_of_known_fields():
    """c = 1: Q_i = rho1 |Delta_i in D| (0.2 x 0.15 for the five boxes cut
    by y = 0, 0.04 otherwise), Q_FW = 0. c = 1 above y = 0.5 only: the boxes
    around y_p = -0.5 are half full, the others empty, Q_FW = 1. c = 1 left
    of x = 1 only: the boxes at x = 0.9 are full, at x = 1.15 empty."""
    ph = H.Physics(field_model=1)
    g = _grid(64, 32, 1, 1.0)
    f = H.fields(g, ph, np.zeros(3))
    x, y = H.cell_centres(g, ph)
    X, Y = np.meshgrid(x, y)
    q = H.qoi(g, ph, f, np.ones((32, 64)))
    area = np.array([0.03] * 5 + [0.04] * 10)
    assert np.allclose(q[7:22], ph.rho1 * area, rtol=1e-13) and q[6] == 0.0
    q = H.qoi(g, ph, f, (Y > 0.5).astype(float))
    assert np.allclose(q[7:17], 0.0) and np.allclose(q[17:22], ph.rho1 * 0.02, rtol=1e-13)
    assert q[6] == pytest.approx(1.0, rel=1e-14)
    q = H.qoi(g, ph, f, (X < 1.0).astype(float))
    assert np.allclose(q[[7, 12, 17]], ph.rho1 * area[[0, 5, 10]], rtol=1e-13)
    assert np.allclose(q[[8, 13, 18]], 0.0)
    # threshold of Eq. integral_fw: c <= 0.012178 counts as fresh water
    assert H.qoi(g, ph, f, np.full((32, 64), 0.012178))[6] == pytest.approx(2.0, rel=1e-14)
    assert H.qoi(g, ph, f, np.full((32, 64), 0.0122))[6] == 0.0


def test_recharge_enters_at_the_new_time_level():
    """With rho1 = rho0 the fluid is incompressible and decoupled from c, so
    after every implicit step the outflow through the seaward side equals
    the inflow of that step: rho0 Ly q0 (1 + 0.5 xi3)(1 + sin(pi t^(n+1) / 40))
    (Eq. e_recharge_of_param at the end of the step, as implicit Euler
    takes boundary data)."""
    ph = H.Physics(field_model=1, rho1=1000.0)
    g = _grid(16, 8, 5, 5 * 13.0)
    xi = np.array([0.3, -0.4, 0.6])
    r = H.solve(g, ph, xi, keep_states=True)
    f = r["fields"]
    for n in range(1, 6):
        p, c = r["states"][n]
        F = H.face_fluxes(g, ph, f, p, c)
        out = np.sum(F["mass_right"])
        want = ph.rho0 * ph.Ly * ph.q0 * (1 + 0.5 * xi[2]) * (1 + math.sin(math.pi * n * 13.0 / 40))
        assert out == pytest.approx(want, rel=1e-10)
